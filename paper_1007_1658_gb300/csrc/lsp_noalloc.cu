// lsp_noalloc.cu -- a periodogram entry point that allocates no memory.
//
// Some callers of this library cannot allocate device memory at call time:
// an application whose memory pool already owns the whole device, or a
// latency-critical loop where cudaMalloc's device-wide synchronization and
// unbounded latency are not acceptable.  For them this file keeps the
// periodogram's scratch (phase records, per-chunk partial sums, per-curve
// statistics) in one file-scope device array of fixed size.  Every GPU that
// loads the library holds that array until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "lsp_ctx.h"

namespace {

constexpr size_t kHeaderBytes = 8192;  // CurveStats, status word, slice counter, slice statistics
constexpr int64_t kMaxSamples = int64_t(1) << 19;      // 524,288 samples
constexpr size_t kRecordBytes = size_t(kMaxSamples) * 32;      // 16 MiB of phase records
constexpr size_t kPartialBytes = size_t(48) << 20;             // 48 MiB of partial sums
constexpr size_t kScratchBytes = kHeaderBytes + kRecordBytes + kPartialBytes;  // 64 MiB + 8 KiB

// Host code sees this name only as a host-side stand-in; the device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of g_scratch on `dev` (which must be current); looked up on
// the first call for that device and cached.
cudaError_t scratch_for(int dev, unsigned char** out, int* sms) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
        g_sms[dev] = n;
    }
    *out = (unsigned char*)g_scratch_dev[dev];
    *sms = g_sms[dev];
    return cudaSuccess;
}

// Device memory of `dev` or managed memory; host memory and device memory of
// another GPU are refused.
bool on_device(const void* p, int dev) { return lsp::host::pointer_kind_of(p, dev) == lsp::host::kPtrDevice; }

// Moves the grid origin of the phase records by dk frequencies: v += dk u
// (mod 2^64), the same exact integer step the main kernel takes for its own
// k, so the next frequency tile starts at bin k_b + dk with an exact phase.
__global__ void __launch_bounds__(256) shift_origin_kernel(uint4* __restrict__ recA, int64_t n, uint32_t dk) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        uint4 a = recA[j];
        const uint64_t u = ((uint64_t)a.y << 32) | a.x;
        const uint64_t v = (((uint64_t)a.w << 32) | a.z) + (uint64_t)dk * u;
        a.z = (uint32_t)v;
        a.w = (uint32_t)(v >> 32);
        recA[j] = a;
    }
}

}  // namespace

extern "C" lsp_status lsp_periodogram_noalloc(const double* t, const double* X, int64_t N_t, double f_0,
                                              double df, int64_t N_f, float* P_out, void* cuda_stream) {
    if (N_t < 2 || N_t > kMaxSamples) return LSP_ERR_INVALID_ARG;
    if (N_f < 0 || N_f >= (int64_t(1) << 31)) return LSP_ERR_INVALID_ARG;
    if (!std::isfinite(f_0) || !std::isfinite(df)) return LSP_ERR_NONFINITE;
    if (N_f == 0) return LSP_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LSP_ERR_CUDA;
    }
    if (!t || !X || !P_out || !on_device(t, dev) || !on_device(X, dev) || !on_device(P_out, dev))
        return LSP_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    int sms = 0;
    if (scratch_for(dev, &base, &sms) != cudaSuccess) {
        cudaGetLastError();
        return LSP_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    lsp::CurveStats* stats = (lsp::CurveStats*)base;
    int* status = (int*)(base + sizeof(lsp::CurveStats));
    unsigned* counter = (unsigned*)(base + sizeof(lsp::CurveStats) + 8);
    lsp::StatPart* sparts = (lsp::StatPart*)(base + 256);
    static_assert(256 + sizeof(lsp::StatPart) * lsp::kMaxStatSlices <= kHeaderBytes, "header too small");
    uint4* recA = (uint4*)(base + kHeaderBytes);
    float4* recB = (float4*)(base + kHeaderBytes + size_t(kMaxSamples) * 16);
    float* part = (float*)(base + kHeaderBytes + kRecordBytes);

    // Launch shape of the default (packed three-term recurrence) path: strips of 24
    // frequencies, and an N_t split with chunks of at most kMaxChunk samples
    // (the bound on the FP32 running sums that lsp_periodogram keeps), more
    // where that fills the SMs.  The partial sums of `need` chunks fit the
    // array for a limited number of frequencies, so the grid is evaluated in
    // frequency tiles of at most that many bins, each a main launch and a
    // finalize, with the records' phase origin moved exactly between tiles.
    const int F = 24;
    const int64_t per_block = lsp::freqs_per_block(F);
    const int64_t need = (N_t + lsp::kMaxChunk - 1) / lsp::kMaxChunk;
    const size_t row_bytes = size_t(4) * 4;  // four FP32 sums per (chunk, frequency)
    int64_t tile = N_f;
    if (need > 1) {
        const int64_t blocks = (int64_t)(kPartialBytes / (row_bytes * (size_t)need * (size_t)per_block));
        tile = std::min<int64_t>(N_f, blocks * per_block);
    }
    const int occ = lsp::main_occupancy(lsp::kModeRecur3x2, F);
    const int64_t slots = (int64_t)occ * (sms > 0 ? sms : 1);

    // the shared array keeps the last call's contents: clear the status word
    // and the slice counter, which must start at zero
    cudaError_t e = cudaMemsetAsync(status, 0, 16, st);
    if (e == cudaSuccess) e = lsp::launch_prep_stats(t, X, nullptr, N_t, 1, stats, status, sparts, counter, st);
    if (e == cudaSuccess)
        e = lsp::launch_prep_records(t, X, nullptr, N_t, 1, N_t, nullptr, nullptr, f_0, df, stats, recA, recB,
                                     nullptr, nullptr, st, nullptr, nullptr, status);
    for (int64_t kb = 0; kb < N_f && e == cudaSuccess; kb += tile) {
        const int64_t nf = std::min<int64_t>(tile, N_f - kb);
        if (kb > 0) {
            const int64_t g = std::min<int64_t>((N_t + 255) / 256, 4096);
            shift_origin_kernel<<<(unsigned)g, 256, 0, st>>>(recA, N_t, (uint32_t)tile);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
        }
        lsp::MainShape s{};
        s.mode = lsp::kModeRecur3x2;
        s.F = F;
        s.nfb = (int)((nf + per_block - 1) / per_block);
        s.nf_pad = (int64_t)s.nfb * per_block;
        const int64_t fit = (int64_t)(kPartialBytes / (row_bytes * (size_t)s.nf_pad));
        int64_t split = (slots + s.nfb - 1) / s.nfb;
        split = std::min<int64_t>(split, std::max<int64_t>(1, N_t / lsp::kMinChunk));
        split = std::min<int64_t>(split, fit);
        split = std::max<int64_t>(split, need);  // need <= fit by the choice of the tile
        if (split < 2) split = 1;
        s.chunk = (N_t + split - 1) / split;
        s.split = (int)((N_t + s.chunk - 1) / s.chunk);
        e = lsp::launch_main(s, recA, recB, nullptr, N_t, nf, f_0, df, part, P_out + kb, st);
        if (e == cudaSuccess && s.split > 1) e = lsp::launch_finalize(s, part, N_t, nf, P_out + kb, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LSP_ERR_CUDA;
    }
    return LSP_OK;
}
