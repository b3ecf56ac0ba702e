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

#include "lsp.h"
#include "lsp_kernels.cuh"

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

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" lsp_status lsp_periodogram_noalloc(const double* t, const double* X, int64_t N_t, double f_0,
                                              double df, int64_t N_f, float* P_out, void* cuda_stream) {
    if (N_t < 2 || N_t > kMaxSamples) return LSP_ERR_INVALID_ARG;
    if (N_f < 0 || N_f >= (int64_t(1) << 31)) return LSP_ERR_INVALID_ARG;
    if (!std::isfinite(f_0) || !std::isfinite(df)) return LSP_ERR_NONFINITE;
    if (N_f == 0) return LSP_OK;
    if (!t || !X || !P_out || !on_device(t) || !on_device(X) || !on_device(P_out)) return LSP_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LSP_ERR_CUDA;
    }
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

    // Launch shape of the default (three-term recurrence) path: strips of 24
    // frequencies; the N_t split fills the SMs and keeps chunks within
    // kMaxChunk samples, but never needs more partial sums than fit.
    lsp::MainShape s{};
    s.mode = lsp::kModeRecur3;
    s.F = 24;
    const int64_t per_block = lsp::freqs_per_block(s.F);
    s.nfb = (int)((N_f + per_block - 1) / per_block);
    s.nf_pad = (int64_t)s.nfb * per_block;
    const int64_t fit = (int64_t)(kPartialBytes / (size_t(4) * 4 * (size_t)s.nf_pad));
    const int occ = lsp::main_occupancy(s.mode, s.F);
    const int64_t slots = (int64_t)occ * (sms > 0 ? sms : 1);
    int64_t split = (slots + s.nfb - 1) / s.nfb;
    split = std::min<int64_t>(split, std::max<int64_t>(1, N_t / lsp::kMinChunk));
    split = std::max<int64_t>(split, (N_t + lsp::kMaxChunk - 1) / lsp::kMaxChunk);
    split = std::min<int64_t>(split, fit);
    if (split < 2) split = 1;
    s.chunk = (N_t + split - 1) / split;
    s.split = (int)((N_t + s.chunk - 1) / s.chunk);

    // the shared array keeps the last call's contents: clear the status word
    // and the slice counter, which must start at zero
    cudaError_t e = cudaMemsetAsync(status, 0, 16, st);
    if (e == cudaSuccess) e = lsp::launch_prep_stats(t, X, nullptr, N_t, 1, stats, status, sparts, counter, st);
    if (e == cudaSuccess)
        e = lsp::launch_prep_records(t, X, nullptr, N_t, 1, N_t, nullptr, nullptr, f_0, df, stats, recA, recB,
                                     nullptr, nullptr, st);
    if (e == cudaSuccess) e = lsp::launch_main(s, recA, recB, nullptr, N_t, N_f, f_0, df, part, P_out, st);
    if (e == cudaSuccess && s.split > 1) e = lsp::launch_finalize(s, part, N_t, N_f, P_out, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LSP_ERR_CUDA;
    }
    return LSP_OK;
}
