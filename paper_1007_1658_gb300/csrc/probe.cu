// probe.cu -- lsp_probe_pipes: per-SM, per-clock rates of the operations the
// periodogram kernels are built from, measured on the part at hand.  Sec. 5.3
// explains the GPU's lead by the throughput of its hardware sin/cos units; the
// kernels here have three bounds of that kind, and these rates are their
// denominators: the MUFU path issues 2 SFU ops (one sin/cos pair) per term,
// the recurrences 8 (RECUR) or 6 (RECUR3) FP32 FMA-pipe ops, and the packed
// form FP32x2 FMA.
//
// Each probe kernel runs kChains independent dependency chains per thread for
// `iters` iterations in kProbeCtas CTAs of kProbeThreads threads per SM,
// brackets the loop with clock64 and stores its cycle count; a rate is the
// operations of the launch / (SMs x the slowest CTA's cycles).  The SM clock
// follows from those cycles and the launch's CUDA-event time.
#include <algorithm>
#include <vector>

#include "lsp_ctx.h"

namespace lsp {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtas = 4;  // per SM: 32 resident warps
constexpr int kProbeIters = 8192;

enum ProbeKind { kProbeSincos = 0, kProbeFfma = 1, kProbeFfma2 = 2 };

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads)
probe_kernel(float* __restrict__ sink, long long* __restrict__ cycles, int iters, float a, float b) {
    float v[kChains];
    float2 p[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        v[i] = (float)threadIdx.x * 1e-3f + (float)i * 0.1f;
        p[i] = make_float2(v[i], -v[i]);
    }
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (KIND == kProbeSincos) {
                float s, c;
                __sincosf(v[i], &s, &c);
                v[i] = s + c;  // stays in [-sqrt 2, sqrt 2]
            } else if (KIND == kProbeFfma) {
                v[i] = fmaf(v[i], a, b);
            } else {
                p[i] = __ffma2_rn(p[i], a2, b2);
            }
        }
    }
    const long long t1 = clock64();
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += v[i] + p[i].x + p[i].y;
    // never true for these inputs; keeps every chain's result live
    if (acc == 1234.5f) sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

using ProbeFn = void (*)(float*, long long*, int, float, float);

}  // namespace
}  // namespace lsp

using lsp::host::fail;

extern "C" lsp_status lsp_probe_pipes(lsp_ctx* ctx, lsp_pipe_rates* out) {
    if (!ctx || !out) return fail(ctx, LSP_ERR_INVALID_ARG, "ctx and out must be non-NULL");
    lsp::host::DeviceGuard guard(ctx->device);
    std::memset(out, 0, sizeof *out);
    const int sms = std::max(1, ctx->sms);
    const int blocks = sms * lsp::kProbeCtas;
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lsp_status rs = LSP_OK;
    std::vector<long long> hc((size_t)blocks);
    const lsp::ProbeFn fns[3] = {lsp::probe_kernel<lsp::kProbeSincos>, lsp::probe_kernel<lsp::kProbeFfma>,
                                 lsp::probe_kernel<lsp::kProbeFfma2>};
    double rate[3] = {0.0, 0.0, 0.0}, mhz = 0.0;
    cudaError_t e = cudaMalloc(&sink, (size_t)blocks * lsp::kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        // one untimed launch, then the timed one
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            if (rep == 1) e = cudaEventRecord(e0, ctx->stream);
            if (e == cudaSuccess) {
                fns[k]<<<blocks, lsp::kProbeThreads, 0, ctx->stream>>>(sink, cyc, lsp::kProbeIters, 0.999f, 1e-3f);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e1, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, hc.size() * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            const long long mx = *std::max_element(hc.begin(), hc.end());
            const double ops = (double)blocks * lsp::kProbeThreads * lsp::kProbeIters * lsp::kChains *
                               (k == lsp::kProbeFfma2 ? 2.0 : 1.0);
            rate[k] = mx > 0 ? ops / ((double)sms * (double)mx) : 0.0;
            if (k == lsp::kProbeFfma && ms > 0.f) mhz = (double)mx / ((double)ms * 1e3);
        }
    }
    if (e != cudaSuccess) rs = lsp::host::cuda_fail(ctx, e, "pipe-rate probe");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cyc) cudaFree(cyc);
    if (sink) cudaFree(sink);
    if (rs != LSP_OK) {
        cudaGetLastError();
        return rs;
    }
    out->sms = sms;
    out->sm_mhz = mhz;
    out->sincos_per_clk_sm = rate[lsp::kProbeSincos];
    out->ffma_per_clk_sm = rate[lsp::kProbeFfma];
    out->ffma2_lanes_per_clk_sm = rate[lsp::kProbeFfma2];
    return LSP_OK;
}
