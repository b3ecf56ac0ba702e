// lsp_ctx.h -- the context structure and host-side helpers shared by the
// C-ABI implementation files (lsp_api.cu, lsp_batch_api.cu).  Internal.
#pragma once

#include <cstdarg>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lsp.h"
#include "lsp_kernels.cuh"

namespace lsp {
namespace host {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Cached plan of the last lsp_batch call: the host copy of its metadata, the
// sorted work list and the instantiated CUDA graph that replays the whole
// batch (prep, noise, persistent kernel, max unpack) in one launch.
struct BatchPlan {
    bool valid = false;
    std::vector<const void*> ptrs;          // every pointer argument of the call
    int n_curves = 0, n_real = 0, mode = 0, F = 0, R = 1, tailF = 0, tile = 0;
    bool noise = false;
    std::vector<int64_t> t_off, nf, p_off;
    std::vector<double> f0, df;
    int n_items = 0, grid = 0;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
};

// One autotuned choice for a (log2 N_t, log2 N_f) size bucket.
struct TuneEntry {
    int nt_bucket, nf_bucket;
    int sincos, F, split;
    float ms;
};

// Launch shape of lsp_batch: kernel mode (kMode*), strip length, realizations
// per pass, tail-strip length (0: none) and samples per shared-memory tile.
struct BatchShape {
    int mode, F, R, tailF, tile;
};

// Size bucket of a batch: log2 of its terms per realization, log2 of its
// mean samples per curve, and its realization count (1, 2-3, 4-7, 8+).
struct BatchBucket {
    int terms, mean_nt, real;
    bool operator==(const BatchBucket& o) const {
        return terms == o.terms && mean_nt == o.mean_nt && real == o.real;
    }
};

// One lsp_autotune_batch choice.
struct BatchTuneEntry {
    BatchBucket bucket;
    BatchShape shape;
    float ms;
};

// State of the false-alarm surrogate's network (lsp_fap_*).
struct FapState {
    bool ready = false;
    int H = 0;
    int64_t n_params = 0;
    int64_t step = 0;
    DevBuf params, grad, m, v, mu_sig, ws, act, X, cnt, y, loss, q, rows, W, W_off, nw, counts;
    DevBuf best, train_state, hist;  // lsp_fap_train: kept weights, loop scalars, histories
};

}  // namespace host
}  // namespace lsp

struct lsp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream that batch graphs are captured on
    lsp_options opt{};
    std::string err;
    int sms = 0;
    // single-curve workspace
    lsp::host::DevBuf recA, recB, recN, part, stats, t_stage, x_stage, p_stage, stat_parts, stat_counters;
    lsp::host::DevBuf recQ, dy_stage;  // floating-mean periodogram: sqrt(w_j), staged errors
    lsp::host::DevBuf pr_acc, pr_z0, pr_z1;  // Press-Rybicki: FP64 grid, FFT ping-pong buffers
    // batch workspace
    lsp::host::DevBuf b_recA, b_recB, b_xr, b_stats, b_items, b_head, b_maxkey, b_seed, b_off, b_nf, b_f0,
        b_df, b_poff, b_t, b_X, b_P, b_maxP, b_argmax,
        b_win, b_woff,  // multi-realization window sums (CC, CS) per frequency and their per-curve offsets
        b_gx;           // floating-mean Monte Carlo: x of every realization
    void* pinned = nullptr;  // host staging for the work list and small values
    size_t pinned_cap = 0;
    lsp::host::BatchPlan plan;
    lsp::host::FapState fap;
    std::vector<lsp::host::TuneEntry> tune;  // lsp_autotune results, used by AUTO
    std::vector<lsp::host::BatchTuneEntry> tune_batch;  // lsp_autotune_batch results, used by AUTO
    int* status_d = nullptr;  // device status word (OR of kStatus* bits)
    int* status_h = nullptr;  // pinned mirror
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t done = nullptr;
    bool timing_valid = false;
    bool has_finalize = false;
    int last_launches = 0;
    int fail_alloc_in = 0;  // test hook: the n-th workspace allocation from now fails (0: never)
};

namespace lsp {
namespace host {

// An NVTX range named for a stage of a call (prep, main, finalize, batch),
// open for the scope of the host code that enqueues it, so that a profiler's
// timeline can tie kernels to the library's stages.  Costs a few nanoseconds
// when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes the context's device current for the scope of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline lsp_status fail(lsp_ctx* ctx, lsp_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

inline lsp_status cuda_fail(lsp_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? LSP_ERR_OOM : LSP_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define LSP_CUDA(ctx, call)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return lsp::host::cuda_fail(ctx, e_, #call); \
    } while (0)

// Grow a workspace buffer to at least `bytes` (contents are not kept).
inline lsp_status ensure(lsp_ctx* ctx, DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return LSP_OK;
    if (b.p) {
        LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        LSP_CUDA(ctx, cudaFree(b.p));
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    if (ctx->fail_alloc_in > 0 && --ctx->fail_alloc_in == 0)
        return fail(ctx, LSP_ERR_OOM, "cudaMalloc(workspace): allocation failure injected by lsp_test_fail_allocation");
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return cuda_fail(ctx, e, "cudaMalloc(workspace)");
    }
    b.cap = want;
    return LSP_OK;
}

// As ensure(), but a newly allocated buffer is zero-filled (for counters
// that kernels leave at zero after use).
inline lsp_status ensure_zeroed(lsp_ctx* ctx, DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return LSP_OK;
    lsp_status st = ensure(ctx, b, bytes);
    if (st != LSP_OK) return st;
    LSP_CUDA(ctx, cudaMemsetAsync(b.p, 0, b.cap, ctx->stream));
    return LSP_OK;
}

// Where a caller's array lives, decided from its CUDA pointer attributes
// (memory type and owning device): host memory (pageable, registered or
// pinned; staged through copies), device memory of the context's GPU or
// managed memory (used in place), or device memory of another GPU, which the
// library refuses: a kernel would reach it only through a peer mapping the
// caller never asked for, or fault.
enum PtrKind : int { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };

inline int pointer_kind(int memory_type, int pointer_device, int device) {
    if (memory_type == cudaMemoryTypeManaged) return kPtrDevice;
    if (memory_type == cudaMemoryTypeDevice) return pointer_device == device ? kPtrDevice : kPtrOtherDevice;
    return kPtrHost;
}

inline int pointer_kind_of(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kPtrHost;
    }
    return pointer_kind((int)a.type, a.device, device);
}

// *on_dev: the array is on the context's GPU (true) or on the host (false);
// INVALID_ARG for an array on another GPU.
inline lsp_status where(lsp_ctx* ctx, const void* p, bool* on_dev) {
    const int k = pointer_kind_of(p, ctx->device);
    if (k == kPtrOtherDevice)
        return fail(ctx, LSP_ERR_INVALID_ARG, "an array argument is device memory of another GPU (context on device %d)",
                    ctx->device);
    *on_dev = k == kPtrDevice;
    return LSP_OK;
}

// Copy n elements of a host or device array into a host vector (ordered on
// the context's stream, then waited for).
template <class T>
inline lsp_status fetch(lsp_ctx* ctx, const T* src, size_t n, std::vector<T>& dst) {
    dst.resize(n);
    if (n == 0) return LSP_OK;
    bool dev = false;
    lsp_status ws = where(ctx, src, &dev);
    if (ws != LSP_OK) return ws;
    if (dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
        LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    } else {
        std::memcpy(dst.data(), src, n * sizeof(T));
    }
    return LSP_OK;
}

// True when a batch's P layout (P_off[0..n], N_f[0..n-1]) leaves slots that
// no bin fills: before the first curve or after a curve's N_f bins.
inline bool p_layout_has_slack(const std::vector<int64_t>& poff, const std::vector<int64_t>& nf) {
    if (poff.empty() || poff[0] != 0) return true;
    for (size_t c = 0; c < nf.size(); ++c)
        if (poff[c + 1] - poff[c] != nf[c]) return true;
    return false;
}

inline lsp_status ensure_pinned(lsp_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->pinned_cap) return LSP_OK;
    if (ctx->pinned) {
        LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
        ctx->pinned_cap = 0;
    }
    const size_t want = bytes + bytes / 4 + 4096;
    LSP_CUDA(ctx, cudaMallocHost(&ctx->pinned, want));
    ctx->pinned_cap = want;
    return LSP_OK;
}

// Device view of a caller array: the array itself if it is on the device,
// else a context buffer filled from it (asynchronously, outside the graph).
template <class T>
inline lsp_status device_view(lsp_ctx* ctx, const T* src, size_t n, DevBuf& buf, const T** out) {
    bool dev = false;
    lsp_status ws = where(ctx, src, &dev);
    if (ws != LSP_OK) return ws;
    if (dev) {
        *out = src;
        return LSP_OK;
    }
    lsp_status st = ensure(ctx, buf, n * sizeof(T) + 16);
    if (st != LSP_OK) return st;
    if (n) LSP_CUDA(ctx, cudaMemcpyAsync(buf.p, src, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    *out = (const T*)buf.p;
    return LSP_OK;
}

// Kernel mode and strip length for the options, with no size-dependent choice.
void default_mode_F(const lsp_options& o, int* mode, int* F);

// Launch shape of the single-curve path for the context's options.
lsp::MainShape choose_shape(const lsp_ctx* ctx, int64_t N, int64_t N_f);

// Frequency blocks, padding and N_t split (split <= 0: the split that a model
// of waves x chunk length plus partial-sum traffic rates fastest) of a shape
// whose mode and F are already set; occ resident CTAs of `threads` per SM,
// `ops` FMA-pipe operations per term, `rows` partial sums per frequency.
void finish_shape(const lsp_ctx* ctx, lsp::MainShape& s, int occ, int64_t N, int64_t N_f, int split,
                  int threads = lsp::kMainThreads, int ops = 6, int rows = 4);

// Autotuned entry for this size bucket, or null.
const TuneEntry* tuned(const lsp_ctx* ctx, int64_t N, int64_t N_f);

// Release the cached batch graph.
void drop_plan(lsp_ctx* ctx);

BatchBucket batch_bucket(int n_curves, int64_t total_samples, int64_t total_freqs, int n_real);
// lsp_autotune_batch entry for this bucket, or null.
const BatchTuneEntry* tuned_batch(const lsp_ctx* ctx, const BatchBucket& b);

// lsp_batch with an optional forced launch shape (the autotuner's candidates).
lsp_status batch_run(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t, const double* X,
                     uint64_t seed, int32_t n_real, const double* f_0, const double* df, const int64_t* N_f,
                     float* P_out, const int64_t* P_off, float* maxP_out, int32_t* argmax_out,
                     const BatchShape* forced);

}  // namespace host
}  // namespace lsp
