// lsp_api.cu -- the C ABI of include/lsp.h: context, workspace, argument
// checks, launch-shape choice and the host<->device staging of host pointers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>

#include "lsp_ctx.h"
#include "lsp_testing.h"

using lsp::CurveStats;
using lsp::MainShape;
using namespace lsp::host;

namespace {

lsp_status check_options(lsp_ctx* ctx, const lsp_options* o) {
    if (o->sincos_mode < 0 || o->sincos_mode > 4)
        return fail(ctx, LSP_ERR_INVALID_ARG, "sincos_mode %d out of range", o->sincos_mode);
    if (o->phase_mode < 0 || o->phase_mode > 1)
        return fail(ctx, LSP_ERR_INVALID_ARG, "phase_mode %d out of range", o->phase_mode);
    const int F = o->freqs_per_thread;
    if (F != 0 && F != 4 && F != 8 && F != 12 && F != 16 && F != 20 && F != 24 && F != 28)
        return fail(ctx, LSP_ERR_INVALID_ARG, "freqs_per_thread must be 0, 4, 8, 12, 16, 20, 24 or 28");
    if ((F == 20 || F == 28) && (o->sincos_mode == LSP_SINCOS_MUFU || o->phase_mode == LSP_PHASE_NAIVE_FP32))
        return fail(ctx, LSP_ERR_INVALID_ARG, "freqs_per_thread 20 and 28 are recurrence-only");
    // the split is the grid's second dimension
    if (o->split < 0 || o->split > 65535) return fail(ctx, LSP_ERR_INVALID_ARG, "split must be in [0, 65535]");
    if (o->batch_rhs != 0 && o->batch_rhs != 1 && o->batch_rhs != 2 && o->batch_rhs != 4 && o->batch_rhs != 8)
        return fail(ctx, LSP_ERR_INVALID_ARG, "batch_rhs must be 0, 1, 2, 4 or 8");
    for (int i = 0; i < 5; ++i)
        if (o->reserved[i] != 0) return fail(ctx, LSP_ERR_INVALID_ARG, "reserved option fields must be zero");
    return LSP_OK;
}

}  // namespace

// Kernel mode and strip length for the options, before any size-dependent
// choice: the strip lengths measured best on GB300 for each mode on large
// curves (gapped_100k), or the one asked for.
void lsp::host::default_mode_F(const lsp_options& o, int* mode, int* F) {
    if (o.phase_mode == LSP_PHASE_NAIVE_FP32) {
        *mode = lsp::kModeNaive;
        *F = 8;
    } else if (o.sincos_mode == LSP_SINCOS_MUFU) {
        *mode = lsp::kModeMufu;
        *F = 8;
    } else if (o.sincos_mode == LSP_SINCOS_RECUR) {
        *mode = lsp::kModeRecur;
        *F = 16;
    } else if (o.sincos_mode == LSP_SINCOS_RECUR3) {
        *mode = lsp::kModeRecur3;
        *F = 24;
    } else {  // AUTO and RECUR3_X2: the packed three-term strip, bit-identical to RECUR3 and faster
        *mode = lsp::kModeRecur3x2;
        *F = 24;
    }
    if (o.freqs_per_thread) *F = o.freqs_per_thread;
}

// Launch shape: mode, strip length F, N_t split.  The split is chosen so the
// grid fills whole waves of resident CTAs, with chunks of at least kMinChunk
// samples; problems that still leave the GPU short of one wave get shorter
// strips as well.
MainShape lsp::host::choose_shape(const lsp_ctx* ctx, int64_t N, int64_t N_f) {
    MainShape s{};
    lsp_options o = ctx->opt;
    // AUTO with an autotuned entry for this size: take its mode, F and split
    if (o.sincos_mode == LSP_SINCOS_AUTO && o.phase_mode == LSP_PHASE_FIXED64 && o.freqs_per_thread == 0 &&
        o.split == 0) {
        if (const TuneEntry* te = tuned(ctx, N, N_f)) {
            o.sincos_mode = te->sincos;
            o.freqs_per_thread = te->F;
            o.split = (int)std::min<int64_t>(te->split, std::max<int64_t>(1, N / lsp::kMinChunk));
        }
    }
    default_mode_F(o, &s.mode, &s.F);
    if (o.freqs_per_thread) {
        s.F = o.freqs_per_thread;
    } else if (s.mode != lsp::kModeNaive) {
        // small problems: shorter strips until the grid (at the shortest
        // chunks) fills a wave of resident CTAs, down to 4 frequencies
        const int64_t max_split = std::max<int64_t>(1, N / lsp::kMinChunk);
        for (int f : {24, 16, 8, 4}) {
            if (f > s.F) continue;
            s.F = f;
            const int64_t per = lsp::freqs_per_block(f);
            const int64_t slots = (int64_t)std::max(1, lsp::main_occupancy(s.mode, f)) * std::max(1, ctx->sms);
            if ((N_f + per - 1) / per * max_split >= slots) break;
        }
    }
    finish_shape(ctx, s, lsp::main_occupancy(s.mode, s.F), N, N_f, o.split);
    return s;
}

// Frequency blocks, padding and the N_t split of a shape whose mode and F are
// set; occ = resident CTAs per SM of its kernel, `threads` its CTA size,
// `ops` its FMA-pipe operations per term and `rows` its partial sums per
// frequency.  The automatic split minimizes a time model: the CTAs of equal
// work run in waves of occ x SMs, so the main kernel takes about
// ceil(CTAs / slots) x chunk sample-steps, each costing (ops F + 16) issue
// slots for every warp sharing a sub-partition; the partial sums of the
// chunks are written and read back once (at ~4 TB/s).  Chunks stay within
// kMaxChunk samples (precision) and above kMinChunk.  On the 100k x 200k
// periodogram this picks 65 chunks over 7 waves (main kernel 3.74 ms) where
// filling a single wave as fully as possible took 9 chunks (3.88 ms: 2,349 of
// 2,432 slots busy).
void lsp::host::finish_shape(const lsp_ctx* ctx, MainShape& s, int occ_in, int64_t N, int64_t N_f, int split,
                             int threads, int ops, int rows) {
    const int64_t per_block = (int64_t)threads * s.F;
    s.nfb = (int)((N_f + per_block - 1) / per_block);
    s.nf_pad = (int64_t)s.nfb * per_block;
    if (split <= 0) {
        const int occ = std::max(1, occ_in);
        const int64_t slots = (int64_t)occ * std::max(1, ctx->sms);
        const int64_t max_split = std::max<int64_t>(1, N / lsp::kMinChunk);
        // at most kMaxChunk samples per chunk, then up to 255 more splits
        const int64_t lo = std::min<int64_t>(65535, std::max<int64_t>(1, (N + lsp::kMaxChunk - 1) / lsp::kMaxChunk));
        const int64_t hi = std::min<int64_t>(65535, std::max<int64_t>(lo, std::min<int64_t>(max_split, lo + 255)));
        const double warps_per_subpartition = std::max(1.0, (double)occ * (threads / 32) / 4.0);
        const double step_s = (ops * s.F + 16.0) * warps_per_subpartition / (0.9 * 2.0e9);
        const double part_bytes_per_split = (double)s.nf_pad * rows * 4.0 * 2.0;  // written, then read
        double best = 1e300;
        int64_t best_s = lo;
        for (int64_t sp = lo; sp <= hi; ++sp) {
            const int64_t ctas = (int64_t)s.nfb * sp;
            const int64_t waves = (ctas + slots - 1) / slots;
            const int64_t chunk = (N + sp - 1) / sp;
            const double t = (double)waves * (double)chunk * step_s +
                             (sp > 1 ? (double)sp * part_bytes_per_split / 4.0e12 : 0.0);
            if (t < best * (1.0 - 1e-3)) {  // a new split must win by 0.1%
                best = t;
                best_s = sp;
            }
        }
        split = (int)best_s;
    }
    if (split > N) split = (int)std::max<int64_t>(1, N);
    s.chunk = (N + split - 1) / split;
    s.split = (int)((N + s.chunk - 1) / s.chunk);
}

extern "C" {

void lsp_default_options(lsp_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->sincos_mode = LSP_SINCOS_AUTO;
    opt->phase_mode = LSP_PHASE_FIXED64;
}

lsp_status lsp_create(lsp_ctx** out, int device, const lsp_options* opt, void* cuda_stream) {
    if (!out) return LSP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return LSP_ERR_INVALID_ARG;
    }
    DeviceGuard guard(device);
    lsp_ctx* ctx = new lsp_ctx();
    ctx->device = device;
    lsp_default_options(&ctx->opt);
    if (opt) {
        if (check_options(ctx, opt) != LSP_OK) {
            delete ctx;
            return LSP_ERR_INVALID_ARG;
        }
        ctx->opt = *opt;
    }
    cudaError_t e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess && !cuda_stream) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status_d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->status_d, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->status_h, sizeof(int));
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lsp_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? LSP_ERR_OOM : LSP_ERR_CUDA;
    }
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
    *out = ctx;
    return LSP_OK;
}

lsp_status lsp_set_options(lsp_ctx* ctx, const lsp_options* opt) {
    if (!ctx || !opt) return LSP_ERR_INVALID_ARG;
    lsp_status st = check_options(ctx, opt);
    if (st != LSP_OK) return st;
    ctx->opt = *opt;
    return LSP_OK;
}

lsp_status lsp_set_stream(lsp_ctx* ctx, void* cuda_stream) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    if (!cuda_stream && !ctx->own_stream) {
        DeviceGuard guard(ctx->device);
        if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(ctx, LSP_ERR_CUDA, "cannot create stream");
    }
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
    return LSP_OK;
}

lsp_status lsp_grid(double t_min, double t_max, int64_t N_t, double F_over, double F_high, double* f_0,
                    double* df, int64_t* N_f) {
    if (!f_0 || !df || !N_f) return LSP_ERR_INVALID_ARG;
    const double span = t_max - t_min;
    if (!(span > 0.0) || !std::isfinite(span) || !(F_over > 0.0) || !(F_high > 0.0) || N_t < 1)
        return LSP_ERR_INVALID_ARG;
    *df = 1.0 / (F_over * span);
    *f_0 = *df;
    *N_f = (int64_t)std::floor(F_high * F_over * (double)N_t / 2.0);
    return LSP_OK;
}

lsp_status lsp_periodogram(lsp_ctx* ctx, const double* t, const double* X, int64_t N_t, double f_0,
                           double df, int64_t N_f, float* P_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->timing_valid = false;
    ctx->last_launches = 0;
    if (N_t < 2) return fail(ctx, LSP_ERR_INVALID_ARG, "N_t = %lld: need at least 2 samples", (long long)N_t);
    if (N_f < 0 || N_f >= (int64_t(1) << 31))
        return fail(ctx, LSP_ERR_INVALID_ARG, "N_f = %lld out of range [0, 2^31)", (long long)N_f);
    if (!std::isfinite(f_0) || !std::isfinite(df)) return fail(ctx, LSP_ERR_NONFINITE, "f_0 or df is not finite");
    if (N_f == 0) return LSP_OK;
    if (!t || !X || !P_out) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;

    lsp_status rs;
    bool t_dev = false, x_dev = false, p_dev = false;
    if ((rs = where(ctx, t, &t_dev)) != LSP_OK || (rs = where(ctx, X, &x_dev)) != LSP_OK ||
        (rs = where(ctx, P_out, &p_dev)) != LSP_OK)
        return rs;
    const MainShape s = choose_shape(ctx, N_t, N_f);
    if ((rs = ensure(ctx, ctx->recA, (size_t)N_t * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->recB, (size_t)N_t * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->stats, sizeof(CurveStats))) != LSP_OK) return rs;
    const int slices = lsp::prep_stats_slices(1, N_t);
    if ((rs = ensure(ctx, ctx->stat_parts, sizeof(lsp::StatPart) * (size_t)slices)) != LSP_OK) return rs;
    if ((rs = ensure_zeroed(ctx, ctx->stat_counters, sizeof(unsigned))) != LSP_OK) return rs;
    if (s.mode == lsp::kModeNaive && (rs = ensure(ctx, ctx->recN, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (s.split > 1 && (rs = ensure(ctx, ctx->part, (size_t)s.split * 4 * (size_t)s.nf_pad * 4)) != LSP_OK)
        return rs;
    if (!t_dev && (rs = ensure(ctx, ctx->t_stage, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (!x_dev && (rs = ensure(ctx, ctx->x_stage, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (!p_dev && (rs = ensure(ctx, ctx->p_stage, (size_t)N_f * 4)) != LSP_OK) return rs;

    const double* td = t;
    const double* xd = X;
    float* pd = p_dev ? P_out : (float*)ctx->p_stage.p;
    if (!t_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->t_stage.p, t, (size_t)N_t * 8, cudaMemcpyHostToDevice, st));
        td = (const double*)ctx->t_stage.p;
    }
    if (!x_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->x_stage.p, X, (size_t)N_t * 8, cudaMemcpyHostToDevice, st));
        xd = (const double*)ctx->x_stage.p;
    }
    const bool timing = ctx->opt.timing != 0;
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
    CurveStats* stats = (CurveStats*)ctx->stats.p;
    {
        NvtxRange r("lsp_periodogram.prep");
        LSP_CUDA(ctx, lsp::launch_prep_stats(td, xd, nullptr, N_t, 1, stats, ctx->status_d,
                                             (lsp::StatPart*)ctx->stat_parts.p, (unsigned*)ctx->stat_counters.p, st));
        LSP_CUDA(ctx, lsp::launch_prep_records(td, xd, nullptr, N_t, 1, N_t, nullptr, nullptr, f_0, df, stats,
                                               (uint4*)ctx->recA.p, (float4*)ctx->recB.p,
                                               s.mode == lsp::kModeNaive ? (float2*)ctx->recN.p : nullptr, nullptr,
                                               st, nullptr, nullptr, ctx->status_d));
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    {
        NvtxRange r("lsp_periodogram.main");
        LSP_CUDA(ctx, lsp::launch_main(s, (const uint4*)ctx->recA.p, (const float4*)ctx->recB.p,
                                       (const float2*)ctx->recN.p, N_t, N_f, f_0, df, (float*)ctx->part.p, pd, st));
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
    ctx->last_launches = 3;
    if (s.split > 1) {
        NvtxRange r("lsp_periodogram.finalize");
        LSP_CUDA(ctx, lsp::launch_finalize(s, (const float*)ctx->part.p, N_t, N_f, pd, st));
        ctx->last_launches = 4;
    }
    if (timing) {
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[3], st));
        ctx->timing_valid = true;
        ctx->has_finalize = s.split > 1;
    }
    if (!p_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(P_out, pd, (size_t)N_f * 4, cudaMemcpyDeviceToHost, st));
        return lsp_sync(ctx, -1.0);
    }
    return LSP_OK;
}

lsp_status lsp_sync(lsp_ctx* ctx, double timeout_s) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    LSP_CUDA(ctx, cudaMemcpyAsync(ctx->status_h, ctx->status_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LSP_CUDA(ctx, cudaEventRecord(ctx->done, ctx->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaEventQuery(ctx->done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "cudaEventQuery");
        if (timeout_s >= 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) return fail(ctx, LSP_ERR_TIMEOUT, "lsp_sync: %.3f s deadline passed", timeout_s);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    const int flags = *ctx->status_h;
    if (flags) {
        LSP_CUDA(ctx, cudaMemsetAsync(ctx->status_d, 0, sizeof(int), ctx->stream));
        LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (flags & lsp::kStatusNonFinite) return fail(ctx, LSP_ERR_NONFINITE, "non-finite value in t or X");
        if (flags & lsp::kStatusBadWeight) return fail(ctx, LSP_ERR_INVALID_ARG, "dy must be finite and > 0");
        if (flags & lsp::kStatusPhaseRange)
            return fail(ctx, LSP_ERR_INVALID_ARG,
                        "(t - t_min) f_0 or (t - t_min) df reaches 2^52 turns: beyond the exact fixed-point phase");
        return fail(ctx, LSP_ERR_DEGENERATE, "X has zero variance");
    }
    return LSP_OK;
}

lsp_status lsp_last_timing(lsp_ctx* ctx, float* ms_prep, float* ms_main, float* ms_finalize) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    if (!ctx->timing_valid) return fail(ctx, LSP_ERR_INVALID_ARG, "no timed call (set the timing option)");
    LSP_CUDA(ctx, cudaEventSynchronize(ctx->ev[3]));
    float a = 0, b = 0, c = 0;
    LSP_CUDA(ctx, cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
    LSP_CUDA(ctx, cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]));
    LSP_CUDA(ctx, cudaEventElapsedTime(&c, ctx->ev[2], ctx->ev[3]));
    if (ms_prep) *ms_prep = a;
    if (ms_main) *ms_main = b;
    if (ms_finalize) *ms_finalize = ctx->has_finalize ? c : 0.f;
    return LSP_OK;
}

int32_t lsp_last_launch_count(const lsp_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

int32_t lsp_test_pointer_kind(int32_t memory_type, int32_t pointer_device, int32_t device) {
    return pointer_kind(memory_type, pointer_device, device);
}

lsp_status lsp_test_last_batch_shape(const lsp_ctx* ctx, int32_t shape[5]) {
    if (!ctx || !shape || !ctx->plan.valid) return LSP_ERR_INVALID_ARG;
    shape[0] = ctx->plan.mode;
    shape[1] = ctx->plan.F;
    shape[2] = ctx->plan.R;
    shape[3] = ctx->plan.tailF;
    shape[4] = ctx->plan.tile;
    return LSP_OK;
}

lsp_status lsp_test_fail_allocation(lsp_ctx* ctx, int32_t n) {
    if (!ctx || n < 0) return LSP_ERR_INVALID_ARG;
    ctx->fail_alloc_in = n;
    return LSP_OK;
}

const char* lsp_last_error(const lsp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void lsp_destroy(lsp_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_plan(ctx);
    DevBuf* bufs[] = {&ctx->recQ,   &ctx->dy_stage, &ctx->pr_acc, &ctx->pr_z0, &ctx->pr_z1,
                      &ctx->recA,   &ctx->recB,   &ctx->recN,   &ctx->part,    &ctx->stats,  &ctx->t_stage,
                      &ctx->x_stage, &ctx->p_stage, &ctx->stat_parts, &ctx->stat_counters, &ctx->b_recA,
                      &ctx->b_recB,  &ctx->b_xr,   &ctx->b_stats, &ctx->b_items, &ctx->b_head, &ctx->b_maxkey,
                      &ctx->b_seed,  &ctx->b_off,  &ctx->b_nf,   &ctx->b_f0,    &ctx->b_df,   &ctx->b_poff,
                      &ctx->b_t,     &ctx->b_X,    &ctx->b_P,    &ctx->b_maxP,  &ctx->b_argmax,
                      &ctx->b_win,   &ctx->b_woff, &ctx->b_gx};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    lsp::host::FapState& f = ctx->fap;
    DevBuf* fbufs[] = {&f.params, &f.grad, &f.m,    &f.v,    &f.mu_sig, &f.ws,    &f.act,  &f.X,
                       &f.cnt,    &f.y,    &f.loss, &f.q,    &f.rows,   &f.W,     &f.W_off, &f.nw,
                       &f.counts, &f.best, &f.train_state, &f.hist};
    for (DevBuf* b : fbufs)
        if (b->p) cudaFree(b->p);
    if (ctx->status_d) cudaFree(ctx->status_d);
    if (ctx->status_h) cudaFreeHost(ctx->status_h);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (cudaEvent_t& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->done) cudaEventDestroy(ctx->done);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaGetLastError();
    delete ctx;
}

}  // extern "C"
