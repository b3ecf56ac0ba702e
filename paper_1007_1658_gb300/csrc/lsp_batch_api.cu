// lsp_batch_api.cu -- lsp_batch and lsp_noise of include/lsp.h.
//
// lsp_batch plans a batch on the host (metadata checks, the work list sorted
// longest curve first) and runs it as one CUDA graph: statistics and phase
// records of every curve, the noise of every realization (when X is NULL),
// the persistent periodogram kernel and the unpacking of the per-curve
// maxima.  The graph is cached with the plan and replayed as long as the
// pointers and the metadata of later calls are the same; a new seed is
// written to device memory before the launch, so it does not need a new graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "lsp_ctx.h"

using namespace lsp::host;
using lsp::MainShape;

void lsp::host::drop_plan(lsp_ctx* ctx) {
    if (ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
    ctx->plan = BatchPlan();
}

lsp_status lsp::host::batch_run(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t,
                                const double* X, uint64_t seed, int32_t n_real, const double* f_0, const double* df,
                                const int64_t* N_f, float* P_out, const int64_t* P_off, float* maxP_out,
                                int32_t* argmax_out, const BatchShape* forced) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->timing_valid = false;
    ctx->last_launches = 0;
    if (n_curves < 1 || n_curves > 65535)
        return fail(ctx, LSP_ERR_INVALID_ARG, "n_curves = %d out of range [1, 65535]", n_curves);
    if (n_real < 1 || n_real > 65535) return fail(ctx, LSP_ERR_INVALID_ARG, "n_real = %d out of range", n_real);
    if (X && n_real != 1) return fail(ctx, LSP_ERR_INVALID_ARG, "with measured X, n_real must be 1");
    if (!t_off || !t || !f_0 || !df || !N_f) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    if (!P_out && !maxP_out && !argmax_out) return fail(ctx, LSP_ERR_INVALID_ARG, "no output requested");
    if (P_out && !P_off) return fail(ctx, LSP_ERR_INVALID_ARG, "P_out needs P_off");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    lsp_status rs;

    // ---- metadata on the host, checked ----
    std::vector<int64_t> off, nf, poff;
    std::vector<double> f0v, dfv;
    if ((rs = fetch(ctx, t_off, (size_t)n_curves + 1, off)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, N_f, (size_t)n_curves, nf)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, f_0, (size_t)n_curves, f0v)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, df, (size_t)n_curves, dfv)) != LSP_OK) return rs;
    if (P_out && (rs = fetch(ctx, P_off, (size_t)n_curves + 1, poff)) != LSP_OK) return rs;
    if (off[0] != 0) return fail(ctx, LSP_ERR_INVALID_ARG, "t_off[0] must be 0");
    for (int c = 0; c < n_curves; ++c) {
        if (off[c + 1] - off[c] < 2)
            return fail(ctx, LSP_ERR_INVALID_ARG, "curve %d has %lld samples (need >= 2)", c,
                        (long long)(off[c + 1] - off[c]));
        if (nf[c] < 0 || nf[c] >= (int64_t(1) << 31))
            return fail(ctx, LSP_ERR_INVALID_ARG, "N_f[%d] = %lld out of range", c, (long long)nf[c]);
        if (!std::isfinite(f0v[c]) || !std::isfinite(dfv[c]))
            return fail(ctx, LSP_ERR_NONFINITE, "grid of curve %d is not finite", c);
        if (P_out && (poff[c + 1] - poff[c] < nf[c] || poff[c] < 0))
            return fail(ctx, LSP_ERR_INVALID_ARG, "P_off leaves fewer than N_f[%d] slots", c);
    }
    const int64_t total = off[n_curves];
    const int64_t P_total = P_out ? poff[n_curves] : 0;
    const bool noise = X == nullptr;

    // ---- launch shape: the single-curve choice of mode and strip length ----
    int mode = 0, F1 = 0;
    default_mode_F(ctx->opt, &mode, &F1);
    if (mode == lsp::kModeNaive)
        return fail(ctx, LSP_ERR_UNSUPPORTED, "lsp_batch does not offer the naive FP32 phase");
    // realizations per pass over the samples (multi-RHS) and the strip length that goes with it
    // (auto: 8 from 8 realizations on -- 4096 patterns x 8 realizations in one
    // packed group of 8 took 224 ms against 2 x 138 for groups of 4 -- else 4)
    int R = 1;
    if (n_real > 1) {
        R = ctx->opt.batch_rhs ? ctx->opt.batch_rhs : (n_real >= 8 ? 8 : 4);
        if (R > n_real) R = n_real >= 8 ? 8 : (n_real >= 4 ? 4 : 2);
    }
    // strip lengths measured best on GB300 for each group size (256 patterns x 64 realizations)
    int F = R == 1 ? F1 : (R == 8 ? 8 : (R == 4 ? 12 : 16));
    // multi-realization strips: a strip length asked for replaces the default when that shape exists
    if (R > 1 && ctx->opt.freqs_per_thread &&
        lsp::mrhs_occupancy(mode, ctx->opt.freqs_per_thread, R, lsp::kTile, false) > 0)
        F = ctx->opt.freqs_per_thread;
    int tailF = lsp::batch_default_tail(F), tile = lsp::kTile;
    // a shape from lsp_autotune_batch for batches like this one, when the
    // options leave the choice to the library
    int64_t nf_total = 0;
    for (int c = 0; c < n_curves; ++c) nf_total += nf[c];
    const BatchShape* shape = forced;
    if (!shape && ctx->opt.sincos_mode == LSP_SINCOS_AUTO && ctx->opt.freqs_per_thread == 0 && ctx->opt.batch_rhs == 0)
        if (const BatchTuneEntry* te = tuned_batch(ctx, batch_bucket(n_curves, off[n_curves], nf_total, n_real)))
            shape = &te->shape;
    if (shape) {
        mode = shape->mode;
        F = shape->F;
        R = std::min<int>(shape->R, n_real);
        if (R > 1 && R < shape->R) R = n_real >= 8 ? 8 : (n_real >= 4 ? 4 : 2);
        tailF = shape->tailF;
        tile = shape->tile;
        if (R != shape->R) {  // fewer realizations than the tuned group: the default shape of this group
            F = R == 1 ? 24 : (R == 8 ? 8 : (R == 4 ? 12 : 16));
            tailF = lsp::batch_default_tail(F);
            tile = lsp::kTile;
        }
    }
    const bool xrec = n_real == 1;  // x travels inside the sample records
    // with four groups of realizations or more per pattern, CC and CS come from
    // one window pass per pattern (4 FMA-pipe ops per term) instead of from every
    // group (2 per term and group), which also frees 2F registers per thread
    // (in the packed mode, the AUTO default, the groups run the packed
    // multi-realization strip, bit-identical to the scalar one: 256 patterns x
    // 64 realizations at R = 8 131.4 -> 104.2 ms with the window sums, 4096
    // patterns x 8 realizations 285.1 -> 224.1 ms with their own).  The window
    // pass pays from four groups per pattern on: 256 patterns at R = 8, with
    // and without it, 3 groups 42.4 / 41.0 ms, 4 groups 54.7 / 54.6, 5 groups
    // 67.1 / 68.0, 8 groups 104.2 / 108.6; at R = 4, 3 groups 26.3 / 25.4,
    // 4 groups 33.2 / 33.6.
    const bool use_win = R > 1 && n_real >= 4 * R;
    if ((R > 1 ? lsp::mrhs_occupancy(mode, F, R, tile, use_win) : lsp::batch_occupancy(mode, F, xrec, tailF, tile)) <= 0 ||
        (use_win && lsp::window_occupancy(mode, F) <= 0))
        return fail(ctx, LSP_ERR_UNSUPPORTED, "batch shape (mode %d, F %d, R %d, tail %d, tile %d) is not built", mode,
                    F, R, tailF, tile);
    const int64_t per_block = lsp::freqs_per_block(F);

    // ---- device views of the inputs (host arrays are copied in, outside the graph) ----
    const int64_t *d_off = nullptr, *d_nf = nullptr, *d_poff = nullptr;
    const double *d_f0 = nullptr, *d_df = nullptr, *d_t = nullptr, *d_X = nullptr;
    if ((rs = device_view(ctx, t_off, (size_t)n_curves + 1, ctx->b_off, &d_off)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, N_f, (size_t)n_curves, ctx->b_nf, &d_nf)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, f_0, (size_t)n_curves, ctx->b_f0, &d_f0)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, df, (size_t)n_curves, ctx->b_df, &d_df)) != LSP_OK) return rs;
    if (P_out && (rs = device_view(ctx, P_off, (size_t)n_curves + 1, ctx->b_poff, &d_poff)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, t, (size_t)total, ctx->b_t, &d_t)) != LSP_OK) return rs;
    if (!noise && (rs = device_view(ctx, X, (size_t)total, ctx->b_X, &d_X)) != LSP_OK) return rs;
    bool p_dev = true, m_dev = true, a_dev = true;
    if (P_out && (rs = where(ctx, P_out, &p_dev)) != LSP_OK) return rs;
    if (maxP_out && (rs = where(ctx, maxP_out, &m_dev)) != LSP_OK) return rs;
    if (argmax_out && (rs = where(ctx, argmax_out, &a_dev)) != LSP_OK) return rs;
    const size_t n_out = (size_t)n_real * (size_t)n_curves;

    // ---- workspace (all allocations happen before any capture) ----
    if ((rs = ensure(ctx, ctx->b_recA, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_recB, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_xr, (size_t)n_real * (size_t)total * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_stats, sizeof(lsp::CurveStats) * (size_t)n_curves)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_head, 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_seed, 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_maxkey, n_out * 8)) != LSP_OK) return rs;
    if (!p_dev && (rs = ensure(ctx, ctx->b_P, (size_t)n_real * (size_t)P_total * 4)) != LSP_OK) return rs;
    if (!m_dev && (rs = ensure(ctx, ctx->b_maxP, n_out * 4)) != LSP_OK) return rs;
    if (!a_dev && (rs = ensure(ctx, ctx->b_argmax, n_out * 4)) != LSP_OK) return rs;
    if (use_win) {
        if ((rs = ensure(ctx, ctx->b_win, (size_t)nf_total * 8)) != LSP_OK) return rs;
        if ((rs = ensure(ctx, ctx->b_woff, ((size_t)n_curves + 1) * 8)) != LSP_OK) return rs;
    }
    float* d_P = P_out ? (p_dev ? P_out : (float*)ctx->b_P.p) : nullptr;
    float* d_maxP = maxP_out ? (m_dev ? maxP_out : (float*)ctx->b_maxP.p) : nullptr;
    int32_t* d_argmax = argmax_out ? (a_dev ? argmax_out : (int32_t*)ctx->b_argmax.p) : nullptr;

    // ---- plan: reuse the cached graph when nothing it depends on changed ----
    const std::vector<const void*> ptrs = {d_off, d_nf, d_f0, d_df, d_poff, d_t, d_X, d_P, d_maxP, d_argmax,
                                           ctx->b_recA.p, ctx->b_recB.p, ctx->b_xr.p, ctx->b_stats.p,
                                           ctx->b_head.p, ctx->b_seed.p, ctx->b_maxkey.p,
                                           use_win ? ctx->b_win.p : nullptr, use_win ? ctx->b_woff.p : nullptr,
                                           ctx->b_items.p};
    BatchPlan& pl = ctx->plan;
    const bool same = pl.valid && pl.n_curves == n_curves && pl.n_real == n_real && pl.mode == mode &&
                      pl.F == F && pl.R == R && pl.tailF == tailF && pl.tile == tile && pl.noise == noise &&
                      pl.ptrs == ptrs && pl.t_off == off &&
                      pl.nf == nf && pl.f0 == f0v && pl.df == dfv && pl.p_off == poff;
    if (!same) {
        NvtxRange r("lsp_batch.plan");
        drop_plan(ctx);
        // work list: curves longest first (each item costs ~N_t), then blocks, then realizations;
        // with single-realization strips longer than the tail strip, the frequencies after a
        // curve's last full block go to tail items of kMainThreads * tailF frequencies
        std::vector<int> order(n_curves);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
        const bool tails = R == 1 && tailF > 0 && F > tailF;
        const int64_t tail_block = lsp::freqs_per_block(tails ? tailF : 1);
        std::vector<lsp::BatchItem> items;
        for (int c : order) {
            const int64_t nfb = tails ? nf[c] / per_block : (nf[c] + per_block - 1) / per_block;
            for (int64_t fb = 0; fb < nfb; ++fb)
                for (int r = 0; r < n_real; r += R) items.push_back({c, r, (int32_t)fb, std::min(R, n_real - r)});
            if (tails) {
                const int64_t ntail = (nf[c] - nfb * per_block + tail_block - 1) / tail_block;
                for (int64_t tb = 0; tb < ntail; ++tb)
                    for (int r = 0; r < n_real; ++r) items.push_back({c, r, (int32_t)nfb, (int32_t)(-1 - tb)});
            }
        }
        // window pass: one item per (curve, block of strips of F), after the main items
        const size_t n_main = items.size();
        std::vector<int64_t> woff;
        if (use_win) {
            woff.assign((size_t)n_curves + 1, 0);
            for (int c = 0; c < n_curves; ++c) woff[c + 1] = woff[c] + nf[c];
            for (int c : order)
                for (int64_t fb = 0; fb < (nf[c] + per_block - 1) / per_block; ++fb) items.push_back({c, 0, (int32_t)fb, 0});
        }
        const size_t n_win = items.size() - n_main;
        if (items.size() >= (size_t)(1u << 31)) return fail(ctx, LSP_ERR_INVALID_ARG, "batch too large");
        const size_t item_bytes = items.size() * sizeof(lsp::BatchItem);
        const size_t woff_bytes = woff.size() * sizeof(int64_t);
        const void* old_items = ctx->b_items.p;
        if ((rs = ensure(ctx, ctx->b_items, item_bytes + 16)) != LSP_OK) return rs;
        if ((rs = ensure_pinned(ctx, item_bytes + woff_bytes + 64)) != LSP_OK) return rs;
        LSP_CUDA(ctx, cudaStreamSynchronize(st));  // the pinned buffer may still feed an earlier copy
        if (!items.empty()) {
            std::memcpy(ctx->pinned, items.data(), item_bytes);
            LSP_CUDA(ctx, cudaMemcpyAsync(ctx->b_items.p, ctx->pinned, item_bytes, cudaMemcpyHostToDevice, st));
        }
        if (use_win) {
            char* hw = (char*)ctx->pinned + ((item_bytes + 15) & ~(size_t)15);
            std::memcpy(hw, woff.data(), woff_bytes);
            LSP_CUDA(ctx, cudaMemcpyAsync(ctx->b_woff.p, hw, woff_bytes, cudaMemcpyHostToDevice, st));
        }
        std::vector<const void*> ptrs2 = ptrs;
        ptrs2.back() = ctx->b_items.p;
        (void)old_items;
        const int occ =
            R > 1 ? lsp::mrhs_occupancy(mode, F, R, tile, use_win) : lsp::batch_occupancy(mode, F, xrec, tailF, tile);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * ctx->sms, (int64_t)n_main));
        const int grid_w = use_win ? (int)std::max<int64_t>(
                                         1, std::min<int64_t>((int64_t)lsp::window_occupancy(mode, F) * ctx->sms,
                                                              (int64_t)n_win))
                                   : 0;

        // capture the batch as one graph, on a private stream (the caller's
        // stream may be the legacy default stream, which cannot be captured);
        // the graph is launched on the caller's stream below
        if (!ctx->cap_stream) LSP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        LSP_CUDA(ctx, cudaStreamSynchronize(st));  // the work list copy must land before replays
        cudaGraph_t g = nullptr;
        const cudaStream_t cst = ctx->cap_stream;
        LSP_CUDA(ctx, cudaStreamBeginCapture(cst, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(ctx->b_head.p, 0, 16, cst);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->b_maxkey.p, 0, n_out * 8, cst);
        if (e == cudaSuccess)
            e = lsp::launch_prep_stats(d_t, d_X, d_off, 0, n_curves, (lsp::CurveStats*)ctx->b_stats.p,
                                       ctx->status_d, nullptr, nullptr, cst);
        if (e == cudaSuccess) {
            const int64_t max_n = off[order[0] + 1] - off[order[0]];
            e = lsp::launch_prep_records(d_t, d_X, d_off, 0, n_curves, max_n, d_f0, d_df, 0.0, 0.0,
                                         (const lsp::CurveStats*)ctx->b_stats.p, (uint4*)ctx->b_recA.p,
                                         (float4*)ctx->b_recB.p, nullptr, noise ? nullptr : (float*)ctx->b_xr.p,
                                         cst, nullptr, nullptr, ctx->status_d);
        }
        if (e == cudaSuccess && noise)
            e = lsp::launch_noise_prep(d_off, n_curves, n_real, (const uint64_t*)ctx->b_seed.p, total,
                                       (float*)ctx->b_xr.p, (float4*)ctx->b_recB.p, cst);
        if (e == cudaSuccess && n_win > 0)
            e = lsp::launch_window(mode, F, grid_w, (const lsp::BatchItem*)ctx->b_items.p + n_main, (int)n_win,
                                   (unsigned*)ctx->b_head.p + 1, d_off, d_nf, (const int64_t*)ctx->b_woff.p,
                                   (const uint4*)ctx->b_recA.p, (const float4*)ctx->b_recB.p,
                                   (float2*)ctx->b_win.p, cst);
        if (e == cudaSuccess && n_main > 0 && R > 1)
            e = lsp::launch_mrhs(mode, F, R, tile, grid, (const lsp::BatchItem*)ctx->b_items.p, (int)n_main,
                                 (unsigned*)ctx->b_head.p, d_off, d_nf, total, n_curves, (const uint4*)ctx->b_recA.p,
                                 (const float4*)ctx->b_recB.p, (const float*)ctx->b_xr.p, d_P, d_poff, P_total,
                                 (unsigned long long*)ctx->b_maxkey.p,
                                 use_win ? (const float2*)ctx->b_win.p : nullptr,
                                 use_win ? (const int64_t*)ctx->b_woff.p : nullptr, cst);
        else if (e == cudaSuccess && n_main > 0)
            e = lsp::launch_batch(mode, F, xrec, tailF, tile, grid, (const lsp::BatchItem*)ctx->b_items.p,
                                  (int)items.size(),
                                  (unsigned*)ctx->b_head.p, d_off, d_nf, total, n_curves,
                                  (const uint4*)ctx->b_recA.p, (const float4*)ctx->b_recB.p,
                                  (const float*)ctx->b_xr.p, d_P, d_poff, P_total,
                                  (unsigned long long*)ctx->b_maxkey.p, cst);
        if (e == cudaSuccess && (d_maxP || d_argmax))
            e = lsp::launch_unpack_max((const unsigned long long*)ctx->b_maxkey.p, (int64_t)n_out, d_maxP,
                                       d_argmax, cst);
        cudaError_t e2 = cudaStreamEndCapture(cst, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&pl.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            drop_plan(ctx);
            return cuda_fail(ctx, e, "capturing the batch graph");
        }
        pl.valid = true;
        pl.ptrs = ptrs2;
        pl.n_curves = n_curves;
        pl.n_real = n_real;
        pl.mode = mode;
        pl.F = F;
        pl.R = R;
        pl.tailF = tailF;
        pl.tile = tile;
        pl.noise = noise;
        pl.t_off = off;
        pl.nf = nf;
        pl.f0 = f0v;
        pl.df = dfv;
        pl.p_off = poff;
        pl.n_items = (int)n_main;
        pl.grid = grid;
        pl.kernels = 3 + (noise ? 1 : 0) + ((d_maxP || d_argmax) ? 1 : 0) + (n_main == 0 ? -1 : 0) + (n_win > 0 ? 1 : 0);
    }

    // ---- run: new seed, one graph launch, outputs back if they live on the host ----
    if ((rs = ensure_pinned(ctx, 64)) != LSP_OK) return rs;
    LSP_CUDA(ctx, cudaStreamSynchronize(st));  // the pinned seed slot may still feed an earlier copy
    std::memcpy(ctx->pinned, &seed, sizeof seed);
    LSP_CUDA(ctx, cudaMemcpyAsync(ctx->b_seed.p, ctx->pinned, sizeof seed, cudaMemcpyHostToDevice, st));
    const bool timing = ctx->opt.timing != 0;
    // a host P_out whose layout leaves slack between curves gets its own values
    // staged first, so that the copy back returns the slack unchanged: the
    // call writes only the bins, wherever P_out lives
    if (P_out && !p_dev && p_layout_has_slack(poff, nf))
        LSP_CUDA(ctx, cudaMemcpyAsync(d_P, P_out, (size_t)n_real * (size_t)P_total * 4, cudaMemcpyHostToDevice, st));
    if (timing) {
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    }
    {
        NvtxRange r("lsp_batch.launch");
        LSP_CUDA(ctx, cudaGraphLaunch(pl.exec, st));
    }
    if (timing) {
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[3], st));
        ctx->timing_valid = true;
        ctx->has_finalize = false;
    }
    ctx->last_launches = pl.kernels;
    bool host_out = false;
    if (P_out && !p_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(P_out, d_P, (size_t)n_real * (size_t)P_total * 4, cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (maxP_out && !m_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(maxP_out, d_maxP, n_out * 4, cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (argmax_out && !a_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(argmax_out, d_argmax, n_out * 4, cudaMemcpyDeviceToHost, st));
        host_out = true;
    }
    if (host_out) return lsp_sync(ctx, -1.0);
    return LSP_OK;
}

extern "C" {

lsp_status lsp_batch(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t, const double* X,
                     uint64_t seed, int32_t n_real, const double* f_0, const double* df, const int64_t* N_f,
                     float* P_out, const int64_t* P_off, float* maxP_out, int32_t* argmax_out) {
    return batch_run(ctx, n_curves, t_off, t, X, seed, n_real, f_0, df, N_f, P_out, P_off, maxP_out, argmax_out,
                     nullptr);
}

lsp_status lsp_noise(lsp_ctx* ctx, uint64_t seed, int32_t curve, int32_t real, int64_t N, float* out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    if (N < 0 || curve < 0 || real < 0 || (N > 0 && !out)) return fail(ctx, LSP_ERR_INVALID_ARG, "bad argument");
    if (N == 0) return LSP_OK;
    if (N > (int64_t(1) << 34)) return fail(ctx, LSP_ERR_INVALID_ARG, "N too large");
    DeviceGuard guard(ctx->device);
    bool dev = false;
    lsp_status rs = where(ctx, out, &dev);
    if (rs != LSP_OK) return rs;
    float* d = out;
    if (!dev) {
        rs = ensure(ctx, ctx->p_stage, (size_t)N * 4);
        if (rs != LSP_OK) return rs;
        d = (float*)ctx->p_stage.p;
    }
    LSP_CUDA(ctx, lsp::launch_noise_raw(seed, (uint32_t)curve, (uint32_t)real, N, d, ctx->stream));
    ctx->last_launches = 1;
    if (!dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(out, d, (size_t)N * 4, cudaMemcpyDeviceToHost, ctx->stream));
        return lsp_sync(ctx, -1.0);
    }
    return LSP_OK;
}

}  // extern "C"
