// lsp_gls_api.cu -- lsp_periodogram_gls, lsp_batch_gls and lsp_batch_gls_noise: the floating-mean
// (generalized, weighted) periodogram of one curve or of many (gls.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lsp_ctx.h"

using lsp::CurveStats;
using lsp::MainShape;
using namespace lsp::host;

namespace {

// Mode from the options (AUTO = the three-term recurrence in packed FP32x2
// form, measured fastest for six sums per frequency); strips are 16
// (recurrences) or 8 (MUFU) frequencies long unless 8, 12 or 16 is asked for
// (12 measured equal to 16, 8 slower).
MainShape choose_gls_shape(const lsp_ctx* ctx, int64_t N, int64_t N_f) {
    MainShape s{};
    const lsp_options& o = ctx->opt;
    if (o.sincos_mode == LSP_SINCOS_MUFU) {
        s.mode = lsp::kModeMufu;
        s.F = 8;
    } else if (o.sincos_mode == LSP_SINCOS_RECUR) {
        s.mode = lsp::kModeRecur;
        s.F = 16;
    } else if (o.sincos_mode == LSP_SINCOS_RECUR3) {
        s.mode = lsp::kModeRecur3;
        s.F = 16;
    } else {
        s.mode = lsp::kModeRecur3x2;
        s.F = 16;
    }
    if (o.freqs_per_thread == 8 || o.freqs_per_thread == 12 || o.freqs_per_thread == 16) s.F = o.freqs_per_thread;
    finish_shape(ctx, s, lsp::gls_occupancy(s.mode, s.F), N, N_f, o.split, lsp::kGlsThreads, 8, lsp::kGlsRows);
    return s;
}

}  // namespace

extern "C" {

lsp_status lsp_periodogram_gls(lsp_ctx* ctx, const double* t, const double* X, const double* dy, int64_t N_t,
                               double f_0, double df, int64_t N_f, float* P_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->timing_valid = false;
    ctx->last_launches = 0;
    if (N_t < 3) return fail(ctx, LSP_ERR_INVALID_ARG, "N_t = %lld: need at least 3 samples", (long long)N_t);
    if (N_f < 0 || N_f >= (int64_t(1) << 31))
        return fail(ctx, LSP_ERR_INVALID_ARG, "N_f = %lld out of range [0, 2^31)", (long long)N_f);
    if (!std::isfinite(f_0) || !std::isfinite(df)) return fail(ctx, LSP_ERR_NONFINITE, "f_0 or df is not finite");
    if (ctx->opt.phase_mode != LSP_PHASE_FIXED64)
        return fail(ctx, LSP_ERR_UNSUPPORTED, "the floating-mean periodogram uses the fixed-point phase only");
    if (N_f == 0) return LSP_OK;
    if (!t || !X || !P_out) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;

    bool t_dev = false, x_dev = false, p_dev = false, dy_dev = false;
    {
        lsp_status ws;
        if ((ws = where(ctx, t, &t_dev)) != LSP_OK || (ws = where(ctx, X, &x_dev)) != LSP_OK ||
            (ws = where(ctx, P_out, &p_dev)) != LSP_OK || (dy && (ws = where(ctx, dy, &dy_dev)) != LSP_OK))
            return ws;
    }
    const MainShape s = choose_gls_shape(ctx, N_t, N_f);
    lsp_status rs;
    if ((rs = ensure(ctx, ctx->recA, (size_t)N_t * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->recB, (size_t)N_t * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->recQ, (size_t)N_t * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->stats, sizeof(CurveStats))) != LSP_OK) return rs;
    const int slices = lsp::prep_stats_slices(1, N_t);
    if ((rs = ensure(ctx, ctx->stat_parts, sizeof(lsp::StatPart) * (size_t)slices)) != LSP_OK) return rs;
    if ((rs = ensure_zeroed(ctx, ctx->stat_counters, sizeof(unsigned))) != LSP_OK) return rs;
    if (s.split > 1 &&
        (rs = ensure(ctx, ctx->part, (size_t)s.split * lsp::kGlsRows * (size_t)s.nf_pad * 4)) != LSP_OK)
        return rs;
    if (!t_dev && (rs = ensure(ctx, ctx->t_stage, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (!x_dev && (rs = ensure(ctx, ctx->x_stage, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (dy && !dy_dev && (rs = ensure(ctx, ctx->dy_stage, (size_t)N_t * 8)) != LSP_OK) return rs;
    if (!p_dev && (rs = ensure(ctx, ctx->p_stage, (size_t)N_f * 4)) != LSP_OK) return rs;

    const double* td = t;
    const double* xd = X;
    const double* dyd = dy;
    float* pd = p_dev ? P_out : (float*)ctx->p_stage.p;
    if (!t_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->t_stage.p, t, (size_t)N_t * 8, cudaMemcpyHostToDevice, st));
        td = (const double*)ctx->t_stage.p;
    }
    if (!x_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->x_stage.p, X, (size_t)N_t * 8, cudaMemcpyHostToDevice, st));
        xd = (const double*)ctx->x_stage.p;
    }
    if (dy && !dy_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->dy_stage.p, dy, (size_t)N_t * 8, cudaMemcpyHostToDevice, st));
        dyd = (const double*)ctx->dy_stage.p;
    }
    const bool timing = ctx->opt.timing != 0;
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
    CurveStats* stats = (CurveStats*)ctx->stats.p;
    {
        NvtxRange r("lsp_periodogram_gls.prep");
        LSP_CUDA(ctx, lsp::launch_prep_stats(td, xd, nullptr, N_t, 1, stats, ctx->status_d,
                                             (lsp::StatPart*)ctx->stat_parts.p, (unsigned*)ctx->stat_counters.p, st,
                                             dyd));
        LSP_CUDA(ctx, lsp::launch_prep_records(td, xd, nullptr, N_t, 1, N_t, nullptr, nullptr, f_0, df, stats,
                                               (uint4*)ctx->recA.p, (float4*)ctx->recB.p, nullptr, nullptr, st, dyd,
                                               (float*)ctx->recQ.p, ctx->status_d));
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    {
        NvtxRange r("lsp_periodogram_gls.main");
        LSP_CUDA(ctx, lsp::launch_gls(s, (const uint4*)ctx->recA.p, (const float4*)ctx->recB.p,
                                      (const float*)ctx->recQ.p, N_t, N_f, (float*)ctx->part.p, pd, st));
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
    ctx->last_launches = 3;
    if (s.split > 1) {
        NvtxRange r("lsp_periodogram_gls.finalize");
        LSP_CUDA(ctx, lsp::launch_gls_finalize(s, (const float*)ctx->part.p, N_t, N_f, pd, st));
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

}  // extern "C"

namespace {

// lsp_batch_gls (measured X, one realization) and lsp_batch_gls_noise (X =
// NULL: n_real noise realizations drawn on the device) share this body; with
// noise, item (curve, realization) takes its x from the realization's row.
lsp_status gls_batch_run(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t, const double* X,
                         const double* dy, uint64_t seed, int32_t n_real, const double* f_0, const double* df,
                         const int64_t* N_f, float* P_out, const int64_t* P_off, float* maxP_out,
                         int32_t* argmax_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->timing_valid = false;
    ctx->last_launches = 0;
    if (n_curves < 1 || n_curves > 65535)
        return fail(ctx, LSP_ERR_INVALID_ARG, "n_curves = %d out of range [1, 65535]", n_curves);
    if (n_real < 1 || n_real > 65535) return fail(ctx, LSP_ERR_INVALID_ARG, "n_real = %d out of range", n_real);
    const bool noise = X == nullptr;
    if (!t_off || !t || !f_0 || !df || !N_f) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    if (!P_out && !maxP_out && !argmax_out) return fail(ctx, LSP_ERR_INVALID_ARG, "no output requested");
    if (P_out && !P_off) return fail(ctx, LSP_ERR_INVALID_ARG, "P_out needs P_off");
    if (ctx->opt.phase_mode != LSP_PHASE_FIXED64)
        return fail(ctx, LSP_ERR_UNSUPPORTED, "the floating-mean periodogram uses the fixed-point phase only");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    lsp_status rs;

    std::vector<int64_t> off, nf, poff;
    std::vector<double> f0v, dfv;
    if ((rs = fetch(ctx, t_off, (size_t)n_curves + 1, off)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, N_f, (size_t)n_curves, nf)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, f_0, (size_t)n_curves, f0v)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, df, (size_t)n_curves, dfv)) != LSP_OK) return rs;
    if (P_out && (rs = fetch(ctx, P_off, (size_t)n_curves + 1, poff)) != LSP_OK) return rs;
    if (off[0] != 0) return fail(ctx, LSP_ERR_INVALID_ARG, "t_off[0] must be 0");
    for (int c = 0; c < n_curves; ++c) {
        if (off[c + 1] - off[c] < 3)
            return fail(ctx, LSP_ERR_INVALID_ARG, "curve %d has %lld samples (need >= 3)", c,
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

    // the batch buffers are shared with lsp_batch: its cached work list is rebuilt next time
    drop_plan(ctx);
    const int64_t *d_off = nullptr, *d_nf = nullptr, *d_poff = nullptr;
    const double *d_f0 = nullptr, *d_df = nullptr, *d_t = nullptr, *d_X = nullptr, *d_dy = nullptr;
    if ((rs = device_view(ctx, t_off, (size_t)n_curves + 1, ctx->b_off, &d_off)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, N_f, (size_t)n_curves, ctx->b_nf, &d_nf)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, f_0, (size_t)n_curves, ctx->b_f0, &d_f0)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, df, (size_t)n_curves, ctx->b_df, &d_df)) != LSP_OK) return rs;
    if (P_out && (rs = device_view(ctx, P_off, (size_t)n_curves + 1, ctx->b_poff, &d_poff)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, t, (size_t)total, ctx->b_t, &d_t)) != LSP_OK) return rs;
    if (!noise && (rs = device_view(ctx, X, (size_t)total, ctx->b_X, &d_X)) != LSP_OK) return rs;
    if (dy && (rs = device_view(ctx, dy, (size_t)total, ctx->dy_stage, &d_dy)) != LSP_OK) return rs;
    bool p_dev = true, m_dev = true, a_dev = true;
    if (P_out && (rs = where(ctx, P_out, &p_dev)) != LSP_OK) return rs;
    if (maxP_out && (rs = where(ctx, maxP_out, &m_dev)) != LSP_OK) return rs;
    if (argmax_out && (rs = where(ctx, argmax_out, &a_dev)) != LSP_OK) return rs;

    // mode and strip length as for the single-curve floating-mean call
    const MainShape shape = choose_gls_shape(ctx, 1 << 20, 1 << 24);
    const int mode = shape.mode;
    int F = shape.F;
    if (noise && lsp::gls_batch_occupancy(mode, F, false, true) <= 0)
        return fail(ctx, LSP_ERR_UNSUPPORTED, "noise realizations run the packed three-term strip of 16 or 8 "
                                              "frequencies only (sin/cos mode AUTO or RECUR3_X2)");
    // realizations sharing one pass over the samples (the batch_rhs option;
    // auto: groups of 8 from 8 realizations on, else 4), each group in strips
    // of 8 (of 4 for groups of 8).  256 patterns x 64 realizations: one at a
    // time 344 ms, groups of 2, 4, 8: 246, 175, 139 ms.
    int R = 1;
    if (noise && n_real > 1) {
        R = ctx->opt.batch_rhs ? ctx->opt.batch_rhs : (n_real >= 8 ? 8 : 4);
        if (R > n_real) R = n_real >= 8 ? 8 : (n_real >= 4 ? 4 : 2);
        if (R > 1) F = R == 8 ? 4 : 8;
        if (R > 1 && lsp::gls_mrhs_occupancy(F, R) <= 0)
            return fail(ctx, LSP_ERR_UNSUPPORTED, "batch_rhs = %d is not built for the floating-mean form", R);
    }
    const int64_t per_block = lsp::gls_batch_freqs_per_block(F);
    std::vector<int> order(n_curves);
    for (int c = 0; c < n_curves; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    // longest curve first, each curve's realizations together (in groups of R)
    std::vector<lsp::BatchItem> items;
    for (int c : order) {
        const int64_t nfb = (nf[c] + per_block - 1) / per_block;
        for (int r = 0; r < n_real; r += R)
            for (int64_t fb = 0; fb < nfb; ++fb) items.push_back({c, r, (int32_t)fb, std::min(R, n_real - r)});
        if (items.size() >= (size_t)(1u << 31)) return fail(ctx, LSP_ERR_INVALID_ARG, "batch too large");
    }
    const size_t n_out = (size_t)n_real * (size_t)n_curves;

    if ((rs = ensure(ctx, ctx->b_recA, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_recB, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_xr, (size_t)total * 4)) != LSP_OK) return rs;  // the sqrt-weights
    if ((rs = ensure(ctx, ctx->b_stats, sizeof(lsp::CurveStats) * (size_t)n_curves)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_head, 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_maxkey, n_out * 8)) != LSP_OK) return rs;
    if (noise && (rs = ensure(ctx, ctx->b_gx, (size_t)n_real * (size_t)total * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_items, items.size() * sizeof(lsp::BatchItem) + 16)) != LSP_OK) return rs;
    if (!p_dev && (rs = ensure(ctx, ctx->b_P, (size_t)n_real * (size_t)P_total * 4)) != LSP_OK) return rs;
    if (!m_dev && (rs = ensure(ctx, ctx->b_maxP, n_out * 4)) != LSP_OK) return rs;
    if (!a_dev && (rs = ensure(ctx, ctx->b_argmax, n_out * 4)) != LSP_OK) return rs;
    float* d_P = P_out ? (p_dev ? P_out : (float*)ctx->b_P.p) : nullptr;
    float* d_maxP = maxP_out ? (m_dev ? maxP_out : (float*)ctx->b_maxP.p) : nullptr;
    int32_t* d_argmax = argmax_out ? (a_dev ? argmax_out : (int32_t*)ctx->b_argmax.p) : nullptr;

    const size_t item_bytes = items.size() * sizeof(lsp::BatchItem);
    if ((rs = ensure_pinned(ctx, item_bytes + 64)) != LSP_OK) return rs;
    LSP_CUDA(ctx, cudaStreamSynchronize(st));  // the pinned buffer may still feed an earlier copy
    if (!items.empty()) {
        std::memcpy(ctx->pinned, items.data(), item_bytes);
        LSP_CUDA(ctx, cudaMemcpyAsync(ctx->b_items.p, ctx->pinned, item_bytes, cudaMemcpyHostToDevice, st));
    }
    // a host P_out whose layout leaves slack between curves gets its own values
    // staged first, so that the copy back returns the slack unchanged
    if (P_out && !p_dev && p_layout_has_slack(poff, nf))
        LSP_CUDA(ctx, cudaMemcpyAsync(d_P, P_out, (size_t)n_real * (size_t)P_total * 4, cudaMemcpyHostToDevice, st));
    const bool timing = ctx->opt.timing != 0;
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
    LSP_CUDA(ctx, cudaMemsetAsync(ctx->b_head.p, 0, 16, st));
    LSP_CUDA(ctx, cudaMemsetAsync(ctx->b_maxkey.p, 0, n_out * 8, st));
    lsp::CurveStats* stats = (lsp::CurveStats*)ctx->b_stats.p;
    LSP_CUDA(ctx, lsp::launch_prep_stats(d_t, d_X, d_off, 0, n_curves, stats, ctx->status_d, nullptr, nullptr, st,
                                         d_dy));
    const int64_t max_n = off[order[0] + 1] - off[order[0]];
    LSP_CUDA(ctx, lsp::launch_prep_records(d_t, d_X, d_off, 0, n_curves, max_n, d_f0, d_df, 0.0, 0.0, stats,
                                           (uint4*)ctx->b_recA.p, (float4*)ctx->b_recB.p, nullptr, nullptr, st,
                                           d_dy, (float*)ctx->b_xr.p, ctx->status_d));
    int launches = 2;
    if (noise) {
        LSP_CUDA(ctx, lsp::launch_gls_noise_prep(d_off, n_curves, n_real, seed, total, d_dy, (const float*)ctx->b_xr.p,
                                                 (float*)ctx->b_gx.p, st));
        ++launches;
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    if (!items.empty()) {
        NvtxRange r("lsp_batch_gls.main");
        // the packed form when the work is many times the longest curve's, per
        // SM sub-partition: its throughput then counts, not one warp's speed on
        // the longest item (measured at ratios 4, 15 and 58: packed 14 % slower,
        // equal, 2 % faster)
        double work = 0.0;
        for (int c = 0; c < n_curves; ++c)
            work += (double)(off[c + 1] - off[c]) * (double)((nf[c] + per_block - 1) / per_block);
        work *= (double)n_real;
        if (R > 1) {
            // realization groups (noise only)
            const int occ = std::max(1, lsp::gls_mrhs_occupancy(F, R));
            const int grid =
                (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * ctx->sms, (int64_t)items.size()));
            LSP_CUDA(ctx, lsp::launch_gls_mrhs(F, R, grid, (const lsp::BatchItem*)ctx->b_items.p, (int)items.size(),
                                               (unsigned*)ctx->b_head.p, d_off, d_nf, (const uint4*)ctx->b_recA.p,
                                               (const float4*)ctx->b_recB.p, (const float*)ctx->b_xr.p, d_P, d_poff,
                                               (unsigned long long*)ctx->b_maxkey.p, (const float*)ctx->b_gx.p,
                                               total, P_total, n_curves, st));
        } else {
            const bool packed = lsp::gls_batch_occupancy(mode, F, true, noise) > 0 &&
                                work >= 12.0 * 4.0 * ctx->sms * (double)max_n;
            const int occ = std::max(1, lsp::gls_batch_occupancy(mode, F, packed, noise));
            const int grid =
                (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * ctx->sms, (int64_t)items.size()));
            LSP_CUDA(ctx, lsp::launch_gls_batch(mode, F, packed, grid, (const lsp::BatchItem*)ctx->b_items.p,
                                                (int)items.size(), (unsigned*)ctx->b_head.p, d_off, d_nf,
                                                (const uint4*)ctx->b_recA.p, (const float4*)ctx->b_recB.p,
                                                (const float*)ctx->b_xr.p, d_P, d_poff,
                                                (unsigned long long*)ctx->b_maxkey.p, st,
                                                noise ? (const float*)ctx->b_gx.p : nullptr, total, P_total,
                                                n_curves));
        }
        ++launches;
    }
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
    if (d_maxP || d_argmax) {
        LSP_CUDA(ctx, lsp::launch_unpack_max((const unsigned long long*)ctx->b_maxkey.p, (int64_t)n_out, d_maxP,
                                             d_argmax, st));
        ++launches;
    }
    if (timing) {
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[3], st));
        ctx->timing_valid = true;
        ctx->has_finalize = true;
    }
    ctx->last_launches = launches;
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

}  // namespace

extern "C" {

lsp_status lsp_batch_gls(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t, const double* X,
                         const double* dy, const double* f_0, const double* df, const int64_t* N_f, float* P_out,
                         const int64_t* P_off, float* maxP_out, int32_t* argmax_out) {
    if (ctx && !X) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    return gls_batch_run(ctx, n_curves, t_off, t, X, dy, 0, 1, f_0, df, N_f, P_out, P_off, maxP_out, argmax_out);
}

lsp_status lsp_batch_gls_noise(lsp_ctx* ctx, int32_t n_curves, const int64_t* t_off, const double* t,
                               const double* dy, uint64_t seed, int32_t n_real, const double* f_0, const double* df,
                               const int64_t* N_f, float* P_out, const int64_t* P_off, float* maxP_out,
                               int32_t* argmax_out) {
    return gls_batch_run(ctx, n_curves, t_off, t, nullptr, dy, seed, n_real, f_0, df, N_f, P_out, P_off, maxP_out,
                         argmax_out);
}

}  // extern "C"
