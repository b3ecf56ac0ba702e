// lsp_gls_api.cu -- lsp_periodogram_gls: the floating-mean (generalized,
// weighted) periodogram of one curve (gls.cu).
#include <algorithm>
#include <cmath>

#include "lsp_ctx.h"

using lsp::CurveStats;
using lsp::MainShape;
using namespace lsp::host;

namespace {

// Mode from the options (AUTO = the three-term recurrence in packed FP32x2
// form, measured fastest for six sums per frequency); strips are 16
// (recurrences) or 8 (MUFU) frequencies long unless 8 or 16 is asked for.
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
    if (o.freqs_per_thread == 8 || o.freqs_per_thread == 16) s.F = o.freqs_per_thread;
    finish_shape(ctx, s, lsp::gls_occupancy(s.mode, s.F), N, N_f, o.split);
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

    const bool t_dev = is_device_ptr(t), x_dev = is_device_ptr(X), p_dev = is_device_ptr(P_out);
    const bool dy_dev = dy && is_device_ptr(dy);
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
    LSP_CUDA(ctx, lsp::launch_prep_stats(td, xd, nullptr, N_t, 1, stats, ctx->status_d,
                                         (lsp::StatPart*)ctx->stat_parts.p, (unsigned*)ctx->stat_counters.p, st,
                                         dyd));
    LSP_CUDA(ctx, lsp::launch_prep_records(td, xd, nullptr, N_t, 1, N_t, nullptr, nullptr, f_0, df, stats,
                                           (uint4*)ctx->recA.p, (float4*)ctx->recB.p, nullptr, nullptr, st, dyd,
                                           (float*)ctx->recQ.p));
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    LSP_CUDA(ctx, lsp::launch_gls(s, (const uint4*)ctx->recA.p, (const float4*)ctx->recB.p,
                                  (const float*)ctx->recQ.p, N_t, N_f, (float*)ctx->part.p, pd, st));
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
    ctx->last_launches = 3;
    if (s.split > 1) {
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
