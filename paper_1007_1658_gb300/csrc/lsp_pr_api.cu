// lsp_pr_api.cu -- lsp_press_rybicki: the Press & Rybicki fast approximate
// periodogram (press_rybicki.cu) behind the C ABI.
#include <cmath>

#include "lsp_ctx.h"

using lsp::CurveStats;
using namespace lsp::host;

extern "C" {

lsp_status lsp_press_rybicki(lsp_ctx* ctx, const double* t, const double* X, int64_t N_t, double f_0, double df,
                             int64_t N_f, int32_t macc, float* P_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    ctx->timing_valid = false;
    ctx->last_launches = 0;
    if (N_t < 2) return fail(ctx, LSP_ERR_INVALID_ARG, "N_t = %lld: need at least 2 samples", (long long)N_t);
    if (N_f < 0 || N_f >= (int64_t(1) << 31))
        return fail(ctx, LSP_ERR_INVALID_ARG, "N_f = %lld out of range [0, 2^31)", (long long)N_f);
    if (!std::isfinite(f_0) || !std::isfinite(df)) return fail(ctx, LSP_ERR_NONFINITE, "f_0 or df is not finite");
    if (macc == 0) macc = 4;
    if (macc < 2 || macc > 16 || (macc & 1))
        return fail(ctx, LSP_ERR_INVALID_ARG, "macc = %d: need an even number of nodes in [2, 16]", macc);
    if (!(df > 0.0)) return fail(ctx, LSP_ERR_INVALID_ARG, "df must be > 0");
    const double jr = f_0 / df;
    const double j0d = std::nearbyint(jr);
    if (j0d < 0.0 || std::fabs(jr - j0d) > 1e-9 * std::fmax(1.0, std::fabs(jr)))
        return fail(ctx, LSP_ERR_INVALID_ARG, "f_0 must be a non-negative integer multiple of df (FFT grid)");
    if (N_f == 0) return LSP_OK;
    if (!t || !X || !P_out) return fail(ctx, LSP_ERR_INVALID_ARG, "null array pointer");
    const int64_t j0 = (int64_t)j0d;
    const int64_t n_fft = lsp::pr_fft_size(j0 + N_f - 1, macc);
    if (n_fft > (int64_t(1) << 28))
        return fail(ctx, LSP_ERR_INVALID_ARG, "FFT grid of %lld nodes exceeds 2^28", (long long)n_fft);
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;

    bool t_dev = false, x_dev = false, p_dev = false;
    {
        lsp_status ws;
        if ((ws = where(ctx, t, &t_dev)) != LSP_OK || (ws = where(ctx, X, &x_dev)) != LSP_OK ||
            (ws = where(ctx, P_out, &p_dev)) != LSP_OK)
            return ws;
    }
    lsp_status rs;
    if ((rs = ensure(ctx, ctx->stats, sizeof(CurveStats))) != LSP_OK) return rs;
    const int slices = lsp::prep_stats_slices(1, N_t);
    if ((rs = ensure(ctx, ctx->stat_parts, sizeof(lsp::StatPart) * (size_t)slices)) != LSP_OK) return rs;
    if ((rs = ensure_zeroed(ctx, ctx->stat_counters, sizeof(unsigned))) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->pr_acc, (size_t)n_fft * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->pr_z0, (size_t)n_fft * 8)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->pr_z1, (size_t)n_fft * 8)) != LSP_OK) return rs;
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
    LSP_CUDA(ctx, lsp::launch_prep_stats(td, xd, nullptr, N_t, 1, stats, ctx->status_d,
                                         (lsp::StatPart*)ctx->stat_parts.p, (unsigned*)ctx->stat_counters.p, st));
    if (timing) LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    int launches = 0;
    LSP_CUDA(ctx, lsp::launch_pr(td, xd, N_t, stats, df, j0, N_f, macc, n_fft, (double2*)ctx->pr_acc.p,
                                 (float2*)ctx->pr_z0.p, (float2*)ctx->pr_z1.p, pd, &launches, st));
    if (timing) {
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
        LSP_CUDA(ctx, cudaEventRecord(ctx->ev[3], st));
        ctx->timing_valid = true;
        ctx->has_finalize = false;
    }
    ctx->last_launches = 1 + launches;
    if (!p_dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(P_out, pd, (size_t)N_f * 4, cudaMemcpyDeviceToHost, st));
        return lsp_sync(ctx, -1.0);
    }
    return LSP_OK;
}

}  // extern "C"
