// lsp_tune_api.cu -- lsp_autotune: pick the sin/cos mode, strip length F
// (which is also the recurrence's re-seed length K) and N_t split for a
// problem size by timing candidates on the device, behind a precision gate.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "lsp_ctx.h"

using namespace lsp::host;

namespace {

int bucket(int64_t v) {
    int b = 0;
    while (v > 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

}  // namespace

// Entry for (N_t, N_f) in the context's tuning table, or null.
const lsp::host::TuneEntry* lsp::host::tuned(const lsp_ctx* ctx, int64_t N, int64_t N_f) {
    const int a = bucket(N), b = bucket(N_f);
    for (const TuneEntry& e : ctx->tune)
        if (e.nt_bucket == a && e.nf_bucket == b) return &e;
    return nullptr;
}

extern "C" lsp_status lsp_autotune(lsp_ctx* ctx, int64_t N_t, int64_t N_f, lsp_options* chosen) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    if (N_t < 2 || N_t > (int64_t(1) << 26) || N_f < 1 || N_f >= (int64_t(1) << 31))
        return fail(ctx, LSP_ERR_INVALID_ARG, "autotune sizes out of range");
    DeviceGuard guard(ctx->device);
    // synthetic input of the requested size: jittered even sampling, a sinusoid plus a deterministic
    // pseudo-random component (the kernels' cost does not depend on the values)
    std::vector<double> t((size_t)N_t), X((size_t)N_t);
    for (int64_t j = 0; j < N_t; ++j) {
        const double u = std::fmod((double)j * 0.6180339887498949, 1.0);
        t[(size_t)j] = (double)j + 0.45 * u;
        X[(size_t)j] = std::sin(0.37 * t[(size_t)j]) + (std::fmod((double)j * 0.7548776662466927, 1.0) - 0.5);
    }
    const double T = t.back() - t.front();
    const double df = 1.0 / (4.0 * T);
    DevBuf dt, dx, dp;
    auto release = [&]() {
        if (dt.p) cudaFree(dt.p);
        if (dx.p) cudaFree(dx.p);
        if (dp.p) cudaFree(dp.p);
    };
    lsp_status rs;
    if ((rs = ensure(ctx, dt, (size_t)N_t * 8)) != LSP_OK || (rs = ensure(ctx, dx, (size_t)N_t * 8)) != LSP_OK ||
        (rs = ensure(ctx, dp, (size_t)N_f * 4)) != LSP_OK) {
        release();
        return rs;
    }
    cudaMemcpy(dt.p, t.data(), (size_t)N_t * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dx.p, X.data(), (size_t)N_t * 8, cudaMemcpyHostToDevice);
    const lsp_options saved = ctx->opt;
    auto run = [&](int sincos, int F, int split, std::vector<float>* out, float* ms) -> lsp_status {
        lsp_options o = saved;
        o.sincos_mode = sincos;
        o.phase_mode = LSP_PHASE_FIXED64;
        o.freqs_per_thread = F;
        o.split = split;
        o.timing = 0;
        ctx->opt = o;
        cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[3];
        lsp_status s = lsp_periodogram(ctx, (const double*)dt.p, (const double*)dx.p, N_t, df, df, N_f, (float*)dp.p);
        if (s != LSP_OK) return s;
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, ctx->stream);
            s = lsp_periodogram(ctx, (const double*)dt.p, (const double*)dx.p, N_t, df, df, N_f, (float*)dp.p);
            if (s != LSP_OK) return s;
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ctx, LSP_ERR_CUDA, "autotune timing");
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            best = std::min(best, m);
        }
        *ms = best;
        if (out) {
            out->resize((size_t)N_f);
            if (cudaMemcpy(out->data(), dp.p, (size_t)N_f * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(ctx, LSP_ERR_CUDA, "autotune readback");
        }
        return LSP_OK;
    };
    // reference: hardware sin/cos for every term
    std::vector<float> ref, got;
    float ms = 0.f;
    if ((rs = run(LSP_SINCOS_MUFU, 8, 0, &ref, &ms)) != LSP_OK) {
        ctx->opt = saved;
        release();
        return rs;
    }
    float pmax = 0.f;
    for (float v : ref) pmax = std::max(pmax, v);
    struct Cand { int sincos, F; };
    const Cand cands[] = {{LSP_SINCOS_RECUR3, 24}, {LSP_SINCOS_RECUR3, 16}, {LSP_SINCOS_RECUR3, 8},
                          {LSP_SINCOS_RECUR3, 4},  {LSP_SINCOS_RECUR, 16},  {LSP_SINCOS_RECUR, 8},
                          {LSP_SINCOS_MUFU, 8}};
    TuneEntry best{bucket(N_t), bucket(N_f), 0, 0, 0, 1e30f};
    for (const Cand& c : cands) {
        // the heuristic split of this candidate, then half and double of it
        ctx->opt = saved;
        ctx->opt.sincos_mode = c.sincos;
        ctx->opt.freqs_per_thread = c.F;
        ctx->opt.split = 0;
        const int base_split = choose_shape(ctx, N_t, N_f).split;
        const int max_split = (int)std::max<int64_t>(base_split, std::max<int64_t>(1, N_t / lsp::kMinChunk));
        const int splits[3] = {base_split, std::max(1, base_split / 2), std::min<int>(base_split * 2, max_split)};
        for (int si = 0; si < 3; ++si) {
            if (si > 0 && splits[si] == base_split) continue;
            if ((rs = run(c.sincos, c.F, splits[si], &got, &ms)) != LSP_OK) {
                ctx->opt = saved;
                release();
                return rs;
            }
            float err = 0.f;
            for (size_t k = 0; k < got.size(); ++k) err = std::max(err, std::fabs(got[k] - ref[k]));
            const bool pass = std::isfinite(err) && err <= 2e-5f * pmax;  // a fifth of the parity budget
            if (pass && ms < best.ms) best = TuneEntry{bucket(N_t), bucket(N_f), c.sincos, c.F, splits[si], ms};
        }
    }
    ctx->opt = saved;
    release();
    if (best.sincos == 0) return fail(ctx, LSP_ERR_CUDA, "autotune: no candidate passed the precision gate");
    ctx->tune.erase(std::remove_if(ctx->tune.begin(), ctx->tune.end(),
                                   [&](const TuneEntry& e) { return e.nt_bucket == best.nt_bucket && e.nf_bucket == best.nf_bucket; }),
                    ctx->tune.end());
    ctx->tune.push_back(best);
    if (chosen) {
        *chosen = saved;
        chosen->sincos_mode = best.sincos;
        chosen->freqs_per_thread = best.F;
        chosen->split = best.split;
    }
    return LSP_OK;
}
