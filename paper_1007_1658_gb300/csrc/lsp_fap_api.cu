// lsp_fap_api.cu -- C ABI of the learned false-alarm surrogate (lsp_fap_*).
//
// Features of sampling patterns (spectral window + cadence statistics, all on
// the GPU), a 32 -> H -> H -> H -> 9 network trained on the GPU by the
// library's own forward, backward and Adam kernels, inference, and a
// checkpoint format (header, FP32 weights, Adam moments, step, checksum).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "lsp_ctx.h"

using namespace lsp::host;

namespace {

constexpr int kNFeat = 32, kNLev = 9;

lsp_status need_model(lsp_ctx* ctx) {
    return ctx->fap.ready ? LSP_OK : fail(ctx, LSP_ERR_NO_MODEL, "surrogate not initialized (lsp_fap_init/load)");
}

// Output staging: device pointer as is, else a context buffer copied back later.
template <class T>
lsp_status out_view(lsp_ctx* ctx, T* dst, size_t n, DevBuf& buf, T** d, bool* host) {
    bool dev = false;
    lsp_status ws = where(ctx, dst, &dev);
    if (ws != LSP_OK) return ws;
    *host = !dev;
    if (!*host) {
        *d = dst;
        return LSP_OK;
    }
    lsp_status st = ensure(ctx, buf, n * sizeof(T) + 16);
    if (st != LSP_OK) return st;
    *d = (T*)buf.p;
    return LSP_OK;
}

uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

lsp_status fap_alloc(lsp_ctx* ctx, int H) {
    FapState& f = ctx->fap;
    f.H = H;
    f.n_params = lsp::mlp_param_count(H);
    const size_t nb = (size_t)f.n_params * 4;
    lsp_status st;
    if ((st = ensure(ctx, f.params, nb)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.grad, nb)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.m, nb)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.v, nb)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.mu_sig, 2 * kNFeat * 4)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.loss, 64)) != LSP_OK) return st;
    return LSP_OK;
}

lsp_status fap_batch_buffers(lsp_ctx* ctx, int B) {
    FapState& f = ctx->fap;
    lsp_status st;
    if ((st = ensure(ctx, f.ws, lsp::mlp_workspace_floats(f.H, B) * 4)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.act, lsp::mlp_act_bytes(f.H, B, true))) != LSP_OK) return st;
    if ((st = ensure(ctx, f.X, (size_t)B * kNFeat * 4)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.cnt, (size_t)B * 2 * 4)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.y, (size_t)B * 4)) != LSP_OK) return st;
    if ((st = ensure(ctx, f.q, (size_t)B * kNLev * 4)) != LSP_OK) return st;
    return LSP_OK;
}

// Gather B rows (rows == null: the first B) into X, cnt, y; run the network.
lsp_status fap_run(lsp_ctx* ctx, int B, const int32_t* rows, int n_pat, const float* feat, const float* counts,
                   const float* targets, bool want_grad, float** q_dev) {
    FapState& f = ctx->fap;
    lsp_status st = fap_batch_buffers(ctx, B);
    if (st != LSP_OK) return st;
    const float* mu = (const float*)f.mu_sig.p;
    LSP_CUDA(ctx, lsp::mlp_gather(B, rows, n_pat, feat, counts, targets, mu, mu + kNFeat, (float*)f.X.p,
                                  (float*)f.cnt.p, (float*)f.y.p, ctx->stream));
    LSP_CUDA(ctx, lsp::mlp_forward_backward(f.H, B, ctx->opt.mlp_fp32 != 0, (const float*)f.params.p,
                                            (const float*)f.X.p, (const float*)f.cnt.p,
                                            targets ? (const float*)f.y.p : nullptr, (float*)f.q.p,
                                            want_grad ? (float*)f.grad.p : nullptr, (float*)f.loss.p,
                                            (float*)f.ws.p, f.act.p, ctx->stream));
    if (q_dev) *q_dev = (float*)f.q.p;
    return LSP_OK;
}

lsp_status copy_loss(lsp_ctx* ctx, float* loss_out) {
    if (!loss_out) return LSP_OK;
    bool dev = false;
    lsp_status ws = where(ctx, loss_out, &dev);
    if (ws != LSP_OK) return ws;
    if (dev) {
        LSP_CUDA(ctx, cudaMemcpyAsync(loss_out, ctx->fap.loss.p, 4, cudaMemcpyDeviceToDevice, ctx->stream));
        return LSP_OK;
    }
    LSP_CUDA(ctx, cudaMemcpyAsync(loss_out, ctx->fap.loss.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    return lsp_sync(ctx, -1.0);
}

}  // namespace

extern "C" {

lsp_status lsp_fap_features(lsp_ctx* ctx, int32_t n, const int64_t* t_off, const double* t, const double* f_0,
                            const double* df, const int64_t* N_f, float* features) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n < 1 || n > 65535) return fail(ctx, LSP_ERR_INVALID_ARG, "n_patterns = %d out of range", n);
    if (!t_off || !t || !f_0 || !df || !N_f || !features) return fail(ctx, LSP_ERR_INVALID_ARG, "null pointer");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = ctx->stream;
    lsp_status rs;
    std::vector<int64_t> off, nf;
    std::vector<double> f0v, dfv;
    if ((rs = fetch(ctx, t_off, (size_t)n + 1, off)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, N_f, (size_t)n, nf)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, f_0, (size_t)n, f0v)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, df, (size_t)n, dfv)) != LSP_OK) return rs;
    if (off[0] != 0) return fail(ctx, LSP_ERR_INVALID_ARG, "t_off[0] must be 0");
    std::vector<int64_t> nw(n), woff(n + 1, 0);
    int64_t max_n = 0;
    for (int c = 0; c < n; ++c) {
        const int64_t len = off[c + 1] - off[c];
        if (len < 2 || len >= (int64_t(1) << 31))
            return fail(ctx, LSP_ERR_INVALID_ARG, "pattern %d has %lld samples (2 .. 2^31 - 1 allowed)", c,
                        (long long)len);
        if (nf[c] < 1 || nf[c] >= (int64_t(1) << 31) || !(dfv[c] > 0.0) || !std::isfinite(f0v[c]) ||
            !std::isfinite(dfv[c]) || f0v[c] < 0.0)
            return fail(ctx, LSP_ERR_INVALID_ARG, "grid of pattern %d must have N_f >= 1, df > 0, f_0 >= 0", c);
        const double f_max = f0v[c] + (double)(nf[c] - 1) * dfv[c];
        nw[c] = (int64_t)std::floor(f_max / dfv[c]);
        woff[c + 1] = woff[c] + nw[c];
        max_n = std::max(max_n, len);
    }
    const int64_t total = off[n];
    const int F = 24;
    const int64_t per_block = lsp::freqs_per_block(F);
    const int64_t *d_off, *d_nf;
    const double *d_f0, *d_df, *d_t;
    if ((rs = device_view(ctx, t_off, (size_t)n + 1, ctx->b_off, &d_off)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, N_f, (size_t)n, ctx->b_nf, &d_nf)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, f_0, (size_t)n, ctx->b_f0, &d_f0)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, df, (size_t)n, ctx->b_df, &d_df)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, t, (size_t)total, ctx->b_t, &d_t)) != LSP_OK) return rs;
    FapState& f = ctx->fap;
    if ((rs = ensure(ctx, ctx->b_recA, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_recB, (size_t)total * 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_stats, sizeof(lsp::CurveStats) * (size_t)n)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, ctx->b_head, 16)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.W, (size_t)std::max<int64_t>(1, woff[n]) * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.W_off, (size_t)(n + 1) * 8)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.nw, (size_t)n * 8)) != LSP_OK) return rs;
    float* d_feat = nullptr;
    bool feat_host = false;
    if ((rs = out_view(ctx, features, (size_t)n * kNFeat, ctx->b_maxP, &d_feat, &feat_host)) != LSP_OK) return rs;
    // work list for the window pass, longest pattern first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    std::vector<lsp::BatchItem> items;
    for (int c : order)
        for (int64_t fb = 0; fb < (nw[c] + per_block - 1) / per_block; ++fb) items.push_back({c, 0, (int32_t)fb, 0});
    const size_t item_bytes = items.size() * sizeof(lsp::BatchItem);
    const size_t meta = (size_t)(2 * n + 1) * 8;
    if ((rs = ensure(ctx, ctx->b_items, item_bytes + 16)) != LSP_OK) return rs;
    if (ctx->plan.valid) drop_plan(ctx);  // the batch graph's work list is overwritten here
    if ((rs = ensure_pinned(ctx, item_bytes + meta + 64)) != LSP_OK) return rs;
    LSP_CUDA(ctx, cudaStreamSynchronize(st));
    char* pin = (char*)ctx->pinned;
    std::memcpy(pin, woff.data(), (size_t)(n + 1) * 8);
    std::memcpy(pin + (size_t)(n + 1) * 8, nw.data(), (size_t)n * 8);
    if (!items.empty()) std::memcpy(pin + meta, items.data(), item_bytes);
    LSP_CUDA(ctx, cudaMemcpyAsync(f.W_off.p, pin, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st));
    LSP_CUDA(ctx, cudaMemcpyAsync(f.nw.p, pin + (size_t)(n + 1) * 8, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    if (!items.empty()) LSP_CUDA(ctx, cudaMemcpyAsync(ctx->b_items.p, pin + meta, item_bytes, cudaMemcpyHostToDevice, st));
    LSP_CUDA(ctx, cudaMemsetAsync(ctx->b_head.p, 0, 16, st));
    // phases on the window grid f_m = m df: records with f0 := df
    LSP_CUDA(ctx, lsp::launch_prep_stats(d_t, nullptr, d_off, 0, n, (lsp::CurveStats*)ctx->b_stats.p, ctx->status_d,
                                         nullptr, nullptr, st));
    LSP_CUDA(ctx, lsp::launch_prep_records(d_t, nullptr, d_off, 0, n, max_n, d_df, d_df, 0.0, 0.0,
                                           (const lsp::CurveStats*)ctx->b_stats.p, (uint4*)ctx->b_recA.p,
                                           (float4*)ctx->b_recB.p, nullptr, nullptr, st, nullptr, nullptr,
                                           ctx->status_d));
    if (!items.empty()) {
        const int grid = (int)std::min<int64_t>((int64_t)lsp::window_occupancy(F) * ctx->sms, (int64_t)items.size());
        LSP_CUDA(ctx, lsp::launch_window(F, grid, (const lsp::BatchItem*)ctx->b_items.p, (int)items.size(),
                                         (unsigned*)ctx->b_head.p, d_off, (const int64_t*)f.nw.p,
                                         (const uint4*)ctx->b_recA.p, (const float4*)ctx->b_recB.p, (float*)f.W.p,
                                         (const int64_t*)f.W_off.p, st));
    }
    LSP_CUDA(ctx, lsp::launch_features(n, max_n, d_t, d_off, d_f0, d_df, d_nf, (const float*)f.W.p,
                                       (const int64_t*)f.W_off.p, (const int64_t*)f.nw.p, d_feat, ctx->status_d, st));
    ctx->last_launches = 4;
    if (feat_host) {
        LSP_CUDA(ctx, cudaMemcpyAsync(features, d_feat, (size_t)n * kNFeat * 4, cudaMemcpyDeviceToHost, st));
        return lsp_sync(ctx, -1.0);
    }
    return LSP_OK;
}

lsp_status lsp_fap_init(lsp_ctx* ctx, int32_t hidden, uint64_t seed, int32_t n_rows, const float* features) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    if (hidden == 0) hidden = 256;
    if (hidden < 4 || hidden > 4096 || n_rows < 1 || !features)
        return fail(ctx, LSP_ERR_INVALID_ARG, "hidden in [4, 4096], n_rows >= 1, features required");
    DeviceGuard guard(ctx->device);
    lsp_status rs = fap_alloc(ctx, hidden);
    if (rs != LSP_OK) return rs;
    FapState& f = ctx->fap;
    const float* d_feat;
    if ((rs = device_view(ctx, features, (size_t)n_rows * kNFeat, ctx->b_P, &d_feat)) != LSP_OK) return rs;
    LSP_CUDA(ctx, lsp::mlp_init(hidden, seed, (float*)f.params.p, ctx->stream));
    LSP_CUDA(ctx, cudaMemsetAsync(f.m.p, 0, (size_t)f.n_params * 4, ctx->stream));
    LSP_CUDA(ctx, cudaMemsetAsync(f.v.p, 0, (size_t)f.n_params * 4, ctx->stream));
    float* mu = (float*)f.mu_sig.p;
    LSP_CUDA(ctx, lsp::mlp_feature_stats(n_rows, d_feat, mu, mu + kNFeat, ctx->stream));
    f.step = 0;
    f.ready = true;
    return lsp_sync(ctx, -1.0);
}

lsp_status lsp_fap_train_step(lsp_ctx* ctx, int32_t B, const int32_t* rows, int32_t n_pat, const float* features,
                              const float* counts, const float* targets, float lr, float* loss_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    if (B < 1 || n_pat < 1 || !rows || !features || !counts || !targets || !(lr > 0.f))
        return fail(ctx, LSP_ERR_INVALID_ARG, "bad training-step argument");
    {
        bool d0 = false, d1 = false, d2 = false, d3 = false;
        if ((rs = where(ctx, rows, &d0)) != LSP_OK || (rs = where(ctx, features, &d1)) != LSP_OK ||
            (rs = where(ctx, counts, &d2)) != LSP_OK || (rs = where(ctx, targets, &d3)) != LSP_OK)
            return rs;
        if (!d0 || !d1 || !d2 || !d3) return fail(ctx, LSP_ERR_INVALID_ARG, "training tables must be device arrays");
    }
    DeviceGuard guard(ctx->device);
    FapState& f = ctx->fap;
    if ((rs = fap_run(ctx, B, rows, n_pat, features, counts, targets, true, nullptr)) != LSP_OK) return rs;
    f.step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)f.step)), c2 = (float)(1.0 - std::pow(b2, (double)f.step));
    LSP_CUDA(ctx, lsp::mlp_adam(f.n_params, (float*)f.params.p, (const float*)f.grad.p, (float*)f.m.p,
                                (float*)f.v.p, lr, (float)b1, (float)b2, c1, c2, 1e-8f, 0.f, ctx->stream));
    return copy_loss(ctx, loss_out);
}

lsp_status lsp_fap_train(lsp_ctx* ctx, const lsp_train_opts* o) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!o) return fail(ctx, LSP_ERR_INVALID_ARG, "null options");
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    if (o->n_pat < 1 || o->n_rows < 1 || o->n_val_pat < 1 || o->n_val_pat > 65535 || o->n_val_real < 1 ||
        (int64_t)o->n_val_pat * o->n_val_real > (int64_t(1) << 31))
        return fail(ctx, LSP_ERR_INVALID_ARG, "training or validation set size out of range");
    if (o->steps < 1 || o->batch < 1 || o->batch > 65536 || o->warmup_steps < 0 || o->warmup_steps > o->steps ||
        o->eval_every < 0 || o->reserved0 != 0)
        return fail(ctx, LSP_ERR_INVALID_ARG, "steps >= 1, batch in [1, 65536], warmup in [0, steps], eval_every >= 0");
    if (!(o->lr > 0.f) || !std::isfinite(o->lr) || !(o->lr_final >= 0.f && o->lr_final <= 1.f) ||
        !(o->weight_decay >= 0.f) || !std::isfinite(o->weight_decay))
        return fail(ctx, LSP_ERR_INVALID_ARG, "lr > 0, lr_final in [0, 1], weight_decay >= 0");
    const void* tables[] = {o->features, o->counts, o->targets, o->val_features, o->val_counts, o->val_targets};
    for (const void* p : tables) {
        bool dev = false;
        if (!p) return fail(ctx, LSP_ERR_INVALID_ARG, "null training table");
        if ((rs = where(ctx, p, &dev)) != LSP_OK) return rs;
        if (!dev) return fail(ctx, LSP_ERR_INVALID_ARG, "training tables must be device arrays");
    }
    bool vh_dev = false, th_dev = false;
    if (o->val_history && (rs = where(ctx, o->val_history, &vh_dev)) != LSP_OK) return rs;
    if (o->train_history && (rs = where(ctx, o->train_history, &th_dev)) != LSP_OK) return rs;
    DeviceGuard guard(ctx->device);
    FapState& f = ctx->fap;
    cudaStream_t st = ctx->stream;
    const int B = o->batch, V = o->n_val_pat;
    const int passes = o->eval_every > 0 ? 2 + (o->steps - 1) / o->eval_every : 2;
    if ((rs = fap_batch_buffers(ctx, std::max(B, V))) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.rows, (size_t)B * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.best, (size_t)f.n_params * 4)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.train_state, 64)) != LSP_OK) return rs;
    if ((rs = ensure(ctx, f.hist, (size_t)passes * 2 * 4)) != LSP_OK) return rs;
    float* ts = (float*)f.train_state.p;  // {val, best loss, best step, acc sum, acc count, flag}
    float* val = ts;
    float* state = ts + 1;
    float* acc = ts + 3;
    int* flag = (int*)(ts + 5);
    float* vhist = (float*)f.hist.p;
    float* thist = vhist + passes;
    LSP_CUDA(ctx, cudaMemsetAsync(ts, 0, 64, st));
    LSP_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
    int e = 0;
    auto validate = [&](int step) -> lsp_status {
        float* q = nullptr;
        lsp_status r = fap_run(ctx, V, nullptr, V, o->val_features, o->val_counts, nullptr, false, &q);
        if (r != LSP_OK) return r;
        LSP_CUDA(ctx, lsp::train_pinball(q, o->val_targets, V, o->n_val_real, val, st));
        LSP_CUDA(ctx, lsp::train_keep_best(val, state, step, flag, acc, vhist, thist, e, (const float*)f.params.p,
                                           (float*)f.best.p, f.n_params, st));
        ++e;
        return LSP_OK;
    };
    if ((rs = validate(0)) != LSP_OK) return rs;
    const double b1 = 0.9, b2 = 0.999, pi = 3.14159265358979323846;
    for (int s = 0; s < o->steps; ++s) {
        double lr;
        if (s < o->warmup_steps) {
            lr = (double)o->lr * (double)(s + 1) / (double)o->warmup_steps;
        } else {
            const double span = (double)std::max(1, o->steps - o->warmup_steps);
            const double c = 0.5 * (1.0 + std::cos(pi * (double)(s - o->warmup_steps) / span));
            lr = (double)o->lr * ((double)o->lr_final + (1.0 - (double)o->lr_final) * c);
        }
        LSP_CUDA(ctx, lsp::train_draw_rows(o->seed, (uint32_t)s, B, (uint32_t)o->n_rows, (int32_t*)f.rows.p, st));
        if ((rs = fap_run(ctx, B, (const int32_t*)f.rows.p, o->n_pat, o->features, o->counts, o->targets, true,
                          nullptr)) != LSP_OK)
            return rs;
        LSP_CUDA(ctx, lsp::train_accum_loss((const float*)f.loss.p, acc, st));
        f.step += 1;
        const float c1 = (float)(1.0 - std::pow(b1, (double)f.step));
        const float c2 = (float)(1.0 - std::pow(b2, (double)f.step));
        LSP_CUDA(ctx, lsp::mlp_adam(f.n_params, (float*)f.params.p, (const float*)f.grad.p, (float*)f.m.p,
                                    (float*)f.v.p, (float)lr, (float)b1, (float)b2, c1, c2, 1e-8f, o->weight_decay,
                                    st));
        const bool last = s + 1 == o->steps;
        if (last || (o->eval_every > 0 && (s + 1) % o->eval_every == 0))
            if ((rs = validate(s + 1)) != LSP_OK) return rs;
    }
    // the kept weights become the network
    LSP_CUDA(ctx, cudaMemcpyAsync(f.params.p, f.best.p, (size_t)f.n_params * 4, cudaMemcpyDeviceToDevice, st));
    LSP_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    float host_ts[6] = {0, 0, 0, 0, 0, 0};
    std::vector<float> hh((size_t)passes * 2);
    LSP_CUDA(ctx, cudaMemcpyAsync(host_ts, ts, sizeof host_ts, cudaMemcpyDeviceToHost, st));
    LSP_CUDA(ctx, cudaMemcpyAsync(hh.data(), vhist, hh.size() * 4, cudaMemcpyDeviceToHost, st));
    if (o->val_history)
        LSP_CUDA(ctx, cudaMemcpyAsync(o->val_history, vhist, (size_t)e * 4,
                                      vh_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (o->train_history)
        LSP_CUDA(ctx, cudaMemcpyAsync(o->train_history, thist, (size_t)e * 4,
                                      th_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if ((rs = lsp_sync(ctx, -1.0)) != LSP_OK) return rs;
    if (o->report) {
        float ms = 0.f;
        LSP_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        lsp_train_report& r = *o->report;
        r.best_step = (int32_t)host_ts[2];
        r.evaluations = e;
        r.val_loss_initial = hh[0];
        r.val_loss_best = host_ts[1];
        r.train_loss_last = hh[(size_t)passes + (size_t)e - 1];
        r.gpu_ms = ms;
    }
    ctx->timing_valid = false;
    return LSP_OK;
}

lsp_status lsp_fap_gradients(lsp_ctx* ctx, int32_t B, const float* features, const float* counts,
                             const float* targets, float* grad_out, float* loss_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    if (B < 1 || !features || !counts || !targets || !grad_out) return fail(ctx, LSP_ERR_INVALID_ARG, "bad argument");
    DeviceGuard guard(ctx->device);
    FapState& f = ctx->fap;
    const float *d_feat, *d_cnt, *d_y;
    if ((rs = device_view(ctx, features, (size_t)B * kNFeat, ctx->b_P, &d_feat)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, counts, (size_t)B * 2, ctx->b_X, (const float**)&d_cnt)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, targets, (size_t)B, ctx->b_xr, &d_y)) != LSP_OK) return rs;
    if ((rs = fap_run(ctx, B, nullptr, B, d_feat, d_cnt, d_y, true, nullptr)) != LSP_OK) return rs;
    bool g_dev = false;
    if ((rs = where(ctx, grad_out, &g_dev)) != LSP_OK) return rs;
    const cudaMemcpyKind k = g_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LSP_CUDA(ctx, cudaMemcpyAsync(grad_out, f.grad.p, (size_t)f.n_params * 4, k, ctx->stream));
    if (k == cudaMemcpyDeviceToHost) LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return copy_loss(ctx, loss_out);
}

lsp_status lsp_fap_eval(lsp_ctx* ctx, int32_t B, const float* features, const float* counts, float* q_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    if (B < 1 || !features || !counts || !q_out) return fail(ctx, LSP_ERR_INVALID_ARG, "bad argument");
    DeviceGuard guard(ctx->device);
    const float *d_feat, *d_cnt;
    if ((rs = device_view(ctx, features, (size_t)B * kNFeat, ctx->b_P, &d_feat)) != LSP_OK) return rs;
    if ((rs = device_view(ctx, counts, (size_t)B * 2, ctx->b_X, (const float**)&d_cnt)) != LSP_OK) return rs;
    float* q = nullptr;
    if ((rs = fap_run(ctx, B, nullptr, B, d_feat, d_cnt, nullptr, false, &q)) != LSP_OK) return rs;
    bool dev = false;
    if ((rs = where(ctx, q_out, &dev)) != LSP_OK) return rs;
    LSP_CUDA(ctx, cudaMemcpyAsync(q_out, q, (size_t)B * kNLev * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  ctx->stream));
    return dev ? LSP_OK : lsp_sync(ctx, -1.0);
}

lsp_status lsp_fap_predict(lsp_ctx* ctx, int32_t n, const int64_t* t_off, const double* t, const double* f_0,
                           const double* df, const int64_t* N_f, float* quantiles_out) {
    if (!ctx) return LSP_ERR_INVALID_ARG;
    ctx->err.clear();
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    if (!quantiles_out) return fail(ctx, LSP_ERR_INVALID_ARG, "null output");
    DeviceGuard guard(ctx->device);
    FapState& f = ctx->fap;
    if ((rs = ensure(ctx, f.counts, (size_t)n * 2 * 4 + (size_t)n * kNFeat * 4)) != LSP_OK) return rs;
    float* d_cnt = (float*)f.counts.p;
    float* d_feat = d_cnt + 2 * (size_t)n;
    if ((rs = lsp_fap_features(ctx, n, t_off, t, f_0, df, N_f, d_feat)) != LSP_OK) return rs;
    std::vector<int64_t> off, nf;
    if ((rs = fetch(ctx, t_off, (size_t)n + 1, off)) != LSP_OK) return rs;
    if ((rs = fetch(ctx, N_f, (size_t)n, nf)) != LSP_OK) return rs;
    std::vector<float> cnt(2 * (size_t)n);
    for (int c = 0; c < n; ++c) {
        if (off[c + 1] - off[c] < 4) return fail(ctx, LSP_ERR_INVALID_ARG, "Eq. 3 needs N_t >= 4 (pattern %d)", c);
        cnt[2 * c] = (float)(off[c + 1] - off[c]);
        cnt[2 * c + 1] = (float)nf[c];
    }
    if ((rs = ensure_pinned(ctx, cnt.size() * 4 + 64)) != LSP_OK) return rs;
    LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::memcpy(ctx->pinned, cnt.data(), cnt.size() * 4);
    LSP_CUDA(ctx, cudaMemcpyAsync(d_cnt, ctx->pinned, cnt.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    return lsp_fap_eval(ctx, n, d_feat, d_cnt, quantiles_out);
}

lsp_status lsp_fap_get_params(lsp_ctx* ctx, float* out, int64_t capacity, int64_t* n_out) {
    if (!ctx || !n_out) return LSP_ERR_INVALID_ARG;
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    FapState& f = ctx->fap;
    *n_out = f.n_params + 2 * kNFeat;
    if (!out) return LSP_OK;
    if (capacity < *n_out) return fail(ctx, LSP_ERR_INVALID_ARG, "capacity %lld < %lld", (long long)capacity,
                                       (long long)*n_out);
    DeviceGuard guard(ctx->device);
    LSP_CUDA(ctx, cudaMemcpyAsync(out, f.params.p, (size_t)f.n_params * 4, cudaMemcpyDefault, ctx->stream));
    LSP_CUDA(ctx, cudaMemcpyAsync(out + f.n_params, f.mu_sig.p, 2 * kNFeat * 4, cudaMemcpyDefault, ctx->stream));
    LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LSP_OK;
}

lsp_status lsp_fap_set_params(lsp_ctx* ctx, int32_t hidden, const float* in, int64_t n) {
    if (!ctx || !in) return LSP_ERR_INVALID_ARG;
    if (hidden == 0) hidden = 256;
    if (hidden < 4 || hidden > 4096 || n != lsp::mlp_param_count(hidden) + 2 * kNFeat)
        return fail(ctx, LSP_ERR_INVALID_ARG, "parameter count does not match hidden = %d", hidden);
    DeviceGuard guard(ctx->device);
    lsp_status rs = fap_alloc(ctx, hidden);
    if (rs != LSP_OK) return rs;
    FapState& f = ctx->fap;
    LSP_CUDA(ctx, cudaMemcpyAsync(f.params.p, in, (size_t)f.n_params * 4, cudaMemcpyDefault, ctx->stream));
    LSP_CUDA(ctx, cudaMemcpyAsync(f.mu_sig.p, in + f.n_params, 2 * kNFeat * 4, cudaMemcpyDefault, ctx->stream));
    LSP_CUDA(ctx, cudaMemsetAsync(f.m.p, 0, (size_t)f.n_params * 4, ctx->stream));
    LSP_CUDA(ctx, cudaMemsetAsync(f.v.p, 0, (size_t)f.n_params * 4, ctx->stream));
    LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    f.step = 0;
    f.ready = true;
    return LSP_OK;
}

// Checkpoint: "LSPFAP01", int32 hidden, int64 step, int64 n_params, then
// params, mu/sigma, Adam m, Adam v (FP32), then an FNV-1a 64-bit checksum of
// everything before it.
lsp_status lsp_fap_save(lsp_ctx* ctx, const char* path) {
    if (!ctx || !path) return LSP_ERR_INVALID_ARG;
    lsp_status rs = need_model(ctx);
    if (rs != LSP_OK) return rs;
    DeviceGuard guard(ctx->device);
    FapState& f = ctx->fap;
    const size_t np = (size_t)f.n_params;
    std::vector<float> buf(np * 3 + 2 * kNFeat);
    LSP_CUDA(ctx, cudaMemcpyAsync(buf.data(), f.params.p, np * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LSP_CUDA(ctx, cudaMemcpyAsync(buf.data() + np, f.mu_sig.p, 2 * kNFeat * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LSP_CUDA(ctx, cudaMemcpyAsync(buf.data() + np + 2 * kNFeat, f.m.p, np * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LSP_CUDA(ctx, cudaMemcpyAsync(buf.data() + 2 * np + 2 * kNFeat, f.v.p, np * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LSP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(ctx, LSP_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const char magic[8] = {'L', 'S', 'P', 'F', 'A', 'P', '0', '1'};
    const int32_t H = f.H;
    const int64_t step = f.step, n = f.n_params;
    uint64_t h = 14695981039346656037ull;
    h = fnv1a(magic, 8, h);
    h = fnv1a(&H, 4, h);
    h = fnv1a(&step, 8, h);
    h = fnv1a(&n, 8, h);
    h = fnv1a(buf.data(), buf.size() * 4, h);
    bool ok = std::fwrite(magic, 8, 1, fp) == 1 && std::fwrite(&H, 4, 1, fp) == 1 && std::fwrite(&step, 8, 1, fp) == 1 &&
              std::fwrite(&n, 8, 1, fp) == 1 && std::fwrite(buf.data(), 4, buf.size(), fp) == buf.size() &&
              std::fwrite(&h, 8, 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LSP_OK : fail(ctx, LSP_ERR_INVALID_ARG, "write to %s failed", path);
}

lsp_status lsp_fap_load(lsp_ctx* ctx, const char* path) {
    if (!ctx || !path) return LSP_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(ctx, LSP_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int32_t H = 0;
    int64_t step = 0, n = 0;
    uint64_t stored = 0;
    bool ok = std::fread(magic, 8, 1, fp) == 1 && std::memcmp(magic, "LSPFAP01", 8) == 0 &&
              std::fread(&H, 4, 1, fp) == 1 && std::fread(&step, 8, 1, fp) == 1 && std::fread(&n, 8, 1, fp) == 1 &&
              H >= 4 && H <= 4096 && n == lsp::mlp_param_count(H) && step >= 0;
    std::vector<float> buf;
    if (ok) {
        buf.resize((size_t)n * 3 + 2 * kNFeat);
        ok = std::fread(buf.data(), 4, buf.size(), fp) == buf.size() && std::fread(&stored, 8, 1, fp) == 1;
    }
    std::fclose(fp);
    if (!ok) return fail(ctx, LSP_ERR_INVALID_ARG, "%s is not a surrogate checkpoint", path);
    uint64_t h = 14695981039346656037ull;
    h = fnv1a(magic, 8, h);
    h = fnv1a(&H, 4, h);
    h = fnv1a(&step, 8, h);
    h = fnv1a(&n, 8, h);
    h = fnv1a(buf.data(), buf.size() * 4, h);
    if (h != stored) return fail(ctx, LSP_ERR_INVALID_ARG, "%s: checksum mismatch", path);
    lsp_status rs = fap_alloc(ctx, H);
    if (rs != LSP_OK) return rs;
    FapState& f = ctx->fap;
    const size_t np = (size_t)n;
    LSP_CUDA(ctx, cudaMemcpy(f.params.p, buf.data(), np * 4, cudaMemcpyHostToDevice));
    LSP_CUDA(ctx, cudaMemcpy(f.mu_sig.p, buf.data() + np, 2 * kNFeat * 4, cudaMemcpyHostToDevice));
    LSP_CUDA(ctx, cudaMemcpy(f.m.p, buf.data() + np + 2 * kNFeat, np * 4, cudaMemcpyHostToDevice));
    LSP_CUDA(ctx, cudaMemcpy(f.v.p, buf.data() + 2 * np + 2 * kNFeat, np * 4, cudaMemcpyHostToDevice));
    f.step = step;
    f.ready = true;
    return LSP_OK;
}

}  // extern "C"
