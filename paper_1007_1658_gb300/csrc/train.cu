// train.cu -- device pieces of lsp_fap_train's loop that are not the network
// itself (mlp.cu): minibatch row draws from a Philox stream, the validation
// pinball loss as a fixed-order device reduction, and the selection of the
// weights with the lowest validation loss, so that the loop runs on the
// context's stream without a host round trip per step.
#include <algorithm>

#include "lsp_kernels.cuh"
#include "philox.cuh"

namespace lsp {
namespace {

// The levels of the quantiles the surrogate predicts.
__constant__ float kTrainLevels[9] = {0.05f, 0.10f, 0.25f, 0.50f, 0.75f, 0.90f, 0.95f, 0.98f, 0.99f};

// Rows of minibatch `step`: row i is floor(w n_rows / 2^32) for word i % 4 of
// Philox block (i / 4, step, 0x54524e52, 0) under key (seed low, seed high):
// uniform over [0, n_rows) up to a bias below n_rows / 2^32.
__global__ void draw_rows_kernel(uint64_t seed, uint32_t step, int B, uint32_t n_rows, int32_t* __restrict__ rows) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk * 4 >= B) return;
    const uint4 w = dev::philox4x32_10((uint32_t)blk, step, 0x54524e52u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (blk * 4 + q < B) rows[blk * 4 + q] = (int32_t)__umulhi(ws[q], n_rows);
}

// Mean pinball loss of quantiles q[n_pat][9] against samples y[n_real][n_pat]:
// (1 / (n_real n_pat)) sum_{r,i} sum_l max(p_l u, (p_l - 1) u), u = y[r][i] - q[i][l].
// One CTA; each thread sums a fixed stride in FP64, then a fixed-order tree.
constexpr int kPinThreads = 512;
__global__ void __launch_bounds__(kPinThreads)
pinball_kernel(const float* __restrict__ q, const float* __restrict__ y, int n_pat, int n_real,
               float* __restrict__ out) {
    __shared__ double sh[kPinThreads];
    const int64_t n = (int64_t)n_pat * n_real;
    double s = 0.0;
    for (int64_t idx = threadIdx.x; idx < n; idx += kPinThreads) {
        const int i = (int)(idx % n_pat);
        const float yy = y[idx];
        float L = 0.f;
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            const float p = kTrainLevels[l], u = yy - q[(int64_t)i * 9 + l];
            L += fmaxf(p * u, (p - 1.f) * u);
        }
        s += (double)L;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kPinThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(sh[0] / (double)n);
}

// Running sum of the minibatch losses: acc = {sum, count}.
__global__ void accum_loss_kernel(const float* __restrict__ loss, float* __restrict__ acc) {
    acc[0] += *loss;
    acc[1] += 1.f;
}

// After a validation pass: record it (val_hist[e], train_hist[e] = mean
// minibatch loss since the previous pass), and when it beats the best so far
// take it as the best (st: {best loss, best step as float}) and raise *flag
// so that copy_if_kernel keeps the current weights.
__global__ void keep_best_kernel(const float* __restrict__ val, float* __restrict__ st, int step, int* __restrict__ flag,
                                 float* __restrict__ acc, float* __restrict__ val_hist, float* __restrict__ train_hist,
                                 int e) {
    const float v = *val;
    val_hist[e] = v;
    train_hist[e] = acc[1] > 0.f ? acc[0] / acc[1] : __int_as_float(0x7fc00000);
    acc[0] = acc[1] = 0.f;
    const bool better = e == 0 || v < st[0];
    if (better) {
        st[0] = v;
        st[1] = (float)step;
    }
    *flag = better ? 1 : 0;
}

__global__ void copy_if_kernel(const int* __restrict__ flag, const float* __restrict__ src, float* __restrict__ dst,
                               int64_t n) {
    if (!*flag) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

cudaError_t train_draw_rows(uint64_t seed, uint32_t step, int B, uint32_t n_rows, int32_t* rows, cudaStream_t st) {
    const int blocks = (B + 3) / 4;
    draw_rows_kernel<<<(blocks + 127) / 128, 128, 0, st>>>(seed, step, B, n_rows, rows);
    return cudaGetLastError();
}

cudaError_t train_pinball(const float* q, const float* y, int n_pat, int n_real, float* out, cudaStream_t st) {
    pinball_kernel<<<1, kPinThreads, 0, st>>>(q, y, n_pat, n_real, out);
    return cudaGetLastError();
}

cudaError_t train_accum_loss(const float* loss, float* acc, cudaStream_t st) {
    accum_loss_kernel<<<1, 1, 0, st>>>(loss, acc);
    return cudaGetLastError();
}

cudaError_t train_keep_best(const float* val, float* state, int step, int* flag, float* acc, float* val_hist,
                            float* train_hist, int e, const float* params, float* best, int64_t n, cudaStream_t st) {
    keep_best_kernel<<<1, 1, 0, st>>>(val, state, step, flag, acc, val_hist, train_hist, e);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1024);
    copy_if_kernel<<<(unsigned)blocks, 256, 0, st>>>(flag, params, best, n);
    return cudaGetLastError();
}

}  // namespace lsp
