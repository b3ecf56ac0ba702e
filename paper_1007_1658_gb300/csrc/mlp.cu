// mlp.cu -- kernels of the false-alarm surrogate's network: 32 -> H -> H -> H
// -> 9, exact-erf GELU, activations stored in BF16 (or FP32) with FP32 master
// weights, a quantile head on top of Eq. 3's quantiles trained with the
// pinball loss, and Adam (Kingma & Ba 2015).
//
// The GEMMs are tiny (B x 256 x 256), so one tiled SIMT kernel serves every
// product of the forward and backward passes: 64x64 output tiles, K steps of
// 16 through shared memory, 4x4 outputs per thread, FP32 accumulation, any
// operand strides (so transposed operands need no copies), and three
// epilogues (plain store; bias + GELU with the pre-activation kept for the
// backward pass; multiply by GELU'(pre-activation)).
#include <cuda_bf16.h>

#include "lsp_kernels.cuh"

namespace lsp {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, kGemmThreads = 256;

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ void store_act(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_act(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C(m,n) = sum_k A(m,k) B(k,n), A(m,k) = A[m*sAm + k*sAk], B(k,n) = B[k*sBk + n*sBn].
// EPI 0: C[m*ldc+n] = acc (+ bias[n] if bias)
// EPI 1: Z = acc + bias[n]; C[m*ldc+n] = Z; D[m*ldc+n] = GELU(Z)
// EPI 2: C[m*ldc+n] = acc * GELU'(Zs[m*ldc+n])
template <typename TA, typename TB, typename TD, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int64_t sAm, int64_t sAk, const TB* __restrict__ B,
            int64_t sBk, int64_t sBn, const float* __restrict__ bias, float* __restrict__ C, int64_t ldc,
            TD* __restrict__ D, const float* __restrict__ Zs) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tm = tid / 16, tn = tid % 16;  // 16 x 16 threads, 4 x 4 outputs each
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = tid; i < BM * BK; i += kGemmThreads) {
            const int mm = i / BK, kk = i % BK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? to_f(A[(int64_t)gm * sAm + (int64_t)gk * sAk]) : 0.f;
        }
        for (int i = tid; i < BN * BK; i += kGemmThreads) {
            const int nn = i % BN, kk = i / BN;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < K) ? to_f(B[(int64_t)gk * sBk + (int64_t)gn * sBn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tm * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tn * 4 + j;
            if (gn >= N) continue;
            const int64_t o = (int64_t)gm * ldc + gn;
            float v = acc[i][j];
            if (EPI == 0) {
                if (bias) v += bias[gn];
                C[o] = v;
            } else if (EPI == 1) {
                v += bias[gn];
                C[o] = v;
                store_act(&D[o], gelu(v));
            } else {
                C[o] = v * gelu_grad(Zs[o]);
            }
        }
    }
}

// Gather B rows: X = (features[row % n_pat] - mu) / sigma, counts, y[row].
__global__ void gather_kernel(int Bn, const int32_t* __restrict__ rows, int n_pat, const float* __restrict__ feat,
                              const float* __restrict__ counts, const float* __restrict__ y,
                              const float* __restrict__ mu, const float* __restrict__ sig, float* __restrict__ X,
                              float* __restrict__ cnt, float* __restrict__ yy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bn * 32) return;
    const int r = i / 32, f = i % 32;
    const int row = rows ? rows[r] : r;
    const int p = row % n_pat;
    X[i] = (feat[(int64_t)p * 32 + f] - mu[f]) / sig[f];
    if (f < 2) cnt[r * 2 + f] = counts[(int64_t)p * 2 + f];
    if (f == 0 && yy) yy[r] = y ? y[row] : 0.f;
}

__constant__ float kLevels[9] = {0.05f, 0.10f, 0.25f, 0.50f, 0.75f, 0.90f, 0.95f, 0.98f, 0.99f};

__device__ __forceinline__ float softplusf(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// Quantile head.  With e_l = log q_l^Eq3(N, N_f) and d_l = e_l - e_{l-1} > 0
// (Eq. 3's log-spacing): log q_1 = e_1 + z_1, log q_l = log q_{l-1} +
// d_l softplus(z_l) / log 2.  Monotone in l for any z; z = 0 gives Eq. 3's
// quantiles exactly.  With targets: per-row pinball loss
// sum_l max(p u, (p-1) u), u = y - q_l, and dz = d(mean loss)/dz.
__global__ void head_kernel(int Bn, const float* __restrict__ z, const float* __restrict__ cnt,
                            const float* __restrict__ y, float* __restrict__ q, float* __restrict__ loss_row,
                            float* __restrict__ dz) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bn) return;
    const float N = cnt[r * 2], Nf = cnt[r * 2 + 1];
    const float inv_ln2 = 1.4426950408889634f;
    float qq[9], zz[9], d[9], e_prev = 0.f, lq = 0.f;
    for (int l = 0; l < 9; ++l) {
        zz[l] = z[r * 9 + l];
        const float a = -expm1f(logf(kLevels[l]) / Nf);
        const float e = logf(0.5f * N) + logf(-expm1f(2.f / (N - 3.f) * logf(a)));
        if (l == 0) {
            d[0] = 0.f;
            lq = e + zz[0];
        } else {
            d[l] = e - e_prev;
            lq += d[l] * softplusf(zz[l]) * inv_ln2;
        }
        e_prev = e;
        qq[l] = expf(lq);
        if (q) q[r * 9 + l] = qq[l];
    }
    if (!y) return;
    const float yy = y[r];
    float L = 0.f, dl[9];
    for (int l = 0; l < 9; ++l) {
        const float p = kLevels[l], u = yy - qq[l];
        L += fmaxf(p * u, (p - 1.f) * u);
        dl[l] = (u > 0.f ? -p : 1.f - p) / (float)Bn * qq[l];
    }
    loss_row[r] = L;
    float tail = 0.f;
    for (int l = 8; l >= 0; --l) {
        tail += dl[l];
        dz[r * 9 + l] = l == 0 ? tail : tail * d[l] * sigmoidf_(zz[l]) * inv_ln2;
    }
}

// Column sums of a rows x cols matrix (bias gradients), fixed order per column.
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ G, float* __restrict__ out) {
    const int c = blockIdx.x;
    __shared__ float sh[256];
    float s = 0.f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s += G[(int64_t)r * cols + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

// Mean of n values (one CTA, fixed order).
__global__ void mean_kernel(int n, const float* __restrict__ v, float* __restrict__ out) {
    __shared__ float sh[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (float)n;
}

// Adam with bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t, and
// decoupled weight decay wd (Loshchilov & Hutter 2019; wd = 0: plain Adam).
__global__ void adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps,
                            float wd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i];
    p[i] = pi - lr * (mi / c1) / (sqrtf(vi / c2) + eps) - (wd != 0.f ? lr * wd * pi : 0.f);
}

// Column mean and population standard deviation of n x 32 features (FP64 sums).
__global__ void feat_stats_kernel(int n, const float* __restrict__ feat, float* __restrict__ mu,
                                  float* __restrict__ sig) {
    const int f = blockIdx.x;
    __shared__ double sh[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += feat[(int64_t)r * 32 + f];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = sh[0] / n;
    __syncthreads();
    double v = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double d = feat[(int64_t)r * 32 + f] - mean;
        v += d * d;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mu[f] = (float)mean;
        const double sd = sqrt(sh[0] / n);
        sig[f] = sd > 1e-6 ? (float)sd : 1.f;  // a constant feature passes through unscaled
    }
}

__global__ void scale_kernel(int64_t n, float* __restrict__ p, float s) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] *= s;
}

template <typename TA, typename TB, typename TD, int EPI>
cudaError_t gemm(int M, int N, int K, const TA* A, int64_t sAm, int64_t sAk, const TB* B, int64_t sBk,
                 int64_t sBn, const float* bias, float* C, int64_t ldc, TD* D, const float* Zs, cudaStream_t st) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_kernel<TA, TB, TD, EPI><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, sAm, sAk, B, sBk, sBn, bias, C, ldc, D, Zs);
    return cudaGetLastError();
}

}  // namespace

// Parameter layout (flat FP32): W1[32][H] b1[H] W2[H][H] b2[H] W3[H][H] b3[H] W4[H][9] b4[9].
int64_t mlp_param_count(int H) { return 32LL * H + H + 2LL * ((int64_t)H * H + H) + 9LL * H + 9; }

static void offsets(int H, int64_t o[8]) {
    const int64_t s[8] = {32LL * H, H, (int64_t)H * H, H, (int64_t)H * H, H, 9LL * H, 9};
    int64_t a = 0;
    for (int i = 0; i < 8; ++i) {
        o[i] = a;
        a += s[i];
    }
}

cudaError_t mlp_init(int H, uint64_t seed, float* params, cudaStream_t st) {
    int64_t o[8];
    offsets(H, o);
    const int64_t n = mlp_param_count(H);
    cudaError_t e = cudaMemsetAsync(params, 0, (size_t)n * 4, st);
    // He-normal hidden layers; the output layer stays zero, so an untrained
    // network predicts Eq. 3's quantiles exactly
    const int fan[3] = {32, H, H};
    const int64_t sz[3] = {32LL * H, (int64_t)H * H, (int64_t)H * H};
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        e = launch_noise_raw(seed, 0x5EED0000u + l, 0u, sz[l], params + o[2 * l], st);
        if (e == cudaSuccess) {
            const float s = sqrtf(2.f / (float)fan[l]);
            scale_kernel<<<(unsigned)((sz[l] + 255) / 256), 256, 0, st>>>(sz[l], params + o[2 * l], s);
            e = cudaGetLastError();
        }
    }
    return e;
}

cudaError_t mlp_feature_stats(int n, const float* feat, float* mu, float* sig, cudaStream_t st) {
    feat_stats_kernel<<<32, 256, 0, st>>>(n, feat, mu, sig);
    return cudaGetLastError();
}

cudaError_t mlp_gather(int Bn, const int32_t* rows, int n_pat, const float* feat, const float* counts, const float* y,
                       const float* mu, const float* sig, float* X, float* cnt, float* yy, cudaStream_t st) {
    gather_kernel<<<(Bn * 32 + 255) / 256, 256, 0, st>>>(Bn, rows, n_pat, feat, counts, y, mu, sig, X, cnt, yy);
    return cudaGetLastError();
}

// Forward (and with y, loss + backward into grad).  Workspace layout in `ws`
// (floats): Z[3][B][H], dZ[2][B][H], zo[B][9], dzo[B][9], loss_row[B]; acts
// in `act` (3 x B x H, BF16 or FP32 by `fp32`).
template <typename TD>
static cudaError_t mlp_run(int H, int Bn, const float* params, const float* X, const float* cnt, const float* y,
                           float* q, float* grad, float* loss, float* ws, TD* act, cudaStream_t st) {
    int64_t o[8];
    offsets(H, o);
    const int64_t BH = (int64_t)Bn * H;
    float* Z[3] = {ws, ws + BH, ws + 2 * BH};
    float* dZ[2] = {ws + 3 * BH, ws + 4 * BH};
    float* zo = ws + 5 * BH;
    float* dzo = zo + (int64_t)Bn * 9;
    float* lrow = dzo + (int64_t)Bn * 9;
    TD* Aa[3] = {act, act + BH, act + 2 * BH};
    const float* W[4] = {params + o[0], params + o[2], params + o[4], params + o[6]};
    const float* b[4] = {params + o[1], params + o[3], params + o[5], params + o[7]};
    cudaError_t e;
    e = gemm<float, float, TD, 1>(Bn, H, 32, X, 32, 1, W[0], H, 1, b[0], Z[0], H, Aa[0], nullptr, st);
    for (int l = 1; l < 3 && e == cudaSuccess; ++l)
        e = gemm<TD, float, TD, 1>(Bn, H, H, Aa[l - 1], H, 1, W[l], H, 1, b[l], Z[l], H, Aa[l], nullptr, st);
    if (e == cudaSuccess)
        e = gemm<TD, float, float, 0>(Bn, 9, H, Aa[2], H, 1, W[3], 9, 1, b[3], zo, 9, (float*)nullptr, nullptr, st);
    if (e != cudaSuccess) return e;
    head_kernel<<<(Bn + 127) / 128, 128, 0, st>>>(Bn, zo, cnt, y, q, lrow, dzo);
    if ((e = cudaGetLastError()) != cudaSuccess || !y) return e;
    mean_kernel<<<1, 256, 0, st>>>(Bn, lrow, loss);
    if ((e = cudaGetLastError()) != cudaSuccess || !grad) return e;
    float* gW[4] = {grad + o[0], grad + o[2], grad + o[4], grad + o[6]};
    float* gb[4] = {grad + o[1], grad + o[3], grad + o[5], grad + o[7]};
    // output layer
    e = gemm<TD, float, float, 0>(H, 9, Bn, Aa[2], 1, H, dzo, 9, 1, nullptr, gW[3], 9, (float*)nullptr, nullptr, st);
    if (e == cudaSuccess) {
        colsum_kernel<<<9, 256, 0, st>>>(Bn, 9, dzo, gb[3]);
        e = cudaGetLastError();
    }
    // dZ3 = (dzo W4^T) * gelu'(Z3)
    if (e == cudaSuccess)
        e = gemm<float, float, float, 2>(Bn, H, 9, dzo, 9, 1, W[3], 1, 9, nullptr, dZ[0], H, (float*)nullptr, Z[2], st);
    int cur = 0;
    for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
        // weight gradient: A_{l-1}^T dZ_l (the input X for l = 0)
        if (l > 0)
            e = gemm<TD, float, float, 0>(l == 0 ? 32 : H, H, Bn, Aa[l - 1], 1, H, dZ[cur], H, 1, nullptr, gW[l], H,
                                          (float*)nullptr, nullptr, st);
        else
            e = gemm<float, float, float, 0>(32, H, Bn, X, 1, 32, dZ[cur], H, 1, nullptr, gW[0], H, (float*)nullptr,
                                             nullptr, st);
        if (e != cudaSuccess) break;
        colsum_kernel<<<H, 256, 0, st>>>(Bn, H, dZ[cur], gb[l]);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (l > 0) {
            e = gemm<float, float, float, 2>(Bn, H, H, dZ[cur], H, 1, W[l], 1, H, nullptr, dZ[cur ^ 1], H,
                                             (float*)nullptr, Z[l - 1], st);
            cur ^= 1;
        }
    }
    return e;
}

size_t mlp_workspace_floats(int H, int Bn) { return (size_t)5 * Bn * H + (size_t)Bn * 19 + 64; }
size_t mlp_act_bytes(int H, int Bn, bool fp32) { return (size_t)3 * Bn * H * (fp32 ? 4 : 2); }

cudaError_t mlp_forward_backward(int H, int Bn, bool fp32, const float* params, const float* X, const float* cnt,
                                 const float* y, float* q, float* grad, float* loss, float* ws, void* act,
                                 cudaStream_t st) {
    if (fp32) return mlp_run<float>(H, Bn, params, X, cnt, y, q, grad, loss, ws, (float*)act, st);
    return mlp_run<__nv_bfloat16>(H, Bn, params, X, cnt, y, q, grad, loss, ws, (__nv_bfloat16*)act, st);
}

cudaError_t mlp_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float c1,
                     float c2, float eps, float wd, cudaStream_t st) {
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, c1, c2, eps, wd);
    return cudaGetLastError();
}

}  // namespace lsp
