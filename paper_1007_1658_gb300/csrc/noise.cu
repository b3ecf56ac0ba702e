// noise.cu -- Gaussian noise for Monte-Carlo periodograms (Sec. 6.2: the
// statistics of peak heights under pure noise, e.g. the number of independent
// frequencies behind Eq. 3, are estimated from many noise periodograms).
//
// Sample j of realization r of curve c is drawn from Philox-4x32-10 (Salmon,
// Moraes, Dror & Shaw 2011) with counter (j/4, c, r, 0) and key (seed low,
// seed high): every value is a pure function of (seed, c, r, j), so runs are
// reproducible and resumable.  Each 32-bit word w becomes the uniform
// u = (2 (w >> 9) + 1) 2^-24 in (0, 1) (exact in FP32), and the Box-Muller
// transform (Box & Muller 1958) turns (u0, u1), (u2, u3) into four N(0, 1)
// values: sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).
#include <cfloat>

#include "lsp_kernels.cuh"
#include "philox.cuh"

namespace lsp {
namespace {

constexpr int kNoiseThreads = 256;

using dev::philox4x32_10;

__device__ __forceinline__ float unit_uniform(uint32_t w) { return (float)(2u * (w >> 9) + 1u) * 0x1p-24f; }

// Four N(0,1) values of Philox block `blk` of (curve, real).
__device__ __forceinline__ float4 normals4(uint64_t seed, uint32_t blk, uint32_t curve, uint32_t real) {
    const uint4 w = philox4x32_10(blk, curve, real, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float r0 = sqrtf(-2.f * logf(unit_uniform(w.x)));
    const float r1 = sqrtf(-2.f * logf(unit_uniform(w.z)));
    float s0, c0, s1, c1;
    sincospif(2.f * unit_uniform(w.y), &s0, &c0);
    sincospif(2.f * unit_uniform(w.w), &s1, &c1);
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[32] = r;
    __syncthreads();
    return sh[32];
}

// Raw N(0,1) values of one (curve, realization), samples [0, n).
__global__ void __launch_bounds__(kNoiseThreads)
noise_raw_kernel(uint64_t seed, uint32_t curve, uint32_t real, int64_t n, float* __restrict__ out) {
    const int64_t nb = (n + 3) / 4;
    for (int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < nb;
         blk += (int64_t)gridDim.x * blockDim.x) {
        const float4 z = normals4(seed, (uint32_t)blk, curve, real);
        const int64_t j = blk * 4;
        out[j] = z.x;
        if (j + 1 < n) out[j + 1] = z.y;
        if (j + 2 < n) out[j + 2] = z.z;
        if (j + 3 < n) out[j + 3] = z.w;
    }
}

// One CTA per (curve, realization): draw the noise into xr, then normalize it
// in place to zero mean and unit population variance (Sec. 3), mean and
// variance in FP64 over two passes.
__global__ void __launch_bounds__(kNoiseThreads)
noise_prep_kernel(const int64_t* __restrict__ off, const uint64_t* __restrict__ seed_p, int64_t total,
                  float* __restrict__ xr, float4* __restrict__ recB) {
    __shared__ double sh[33];
    const int c = blockIdx.x, r = blockIdx.y;
    const int64_t b = off[c], n = off[c + 1] - off[c];
    float* x = xr + (size_t)r * (size_t)total + b;
    const uint64_t seed = *seed_p;
    double s = 0.0;
    for (int64_t blk = threadIdx.x; blk * 4 < n; blk += blockDim.x) {
        const float4 z = normals4(seed, (uint32_t)blk, (uint32_t)c, (uint32_t)r);
        const int64_t j = blk * 4;
        x[j] = z.x;
        s += z.x;
        if (j + 1 < n) { x[j + 1] = z.y; s += z.y; }
        if (j + 2 < n) { x[j + 2] = z.z; s += z.z; }
        if (j + 3 < n) { x[j + 3] = z.w; s += z.w; }
    }
    __syncthreads();
    const double mean = block_sum(s, sh) / (double)n;
    double v = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double d = (double)x[j] - mean;
        v = fma(d, d, v);
    }
    const double var = block_sum(v, sh) / (double)n;
    const double inv_sd = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const float xh = (float)(((double)x[j] - mean) * inv_sd);
        x[j] = xh;
        if (recB) recB[b + j].x = xh;  // single realization: straight into the sample records
    }
}

// One CTA per (curve, realization) of the floating-mean Monte Carlo: the
// same N(0,1) draws z_j as noise_prep_kernel, X_j = dy_j z_j (z_j without dy),
// then the weighted normalization of prep_records_kernel's floating-mean form,
// x_j = q_j (X_j - mean_w) / sd_w, with v_j = 1/dy_j^2 formed in FP32 as the
// prep kernels form it, mean_w = sum v X / sum v and the population variance
// sum v (X - mean_w)^2 / sum v in FP64.  X_j is re-formed from the stored z_j
// in every pass (exact: a float times a double).
__global__ void __launch_bounds__(kNoiseThreads)
gls_noise_prep_kernel(const int64_t* __restrict__ off, uint64_t seed, int64_t total, const double* __restrict__ dy,
                      const float* __restrict__ q, float* __restrict__ xr) {
    __shared__ double sh[33];
    const int c = blockIdx.x, r = blockIdx.y;
    const int64_t b = off[c], n = off[c + 1] - off[c];
    float* x = xr + (size_t)r * (size_t)total + b;
    auto weight = [&](int64_t j) {
        if (!dy) return 1.0;
        const float ef = (float)dy[b + j];
        return (double)(1.f / (ef * ef));
    };
    auto value = [&](int64_t j) { return dy ? dy[b + j] * (double)x[j] : (double)x[j]; };
    double sv = 0.0, svx = 0.0;
    for (int64_t blk = threadIdx.x; blk * 4 < n; blk += blockDim.x) {
        const float4 z = normals4(seed, (uint32_t)blk, (uint32_t)c, (uint32_t)r);
        const int64_t j = blk * 4;
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j + u < n) {
                x[j + u] = zz[u];
                const double v = weight(j + u);
                sv += v;
                svx += v * value(j + u);
            }
        }
    }
    __syncthreads();
    sv = block_sum(sv, sh);
    const double mean = block_sum(svx, sh) / sv;
    double m2 = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double d = value(j) - mean;
        m2 = fma(d * weight(j), d, m2);
    }
    const double var = block_sum(m2, sh) / sv;
    const double inv_sd = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
    __syncthreads();
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) x[j] = (float)((value(j) - mean) * inv_sd) * q[b + j];
}

}  // namespace

cudaError_t launch_gls_noise_prep(const int64_t* off, int n_curves, int n_real, uint64_t seed, int64_t total,
                                  const double* dy, const float* q, float* xr, cudaStream_t st) {
    dim3 grid((unsigned)n_curves, (unsigned)n_real);
    gls_noise_prep_kernel<<<grid, kNoiseThreads, 0, st>>>(off, seed, total, dy, q, xr);
    return cudaGetLastError();
}

cudaError_t launch_noise_raw(uint64_t seed, uint32_t curve, uint32_t real, int64_t n, float* out, cudaStream_t st) {
    const int64_t nb = (n + 3) / 4;
    int64_t blocks = (nb + kNoiseThreads - 1) / kNoiseThreads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    noise_raw_kernel<<<(unsigned)blocks, kNoiseThreads, 0, st>>>(seed, curve, real, n, out);
    return cudaGetLastError();
}

cudaError_t launch_noise_prep(const int64_t* off, int n_curves, int n_real, const uint64_t* seed_dev,
                              int64_t total, float* xr, float4* recB, cudaStream_t st) {
    dim3 grid((unsigned)n_curves, (unsigned)n_real);
    noise_prep_kernel<<<grid, kNoiseThreads, 0, st>>>(off, seed_dev, total, xr, n_real == 1 ? recB : nullptr);
    return cudaGetLastError();
}

}  // namespace lsp
