// prep.cu -- per-curve normalization and per-sample phase records.
//
// The only FP64 arithmetic on the GPU lives here: the mean and population
// variance of X (Sec. 3: the series is shifted to zero mean and scaled to
// unit variance) and the exact fixed-point phases frac(t' df), frac(t' f0)
// that replace the single-precision range reduction of Sec. 4.3.
#include <cfloat>
#include <cmath>

#include "lsp_kernels.cuh"

namespace lsp {
namespace {

constexpr int kStatsThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum / min; the result is valid in every thread.
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

__device__ double block_min(double v, double* sh) {
    v = warp_min(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : DBL_MAX;
    if (w == 0) r = warp_min(r);
    if (threadIdx.x == 0) sh[32] = r;
    __syncthreads();
    return sh[32];
}

// Joins the statistics (weight sum n, mean, M2 = sum w (x - mean)^2) of a
// second group into the first: one division (Chan, Golub & LeVeque 1979).
__device__ __forceinline__ void chan_merge(double& n, double& mean, double& m2, double nb, double mb, double m2b) {
    if (!(nb > 0.0)) return;
    const double nn = n + nb;
    const double r = nb / nn;
    const double d = mb - mean;
    mean += d * r;
    m2 += m2b + d * d * n * r;
    n = nn;
}

// Statistics of one curve, or of one slice of it (G CTAs per curve): t_ref =
// min t, mean and population variance of X (two passes over the slice, FP64),
// non-finite detection.  With G > 1 each CTA leaves (n, mean, M2, min t) of
// its slice and the last CTA to finish merges the G slices in slice order
// (Chan, Golub & LeVeque's pairwise update), so the result does not depend
// on which CTA finishes last.  A degenerate curve gets inv_sd = NaN, so its
// periodogram comes out NaN and the status word says why.
// With per-sample errors dy (floating-mean periodogram) every sample carries
// the weight v = 1/dy^2: the mean and variance are the weighted ones, n
// becomes the weight sum, and a dy that is not finite and > 0 is flagged.
// Without dy every weight is 1 and the arithmetic is the unweighted one.
__global__ void __launch_bounds__(kStatsThreads)
prep_stats_kernel(const double* __restrict__ t, const double* __restrict__ X,
                  const int64_t* __restrict__ off, int64_t n0, CurveStats* __restrict__ stats,
                  int* __restrict__ status, StatPart* __restrict__ parts, unsigned* __restrict__ counters,
                  const double* __restrict__ dy) {
    __shared__ double sh[33];
    __shared__ int last;
    const int c = blockIdx.y, g = blockIdx.x, G = gridDim.x;
    const int64_t b = off ? off[c] : 0;
    const int64_t e = off ? off[c + 1] : n0;
    const int64_t n = e - b;
    const int64_t L = (n + G - 1) / G;
    const int64_t sb = min(e, b + (int64_t)g * L);
    const int64_t se = min(e, sb + L);
    double s = 0.0, tmin = DBL_MAX, ws = 0.0;
    int bad = 0, badw = 0;
#pragma unroll 4
    for (int64_t j = sb + threadIdx.x; j < se; j += blockDim.x) {
        const double x = X ? X[j] : 0.0, tj = t[j];
        bad |= !(isfinite(x) && isfinite(tj));
        if (dy) {
            // weights in FP32 (relative error ~1e-7; FP64 division is slow on this part)
            const double ej = dy[j];
            const float ef = (float)ej;
            const double wj = (double)(1.f / (ef * ef));
            badw |= !(isfinite(ej) && ej > 0.0 && isfinite(wj) && wj > 0.0);
            ws += wj;
            s += wj * x;
        } else {
            s += x;
        }
        tmin = fmin(tmin, tj);
    }
    bad = __syncthreads_or(bad);
    badw = __syncthreads_or(badw);
    s = block_sum(s, sh);
    tmin = block_min(tmin, sh);
    const double cnt = dy ? block_sum(ws, sh) : (double)(se - sb);
    const double mean_g = cnt > 0 ? s / cnt : 0.0;
    double v = 0.0;
    if (X) {
#pragma unroll 4
        for (int64_t j = sb + threadIdx.x; j < se; j += blockDim.x) {
            const double d = X[j] - mean_g;
            if (dy) {
                const float ef = (float)dy[j];
                v = fma(d * (double)(1.f / (ef * ef)), d, v);
            } else {
                v = fma(d, d, v);
            }
        }
    }
    v = block_sum(v, sh);
    bad |= badw << 1;  // bit 1: bad weight
    double tot_n = cnt, mean = mean_g, m2 = v;
    if (G > 1) {
        if (threadIdx.x == 0) {
            StatPart* pp = parts + (size_t)c * G + g;
            pp->n = cnt;
            pp->mean = mean_g;
            pp->m2 = v;
            pp->tmin = tmin;
            pp->bad = bad;
            __threadfence();
            last = atomicAdd(&counters[c], 1u) == (unsigned)(G - 1);
        }
        __syncthreads();
        if (!last) return;
        if (threadIdx.x < 32) {
            // warp 0 merges the G <= kMaxStatSlices slices: lane l takes slices
            // l, l + 32, ... in order, then a fixed shuffle tree joins the lanes
            // (Chan, Golub & LeVeque's update), so the order never depends on
            // which CTA finished last
            __threadfence();
            const int lane = threadIdx.x;
            tot_n = 0.0;
            mean = 0.0;
            m2 = 0.0;
            tmin = DBL_MAX;
            bad = 0;
            const StatPart* pp = parts + (size_t)c * G;
            for (int q = lane; q < G; q += 32) {
                chan_merge(tot_n, mean, m2, __ldcg(&pp[q].n), __ldcg(&pp[q].mean), __ldcg(&pp[q].m2));
                tmin = fmin(tmin, __ldcg(&pp[q].tmin));
                bad |= __ldcg(&pp[q].bad);
            }
            for (int o = 1; o < 32; o <<= 1) {
                const double nb = __shfl_down_sync(0xffffffffu, tot_n, o);
                const double mb = __shfl_down_sync(0xffffffffu, mean, o);
                const double m2b = __shfl_down_sync(0xffffffffu, m2, o);
                const double tb = __shfl_down_sync(0xffffffffu, tmin, o);
                const int bb = __shfl_down_sync(0xffffffffu, bad, o);
                if ((lane & (2 * o - 1)) == 0 && lane + o < 32) {
                    chan_merge(tot_n, mean, m2, nb, mb, m2b);
                    tmin = fmin(tmin, tb);
                    bad |= bb;
                }
            }
            if (lane == 0) counters[c] = 0u;  // ready for the next call
        }
    }
    if (threadIdx.x == 0) {
        // without X (noise drawn later) only t_ref matters: unit scale
        const double var = X ? m2 / (dy ? tot_n : (double)n) : 1.0;
        const bool ok = !bad && var > 0.0 && n >= 2;
        CurveStats r;
        r.mean = mean;
        r.inv_sd = ok ? 1.0 / sqrt(var) : __longlong_as_double(0x7ff8000000000000ll);
        r.t_ref = bad ? 0.0 : tmin;
        r.pad = dy ? tot_n : var;
        stats[c] = r;
        if (bad & 1) atomicOr(status, kStatusNonFinite);
        else if (bad) atomicOr(status, kStatusBadWeight);
        else if (!ok) atomicOr(status, kStatusDegenerate);
    }
}

// frac(a*b) as a 64-bit fixed-point number of turns, exact to ~1 unit of 2^-64:
// the product is split into p + e exactly (Dekker/Ogita-Rump-Oishi TwoProduct
// through fma), floor(p) is removed exactly, and both pieces are scaled by
// 2^64 and added modulo 2^64.  Requires |a*b| < 2^52.
__device__ __forceinline__ uint64_t frac_turns64(double a, double b) {
    const double p = __dmul_rn(a, b);
    const double e = fma(a, b, -p);
    const double fr = p - floor(p);
    const uint64_t U = __double2ull_rn(fr * 0x1p64);
    const int64_t E = __double2ll_rn(e * 0x1p64);
    return U + (uint64_t)E;
}

// cos/sin(2 pi u) of a 64-bit fixed-point turn u (read as signed, so the turn
// is in [-1/2, 1/2)): the top 24 bits go to sincospif as an exact FP32
// argument; the remaining bits (at most 2^-24 turn, an angle d < 3.8e-7 rad)
// enter by the angle-addition formula to first order, cos(a + d) = cos a -
// d sin a, sin(a + d) = sin a + d cos a, whose neglected terms are below
// d^2/2 < 2^-43.  FP32 throughout (FP64 transcendentals are slow here).
__device__ __forceinline__ void rotation_of(uint64_t u, float* c, float* s) {
    const int64_t su = (int64_t)u;
    const int64_t top = su >> 40;  // in [-2^23, 2^23): exact as a float
    const float th = (float)top * 0x1p-24f;
    const float tl = (float)(su - top * (int64_t(1) << 40)) * 0x1p-64f;
    float sh, ch;
    sincospif(2.f * th, &sh, &ch);
    const float d = 6.28318530717958647692f * tl;
    *c = fmaf(-d, sh, ch);
    *s = fmaf(d, ch, sh);
}

__global__ void __launch_bounds__(256)
prep_records_kernel(const double* __restrict__ t, const double* __restrict__ X,
                    const int64_t* __restrict__ off, int64_t n0,
                    const double* __restrict__ f0a, const double* __restrict__ dfa,
                    double f0s, double dfs, const CurveStats* __restrict__ stats,
                    uint4* __restrict__ recA, float4* __restrict__ recB, float2* __restrict__ recN,
                    float* __restrict__ xout, const double* __restrict__ dy, float* __restrict__ qout,
                    int* __restrict__ status) {
    const int c = blockIdx.y;
    const int64_t b = off ? off[c] : 0;
    const int64_t e = off ? off[c + 1] : n0;
    const CurveStats st = stats[c];
    const double f0 = f0a ? f0a[c] : f0s;
    const double df = dfa ? dfa[c] : dfs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // 1/sqrt(sum of weights): the weight sum from the stats, or N without errors
    const float isw = qout ? (float)rsqrt(dy ? st.pad : (double)(e - b)) : 0.f;
    for (int64_t j = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < e; j += stride) {
        const double tt = t[j] - st.t_ref;
        const uint64_t u = frac_turns64(tt, df);
        const uint64_t v = frac_turns64(tt, f0) + kPhaseOffset;
        // rotation of one grid step, cos/sin(2 pi u), from the exact fixed-point turn
        float sn, cs;
        rotation_of(u, &cs, &sn);
        float xh;
        if (qout) {
            // floating-mean form: q = sqrt(w_j) with w_j = v_j / sum v (sum w = 1;
            // equal weights without dy), x = q (X - mean_w) / sd_w, so sum x^2 = 1
            const float q = dy ? isw / (float)dy[j] : isw;
            qout[j] = q;
            // without X (noise realizations, normalized later per realization) x_hat = 0
            xh = X ? (float)((X[j] - st.mean) * st.inv_sd) * q : 0.f;
        } else {
            xh = X ? (float)((X[j] - st.mean) * st.inv_sd) : 0.f;
        }
        // frac_turns64's range: beyond 2^52 turns the phase is not exact
        if (!(fabs(tt * df) < 0x1p52) || !(fabs(tt * f0) < 0x1p52)) {
            xh = __int_as_float(0x7fc00000);
            if (status) atomicOr(status, kStatusPhaseRange);
        }
        recA[j] = make_uint4((uint32_t)u, (uint32_t)(u >> 32), (uint32_t)v, (uint32_t)(v >> 32));
        recB[j] = make_float4(xh, cs, sn, 2.f * cs);
        if (recN) recN[j] = make_float2(xh, __double2float_rn(tt));
        if (xout) xout[j] = xh;
    }
}

}  // namespace

int prep_stats_slices(int n_curves, int64_t n0) {
    if (n_curves > 1) return 1;
    int64_t g = n0 / 2048;
    return (int)(g < 1 ? 1 : (g > kMaxStatSlices ? kMaxStatSlices : g));
}

cudaError_t launch_prep_stats(const double* t, const double* X, const int64_t* off, int64_t n0,
                              int n_curves, CurveStats* stats, int* status, StatPart* parts,
                              unsigned* counters, cudaStream_t st, const double* dy) {
    // without slice scratch every curve gets one CTA
    const int G = (parts && counters) ? prep_stats_slices(n_curves, n0) : 1;
    dim3 grid((unsigned)G, (unsigned)n_curves);
    prep_stats_kernel<<<grid, kStatsThreads, 0, st>>>(t, X, off, n0, stats, status, parts, counters, dy);
    return cudaGetLastError();
}

cudaError_t launch_prep_records(const double* t, const double* X, const int64_t* off, int64_t n0,
                                int n_curves, int64_t max_n, const double* f0, const double* df,
                                double f0_single, double df_single, const CurveStats* stats,
                                uint4* recA, float4* recB, float2* recN, float* xout, cudaStream_t st,
                                const double* dy, float* qout, int* status) {
    int64_t bx = (max_n + 255) / 256;
    if (bx > 4096) bx = 4096;
    if (bx < 1) bx = 1;
    dim3 grid((unsigned)bx, (unsigned)n_curves);
    prep_records_kernel<<<grid, 256, 0, st>>>(t, X, off, n0, f0, df, f0_single, df_single, stats,
                                              recA, recB, recN, xout, dy, qout, status);
    return cudaGetLastError();
}

}  // namespace lsp
