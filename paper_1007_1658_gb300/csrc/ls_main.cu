// ls_main.cu -- the O(N_t N_f) evaluation of the sums of Eq. 8 and the
// periodogram of Eq. 5-6.
//
// Layout of the work: a CTA of kMainThreads threads owns kMainThreads*F
// adjacent grid frequencies (each thread a strip of F adjacent k) and one
// chunk of the samples (blockIdx.y).  Sample records (32 B each: fixed-point
// phases, normalized x, rotation cos/sin) are staged in shared memory in
// tiles of kTile samples with cp.async, double-buffered; every thread of the
// CTA then reads the same record (a shared-memory broadcast) and updates the
// four running sums XC, XS, CC, CS (Eq. 8; SS = N_t - CC as in the paper's
// kernel) of each of its F frequencies in registers.  Per-thread FP32 sums
// run over at most one chunk (the paper's chunked summation, Sec. 4.2, at a
// coarser grain); chunks are combined by the finalize kernel in a fixed
// order with compensated FP32 sums, so results are bit-reproducible.
//
// Phase (exact): the records hold u = frac(t' df) and v = frac(t' f0) as
// 64-bit fixed-point turns; for frequency k the phase is v + k u mod 2^64.
// A thread forms the top 32 bits once per sample for its first k and then
// steps by round(u / 2^32) (error <= F/2 units of 2^-32 turn), so the
// phase never loses accuracy however large f t grows.
//
// sin/cos, two modes:
//   MUFU  -- every (j, k) takes the hardware sin/cos of the phase (the
//            paper's __sincosf, Sec. 4.3): 2 SFU ops per term.
//   RECUR -- the hardware sin/cos seeds the first k of the strip; the next
//            F-1 follow from the angle-addition formulas with the per-sample
//            rotation (cos, sin)(2 pi u_j): 4 FMA-pipe ops per term.  The
//            recurrence (the trig recursion of Sec. 3, there rejected for
//            drifting at large N_f) is re-seeded from the exact phase every F
//            steps, which bounds the drift by ~F ulp.
// NAIVE_FP32 -- the paper's own single-precision phase f*t - rintf(f*t)
//            (Sec. 4.3), kept as a comparator.
#include <cstdio>

#include "lsp_kernels.cuh"

namespace lsp {
namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kThreePi = 9.42477796076937971538f;

// Top 23 bits of a 32-bit turn fraction, offset by half a turn at prep time,
// become a float in [1, 2) by pasting them under the exponent of 1.0; one FMA
// maps that to an angle in [-pi, pi).  No int->float conversion unit is used.
__device__ __forceinline__ float phase_to_angle(uint32_t p) {
    return fmaf(__uint_as_float(0x3F800000u | (p >> 9)), kTwoPi, -kThreePi);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Eq. 5 with tau from Eq. 6, in closed form.  With A = CC - SS = 2CC - N,
// B = 2CS and R = |A + iB| = |sum exp(2 i w t_j)|, tan 2wtau = B/A gives
// cos 2wtau = A/R, sin 2wtau = B/R, and the two denominators of Eq. 5 are
// (N + R)/2 and (N - R)/2; the two numerators are (|Z|^2 +- Re(e^{-2iwtau} Z^2))/2
// with Z = XC + i XS.  No trig, and R = 0 (tau undefined) takes wtau = 0.
// A term whose denominator is below N 2^-16 is taken as zero.
__device__ __forceinline__ float periodogram_value(float XC, float XS, float CC, float CS, float n) {
    const float A = 2.f * CC - n;
    const float B = 2.f * CS;
    const float R = sqrtf(A * A + B * B);
    float c2 = 1.f, s2 = 0.f;
    if (R > 0.f) {
        c2 = A / R;
        s2 = B / R;
    }
    const float z2 = XC * XC + XS * XS;
    const float cross = c2 * (XC * XC - XS * XS) + s2 * (2.f * XC * XS);
    const float num1 = fmaxf(0.5f * (z2 + cross), 0.f);
    const float num2 = fmaxf(0.5f * (z2 - cross), 0.f);
    const float den1 = 0.5f * (n + R);
    const float den2 = 0.5f * (n - R);
    const float thr = n * (1.f / 65536.f);
    float P = 0.f;
    if (den1 > thr) P += num1 / den1;
    if (den2 > thr) P += num2 / den2;
    return 0.5f * P;
}

template <int F>
__device__ __forceinline__ void write_out(const float (&xc)[F], const float (&xs)[F], const float (&cc)[F],
                                          const float (&cs)[F], uint32_t k0, int N_f, int64_t nf_pad,
                                          int64_t N, float* __restrict__ part, float* __restrict__ P_out) {
    if (P_out) {
        const float n = (float)N;
#pragma unroll
        for (int i = 0; i < F; ++i)
            if (k0 + i < (uint32_t)N_f) P_out[k0 + i] = periodogram_value(xc[i], xs[i], cc[i], cs[i], n);
        return;
    }
    float* base = part + (size_t)blockIdx.y * 4 * (size_t)nf_pad + k0;
#pragma unroll
    for (int i = 0; i < F; i += 4) {
        *reinterpret_cast<float4*>(base + i) = make_float4(xc[i], xc[i + 1], xc[i + 2], xc[i + 3]);
        *reinterpret_cast<float4*>(base + nf_pad + i) = make_float4(xs[i], xs[i + 1], xs[i + 2], xs[i + 3]);
        *reinterpret_cast<float4*>(base + 2 * nf_pad + i) = make_float4(cc[i], cc[i + 1], cc[i + 2], cc[i + 3]);
        *reinterpret_cast<float4*>(base + 3 * nf_pad + i) = make_float4(cs[i], cs[i + 1], cs[i + 2], cs[i + 3]);
    }
}

template <int F, int MODE>
__global__ void __launch_bounds__(kMainThreads)
ls_main_kernel(const uint4* __restrict__ recA, const float4* __restrict__ recB, int64_t N, int64_t chunk,
               int N_f, int64_t nf_pad, float* __restrict__ part, float* __restrict__ P_out) {
    __shared__ __align__(16) uint4 sA[2][kTile];
    __shared__ __align__(16) float4 sB[2][kTile];
    const int tid = threadIdx.x;
    const uint32_t k0 = (uint32_t)blockIdx.x * (kMainThreads * F) + (uint32_t)tid * F;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(N, j0 + chunk);
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + kTile - 1) / kTile) : 0;

    float xc[F], xs[F], cc[F], cs[F];
#pragma unroll
    for (int i = 0; i < F; ++i) xc[i] = xs[i] = cc[i] = cs[i] = 0.f;

    if (ntiles > 0) {
        const int n = (int)min((int64_t)kTile, j1 - j0);
        for (int q = tid; q < n; q += kMainThreads) {
            cp_async16(&sA[0][q], recA + j0 + q);
            cp_async16(&sB[0][q], recB + j0 + q);
        }
    }
    cp_async_commit();

    for (int it = 0; it < ntiles; ++it) {
        const int64_t jt = j0 + (int64_t)it * kTile;
        if (it + 1 < ntiles) {
            const int64_t jn = jt + kTile;
            const int n = (int)min((int64_t)kTile, j1 - jn);
            const int buf = (it + 1) & 1;
            for (int q = tid; q < n; q += kMainThreads) {
                cp_async16(&sA[buf][q], recA + jn + q);
                cp_async16(&sB[buf][q], recB + jn + q);
            }
        }
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int n = (int)min((int64_t)kTile, j1 - jt);
        const uint4* a = sA[it & 1];
        const float4* bb = sB[it & 1];
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
            const uint4 A = a[j];
            const float4 B = bb[j];
            const uint64_t u = ((uint64_t)A.y << 32) | A.x;
            const uint64_t v = ((uint64_t)A.w << 32) | A.z;
            uint32_t p = (uint32_t)((v + (uint64_t)k0 * u) >> 32);
            const float x = B.x;
            if (MODE == 1) {
                const uint32_t du = __float_as_uint(B.w);
#pragma unroll
                for (int i = 0; i < F; ++i) {
                    float s, c;
                    __sincosf(phase_to_angle(p), &s, &c);
                    xc[i] = fmaf(x, c, xc[i]);
                    xs[i] = fmaf(x, s, xs[i]);
                    cc[i] = fmaf(c, c, cc[i]);
                    cs[i] = fmaf(c, s, cs[i]);
                    p += du;
                }
            } else {
                const float C = B.y, S = B.z;
                float s, c;
                __sincosf(phase_to_angle(p), &s, &c);
#pragma unroll
                for (int i = 0; i < F; ++i) {
                    xc[i] = fmaf(x, c, xc[i]);
                    xs[i] = fmaf(x, s, xs[i]);
                    cc[i] = fmaf(c, c, cc[i]);
                    cs[i] = fmaf(c, s, cs[i]);
                    if (i + 1 < F) {
                        const float cn = fmaf(c, C, -s * S);
                        s = fmaf(s, C, c * S);
                        c = cn;
                    }
                }
            }
        }
        __syncthreads();
    }
    write_out<F>(xc, xs, cc, cs, k0, N_f, nf_pad, N, part, P_out);
}

// The paper's single-precision phase (Sec. 4.3): f_k = (float)(f0 + k df),
// t = (float)(t_j - t_ref), ft = f*t rounded to float, ft - rintf(ft), then
// __sincosf(2 pi ft).  Records are {x_hat, (float) t'}.
template <int F>
__global__ void __launch_bounds__(kMainThreads)
ls_naive_kernel(const float2* __restrict__ recN, int64_t N, int64_t chunk, int N_f, int64_t nf_pad,
                double f0, double df, float* __restrict__ part, float* __restrict__ P_out) {
    __shared__ __align__(16) float2 sN[2][kTile];
    const int tid = threadIdx.x;
    const uint32_t k0 = (uint32_t)blockIdx.x * (kMainThreads * F) + (uint32_t)tid * F;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(N, j0 + chunk);
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + kTile - 1) / kTile) : 0;
    float f[F];
#pragma unroll
    for (int i = 0; i < F; ++i) f[i] = __double2float_rn(__dadd_rn(f0, __dmul_rn((double)(k0 + i), df)));
    float xc[F], xs[F], cc[F], cs[F];
#pragma unroll
    for (int i = 0; i < F; ++i) xc[i] = xs[i] = cc[i] = cs[i] = 0.f;
    if (ntiles > 0) {
        const int n = (int)min((int64_t)kTile, j1 - j0);
        for (int q = tid; q < n; q += kMainThreads) cp_async8(&sN[0][q], recN + j0 + q);
    }
    cp_async_commit();
    for (int it = 0; it < ntiles; ++it) {
        const int64_t jt = j0 + (int64_t)it * kTile;
        if (it + 1 < ntiles) {
            const int64_t jn = jt + kTile;
            const int n = (int)min((int64_t)kTile, j1 - jn);
            for (int q = tid; q < n; q += kMainThreads) cp_async8(&sN[(it + 1) & 1][q], recN + jn + q);
        }
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int n = (int)min((int64_t)kTile, j1 - jt);
        const float2* r = sN[it & 1];
        for (int j = 0; j < n; ++j) {
            const float2 R = r[j];
#pragma unroll
            for (int i = 0; i < F; ++i) {
                const float ft = __fmul_rn(f[i], R.y);
                const float red = __fsub_rn(ft, rintf(ft));
                float s, c;
                __sincosf(__fmul_rn(kTwoPi, red), &s, &c);
                xc[i] = fmaf(R.x, c, xc[i]);
                xs[i] = fmaf(R.x, s, xs[i]);
                cc[i] = fmaf(c, c, cc[i]);
                cs[i] = fmaf(c, s, cs[i]);
            }
        }
        __syncthreads();
    }
    write_out<F>(xc, xs, cc, cs, k0, N_f, nf_pad, N, part, P_out);
}

// Fixed-order compensated (Neumaier) FP32 sum of the per-chunk partial sums,
// then Eq. 5-6.
__global__ void __launch_bounds__(256)
finalize_kernel(const float* __restrict__ part, int split, int64_t nf_pad, int N_f, float n,
                float* __restrict__ P_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N_f) return;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int sp = 0; sp < split; ++sp) {
        const float* p = part + (size_t)sp * 4 * (size_t)nf_pad + k;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float v = p[(size_t)q * nf_pad];
            const float tsum = s[q] + v;
            if (fabsf(s[q]) >= fabsf(v))
                c[q] += (s[q] - tsum) + v;
            else
                c[q] += (v - tsum) + s[q];
            s[q] = tsum;
        }
    }
    P_out[k] = periodogram_value(s[0] + c[0], s[1] + c[1], s[2] + c[2], s[3] + c[3], n);
}

using MainFn = void (*)(const uint4*, const float4*, int64_t, int64_t, int, int64_t, float*, float*);
using NaiveFn = void (*)(const float2*, int64_t, int64_t, int, int64_t, double, double, float*, float*);

MainFn main_fn(int mode, int F) {
    if (mode == 1) {
        if (F == 4) return ls_main_kernel<4, 1>;
        if (F == 8) return ls_main_kernel<8, 1>;
        if (F == 16) return ls_main_kernel<16, 1>;
    } else if (mode == 2) {
        if (F == 4) return ls_main_kernel<4, 2>;
        if (F == 8) return ls_main_kernel<8, 2>;
        if (F == 16) return ls_main_kernel<16, 2>;
    }
    return nullptr;
}

NaiveFn naive_fn(int F) {
    if (F == 4) return ls_naive_kernel<4>;
    if (F == 8) return ls_naive_kernel<8>;
    if (F == 16) return ls_naive_kernel<16>;
    return nullptr;
}

}  // namespace

int main_occupancy(int mode, int F) {
    int nb = 0;
    const void* fn = mode == 3 ? (const void*)naive_fn(F) : (const void*)main_fn(mode, F);
    if (!fn) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kMainThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_main(const MainShape& s, const uint4* recA, const float4* recB, const float2* recN,
                        int64_t N, int64_t N_f, double f0, double df, float* part, float* P_out,
                        cudaStream_t st) {
    dim3 grid((unsigned)s.nfb, (unsigned)s.split);
    float* direct = s.split == 1 ? P_out : nullptr;
    if (s.mode == 3) {
        NaiveFn fn = naive_fn(s.F);
        if (!fn) return cudaErrorInvalidValue;
        fn<<<grid, kMainThreads, 0, st>>>(recN, N, s.chunk, (int)N_f, s.nf_pad, f0, df, part, direct);
    } else {
        MainFn fn = main_fn(s.mode, s.F);
        if (!fn) return cudaErrorInvalidValue;
        fn<<<grid, kMainThreads, 0, st>>>(recA, recB, N, s.chunk, (int)N_f, s.nf_pad, part, direct);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const MainShape& s, const float* part, int64_t N, int64_t N_f, float* P_out,
                            cudaStream_t st) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((N_f + threads - 1) / threads);
    finalize_kernel<<<blocks, threads, 0, st>>>(part, s.split, s.nf_pad, (int)N_f, (float)N, P_out);
    return cudaGetLastError();
}

}  // namespace lsp
