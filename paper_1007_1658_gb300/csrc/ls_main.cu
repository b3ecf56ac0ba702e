// ls_main.cu -- the O(N_t N_f) evaluation of the sums of Eq. 8 and the
// periodogram of Eq. 5-6 for one curve.
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
// A thread forms the top 32 bits once per sample for its first k, so the
// phase never loses accuracy however large f t grows.
//
// sin/cos modes (ls_device.cuh, Strip::add and Strip<F, kRecur3x2>):
//   MUFU   -- every (j, k) takes the hardware sin/cos of the phase (the
//             paper's __sincosf, Sec. 4.3), stepping the 32-bit phase by
//             round(u / 2^32): 2 SFU ops per term.
//   RECUR  -- the hardware sin/cos seeds the first k of the strip; the next
//             F-1 follow from the angle-addition formulas with the per-sample
//             rotation (cos, sin)(2 pi u_j): 4 FMA-pipe ops per term.  The
//             recurrence (the trig recursion of Sec. 3, there rejected for
//             drifting at large N_f) is re-seeded from the exact phase every F
//             steps, which bounds the drift by ~F ulp.
//   RECUR3 -- one angle-addition step, then the three-term form of the same
//             identity, z_{k+1} = 2 cos(2 pi u_j) z_k - z_{k-1}: 2 FMA-pipe ops
//             per term.  Its rounding error grows like F^2 ulp, and like
//             F ulp / sin(2 pi u_j) for samples whose step angle is near 0 or pi.
//   RECUR3 x2 -- the same arithmetic in packed FP32x2 FMA (FFMA2), the
//             (cos, sin) pair of a frequency in the two lanes: (XC, XS),
//             (CC, CS) and the step one FFMA2 each per term, half the issue
//             slots; sums bit-identical to RECUR3 at the same F.  The default.
// NAIVE_FP32 -- the paper's own single-precision phase f*t - rintf(f*t)
//             (Sec. 4.3), kept as a comparator.
#include "ls_device.cuh"

namespace lsp {
namespace {

using namespace dev;

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
    __shared__ __align__(16) TileSmem<false> sm;
    const uint32_t k0 = (uint32_t)blockIdx.x * (kMainThreads * F) + (uint32_t)threadIdx.x * F;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(N, j0 + chunk);
    Strip<F, MODE> st;
    st.zero();
    const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
    for_each_tile<false>(sm, recA, recB, nullptr, j0, j1,
                         [&](const uint4* a, const float4* b, const float*, int n) {
                             if (live) strip_tile<kTile>(st, a, b, n, k0);
                         });
    float xc[F], xs[F], cc[F], cs[F];
#pragma unroll
    for (int i = 0; i < F; ++i) st.get(i, xc[i], xs[i], cc[i], cs[i]);
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
    float s[4], c[4];
    merge_chunks<4>(part, split, nf_pad, k, s, c);
    P_out[k] = periodogram_value(s[0] + c[0], s[1] + c[1], s[2] + c[2], s[3] + c[3], n);
}

using MainFn = void (*)(const uint4*, const float4*, int64_t, int64_t, int, int64_t, float*, float*);
using NaiveFn = void (*)(const float2*, int64_t, int64_t, int, int64_t, double, double, float*, float*);

template <int MODE>
MainFn main_fn_f(int F) {
    switch (F) {
        case 4: return ls_main_kernel<4, MODE>;
        case 8: return ls_main_kernel<8, MODE>;
        case 12: return ls_main_kernel<12, MODE>;
        case 16: return ls_main_kernel<16, MODE>;
        case 20: return MODE == kMufu ? nullptr : ls_main_kernel<20, MODE>;
        case 24: return ls_main_kernel<24, MODE>;
        case 28: return MODE == kMufu ? nullptr : ls_main_kernel<28, MODE>;
        default: return nullptr;
    }
}

MainFn main_fn(int mode, int F) {
    switch (mode) {
        case kMufu: return main_fn_f<kMufu>(F);
        case kRecur: return main_fn_f<kRecur>(F);
        case kRecur3: return main_fn_f<kRecur3>(F);
        case kRecur3x2: return main_fn_f<kRecur3x2>(F);
        default: return nullptr;
    }
}

NaiveFn naive_fn(int F) {
    switch (F) {
        case 4: return ls_naive_kernel<4>;
        case 8: return ls_naive_kernel<8>;
        case 12: return ls_naive_kernel<12>;
        case 16: return ls_naive_kernel<16>;
        case 24: return ls_naive_kernel<24>;
        default: return nullptr;
    }
}

}  // namespace

int main_occupancy(int mode, int F) {
    int nb = 0;
    const void* fn = mode == dev::kNaive ? (const void*)naive_fn(F) : (const void*)main_fn(mode, F);
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
    if (s.mode == dev::kNaive) {
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
