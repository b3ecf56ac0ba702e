// gls.cu -- the floating-mean (generalized, weighted) periodogram: the
// extension of the sums of Eq. 8 that Sec. 6.3 points to (Shrager 2001;
// Zechmeister & Kuerster 2009), where a constant offset is fitted together
// with the sinusoid and each sample carries the weight w_j = (1/dy_j^2) /
// sum(1/dy^2).
//
// With centred, weighted data the sums needed per frequency are
//   YC = sum w y' cos,  YS = sum w y' sin         (y' = y - sum w y)
//   C  = sum w cos,     S  = sum w sin
//   CC' = sum w cos^2,  CS' = sum w cos sin       (SS' = 1 - CC')
// and the centred second moments CC = CC' - C^2, SS = SS' - S^2,
// CS = CS' - C S.  The power is the fraction p of the weighted variance
// removed by the best fit a cos + b sin + c, reported as P = (N_t / 2) p.
//
// Per-sample records are the classic ones (fixed-point phases, rotation) with
// x = q (y - mean_w) / sd_w and a second stream q_j = sqrt(w_j).  The sin/cos
// seed of each strip is scaled by q once per sample; the recurrences are
// linear, so every later term of the strip carries the factor q too, and
// with c~ = q cos, s~ = q sin the six running sums are
//   XC += x c~, XS += x s~, C += q c~, S += q s~, CC' += c~ c~, CS' += c~ s~
// -- six FMA per term plus the recurrence (2 FMA in the three-term form):
// 8 FMA-pipe ops per term against 6 for the classic periodogram.
//
// Closed form of p (same algebra as Eq. 5-6 with the trace CC + SS in place
// of N_t): the 2x2 matrix [[CC, CS], [CS, SS]] has eigenvalues (T +- R)/2,
// T = CC + SS, R = |CC - SS + 2i CS|; rotating (YC, YS) onto its eigenvectors
// gives p = num1/den1 + num2/den2 (data variance normalized to 1).  A
// direction whose eigenvalue is at the FP32 rounding level (f = 0, the
// Nyquist frequency of an even grid, two-phase sampling) adds nothing: the
// fit is the projection on the remaining direction.
#include "ls_device.cuh"

namespace lsp {
namespace {

using namespace dev;

constexpr int kGlsSums = kGlsRows;

template <int F, int MODE>
struct GStrip {
    float xc[F], xs[F], c1[F], s1[F], cc[F], cs[F];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) xc[i] = xs[i] = c1[i] = s1[i] = cc[i] = cs[i] = 0.f;
    }

    __device__ __forceinline__ void acc(int i, float x, float q, float c, float s) {
        xc[i] = fmaf(x, c, xc[i]);
        xs[i] = fmaf(x, s, xs[i]);
        c1[i] = fmaf(q, c, c1[i]);
        s1[i] = fmaf(q, s, s1[i]);
        cc[i] = fmaf(c, c, cc[i]);
        cs[i] = fmaf(c, s, cs[i]);
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, float x, float q, uint32_t k0) {
        uint32_t p = top_phase_hi(A, k0);
        if (MODE == kMufu) {
            const uint32_t du = round_top_word(A);
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float s, c;
                __sincosf(phase_to_angle(p), &s, &c);
                acc(i, x, q, q * c, q * s);
                p += du;
            }
        } else {
            const float C = B.y, S = B.z, C2 = B.w;
            float s, c;
            __sincosf(phase_to_angle(p), &s, &c);
            c *= q;
            s *= q;
            float cp = c, sp = s;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                acc(i, x, q, c, s);
                if (i + 1 < F) {
                    float cn, sn;
                    if (MODE == kRecur || i == 0) {
                        cn = fmaf(c, C, -s * S);
                        sn = fmaf(s, C, c * S);
                    } else {
                        cn = fmaf(C2, c, -cp);
                        sn = fmaf(C2, s, -sp);
                    }
                    cp = c;
                    sp = s;
                    c = cn;
                    s = sn;
                }
            }
        }
    }
};

// Packed form of the three-term strip with the sign-folded y_i of
// Strip<F, kRecur3x2>, here with the (cos, sin) pair in the two lanes: the
// pairs (XC, XS), (C, S) and (CC', CS') take one FFMA2 each per term, with the
// data factors +-x, +-q and the pair (c, c), the recurrence one FFMA2: no
// scalar FFMA between the packed ones.  With CC' and CS' as two scalar FFMA
// instead, the mix measured 5.40 against 4.85 ms on 100,000 x 200,000 (FMA
// pipe busy 75 % of cycles, math-pipe throttle the top stall).  Bit-identical
// to GStrip<F, kRecur3>.
template <int F>
struct GStrip<F, kRecur3x2> {
    float xc[F], xs[F], c1[F], s1[F], cc[F], cs[F];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) xc[i] = xs[i] = c1[i] = s1[i] = cc[i] = cs[i] = 0.f;
    }

    __device__ __forceinline__ void acc(int i, float2 xf, float2 qf, float2 y) {
        const float2 a = __ffma2_rn(xf, y, make_float2(xc[i], xs[i]));
        xc[i] = a.x;
        xs[i] = a.y;
        const float2 b = __ffma2_rn(qf, y, make_float2(c1[i], s1[i]));
        c1[i] = b.x;
        s1[i] = b.y;
        const float2 d = __ffma2_rn(make_float2(y.x, y.x), y, make_float2(cc[i], cs[i]));
        cc[i] = d.x;
        cs[i] = d.y;
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, float x, float q, uint32_t k0) {
        const uint32_t p = top_phase_hi(A, k0);
        const float C = B.y, S = B.z, C2 = B.w;
        float s, c;
        __sincosf(phase_to_angle(p), &s, &c);
        c *= q;
        s *= q;
        const float2 xp = make_float2(x, x), xn = make_float2(-x, -x);
        const float2 qp = make_float2(q, q), qn = make_float2(-q, -q);
        const float2 cp2 = make_float2(C2, C2), cn2 = make_float2(-C2, -C2);
        float2 y0 = make_float2(c, s);
        acc(0, xp, qp, y0);
        if (F == 1) return;
        float2 y1 = make_float2(fmaf(c, C, -s * S), fmaf(s, C, c * S));
        acc(1, xp, qp, y1);
#pragma unroll
        for (int i = 2; i < F; ++i) {
            const float2 y2 = __ffma2_rn(((i - 1) & 1) ? cn2 : cp2, y1, y0);
            const bool neg = (i >> 1) & 1;
            acc(i, neg ? xn : xp, neg ? qn : qp, y2);
            y0 = y1;
            y1 = y2;
        }
    }
};

// p from the six sums (weights summing to 1, data variance 1), in FP64.
// Data the prep kernels refuse are reported through the status word (this
// path has no allocation-free form that would need NaN outputs instead).
__device__ __forceinline__ float gls_value(double XC, double XS, double C, double S, double CCp, double CSp,
                                           double n) {
    const double CC = CCp - C * C;
    const double SS = (1.0 - CCp) - S * S;
    const double CS = CSp - C * S;
    const double A = CC - SS, B = 2.0 * CS;
    const double T = CC + SS;
    const double R = sqrt(A * A + B * B);
    double c2 = 1.0, s2 = 0.0;
    if (R > 0.0) {
        const double iR = 1.0 / R;
        c2 = A * iR;
        s2 = B * iR;
    }
    const double z2 = XC * XC + XS * XS;
    const double cross = c2 * (XC * XC - XS * XS) + s2 * (2.0 * XC * XS);
    const double num1 = fmax(0.5 * (z2 + cross), 0.0);
    const double num2 = fmax(0.5 * (z2 - cross), 0.0);
    const double den1 = 0.5 * (T + R);
    const double den2 = 0.5 * (T - R);
    const double thr = 0x1p-24;
    double p = 0.0;
    if (den1 > thr) p += num1 / den1;
    if (den2 > thr) p += num2 / den2;
    return (float)(0.5 * n * p);
}

template <int F, int MODE>
__global__ void __launch_bounds__(kGlsThreads)
gls_main_kernel(const uint4* __restrict__ recA, const float4* __restrict__ recB, const float* __restrict__ q,
                int64_t N, int64_t chunk, int N_f, int64_t nf_pad, float* __restrict__ part,
                float* __restrict__ P_out) {
    __shared__ __align__(16) TileSmemN<1, kGlsTile> sm;
    const uint32_t k0 = (uint32_t)blockIdx.x * (kGlsThreads * F) + (uint32_t)threadIdx.x * F;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(N, j0 + chunk);
    GStrip<F, MODE> st;
    st.zero();
    const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
    for_each_tile_n<1>(sm, recA, recB, q, 0, 1, j0, j1,
                       [&](const uint4* a, const float4* b, const float (*qs)[kGlsTile], int n) {
                           if (!live) return;
#pragma unroll 2
                           for (int j = 0; j < n; ++j) {
                               const float4 B = b[j];
                               st.add(a[j], B, B.x, qs[0][j], k0);
                           }
                       });
    if (P_out) {
#pragma unroll
        for (int i = 0; i < F; ++i)
            if (k0 + i < (uint32_t)N_f)
                P_out[k0 + i] = gls_value(st.xc[i], st.xs[i], st.c1[i], st.s1[i], st.cc[i], st.cs[i], (double)N);
        return;
    }
    float* base = part + (size_t)blockIdx.y * kGlsSums * (size_t)nf_pad + k0;
    auto row = [&](int r, const float (&v)[F]) {
#pragma unroll
        for (int i = 0; i < F; i += 4)
            *reinterpret_cast<float4*>(base + (size_t)r * nf_pad + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    };
    row(0, st.xc);
    row(1, st.xs);
    row(2, st.c1);
    row(3, st.s1);
    row(4, st.cc);
    row(5, st.cs);
}

// Per-chunk partial sums added in chunk order with compensated (Neumaier)
// FP32 sums (deterministic; FP64 adds are slow on this part), then p in FP64.
__global__ void __launch_bounds__(256)
gls_finalize_kernel(const float* __restrict__ part, int split, int64_t nf_pad, int N_f, double n,
                    float* __restrict__ P_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N_f) return;
    float s[kGlsSums], c[kGlsSums];
    merge_chunks<kGlsSums>(part, split, nf_pad, k, s, c);
    P_out[k] = gls_value((double)s[0] + c[0], (double)s[1] + c[1], (double)s[2] + c[2], (double)s[3] + c[3],
                         (double)s[4] + c[4], (double)s[5] + c[5], n);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Many curves in one persistent launch: CTAs take (curve, block of
// kGlsBatchThreads*F frequencies) items from an atomic ticket, run the strip over
// all samples of the curve, finish p in FP64, write P if asked and fold the
// block's largest P into the curve's (P bits << 32 | ~k) maximum.  MINB = 16
// holds the packed strip to 128 registers: four warps per sub-partition
// instead of the two that the compiler's free choice (221 registers) leaves,
// for a few spilled values.  That raises throughput (4096-curve batch 100.9 ->
// 99.0 ms) but halves each warp's own speed, so a batch whose longest curve
// is a large share of the work (256 curves: 7.2 -> 8.2 ms) runs the unbounded
// form; results are the same either way.
// With XROW the items are noise realizations (lsp_batch_gls_noise): item
// (curve, realization r) takes its x from row r of xr (stride `total`) instead
// of from the records, staged into the records' x slot as the tile arrives,
// and writes P and the maximum of realization r (P at r P_total + P_off[c],
// the key at r n_curves + c).  Measured curves are realization 0.
template <int TILE, class Body>
__device__ __forceinline__ void for_each_tile_gx(TileSmemN<1, TILE>& sm, const uint4* __restrict__ recA,
                                                 const float4* __restrict__ recB, const float* __restrict__ q,
                                                 const float* __restrict__ x, int64_t j0, int64_t j1,
                                                 Body&& body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + TILE - 1) / TILE) : 0;
    auto stage = [&](int buf, int64_t jt) {
        const int n = (int)min((int64_t)TILE, j1 - jt);
        for (int i = tid; i < n; i += nt) {
            cp_async16(&sm.A[buf][i], recA + jt + i);
            float* dst = reinterpret_cast<float*>(&sm.B[buf][i]);
            const float* src = reinterpret_cast<const float*>(recB + jt + i);
            cp_async4(dst, x + jt + i);
            cp_async4(dst + 1, src + 1);
            cp_async8(dst + 2, src + 2);
            cp_async4(&sm.X[buf][0][i], q + jt + i);
        }
    };
    if (ntiles > 0) stage(0, j0);
    cp_async_commit();
    for (int it = 0; it < ntiles; ++it) {
        const int64_t jt = j0 + (int64_t)it * TILE;
        if (it + 1 < ntiles) stage((it + 1) & 1, jt + TILE);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        body(sm.A[it & 1], sm.B[it & 1], sm.X[it & 1], (int)min((int64_t)TILE, j1 - jt));
        __syncthreads();
    }
}

template <int F, int MODE, int MINB, bool XROW>
__global__ void __launch_bounds__(kGlsBatchThreads, MINB)
gls_batch_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                 const int64_t* __restrict__ off, const int64_t* __restrict__ nf, const uint4* __restrict__ recA,
                 const float4* __restrict__ recB, const float* __restrict__ q, float* __restrict__ P_out,
                 const int64_t* __restrict__ P_off, unsigned long long* __restrict__ maxkey,
                 const float* __restrict__ xr, int64_t total, int64_t P_total, int n_curves) {
    __shared__ __align__(16) TileSmemN<1, kGlsBatchTile> sm;
    __shared__ int s_item;
    __shared__ unsigned long long s_red[kGlsBatchThreads / 32];
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const int64_t b = off[w.curve], e = off[w.curve + 1];
        const int64_t N_f = nf[w.curve];
        const uint32_t k0 = (uint32_t)w.fblock * (kGlsBatchThreads * F) + (uint32_t)threadIdx.x * F;
        GStrip<F, MODE> st;
        st.zero();
        const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
        auto body = [&](const uint4* a, const float4* bb, const float (*qs)[kGlsBatchTile], int n) {
            if (!live) return;
#pragma unroll 2
            for (int j = 0; j < n; ++j) {
                const float4 B = bb[j];
                st.add(a[j], B, B.x, qs[0][j], k0);
            }
        };
        if constexpr (XROW)
            for_each_tile_gx(sm, recA, recB, q, xr + (size_t)w.real * (size_t)total, b, e, body);
        else
            for_each_tile_n<1>(sm, recA, recB, q, 0, 1, b, e, body);
        float* P = P_out ? P_out + (size_t)w.real * (size_t)P_total + P_off[w.curve] : nullptr;
        unsigned long long best = 0ull;
#pragma unroll
        for (int i = 0; i < F; ++i) {
            const uint32_t k = k0 + i;
            if (k < (uint32_t)N_f) {
                const float p = gls_value(st.xc[i], st.xs[i], st.c1[i], st.s1[i], st.cc[i], st.cs[i], (double)(e - b));
                if (P) P[k] = p;
                best = umax64(best, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(~k));
            }
        }
        for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_down_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = s_red[0];
            for (int x = 1; x < kGlsBatchThreads / 32; ++x) m = umax64(m, s_red[x]);
            if (m) atomicMax(&maxkey[(size_t)w.real * (size_t)n_curves + w.curve], m);
        }
    }
}

// Floating-mean strip for R noise realizations of one curve (packed form):
// the realizations share the phase, the (cos, sin) recurrence and the sums
// of the sampling pattern and weights, (C, S) and (CC', CS'); each keeps its
// own (XC, XS).  Every operation is an FFMA2 with the (cos, sin) pair y in
// the lanes, signs g_i folded into the sums as in the other packed strips:
// per term and realization 2 lane operations plus 6 / R for the shared ones,
// against 8 one at a time.  Each (frequency, realization) comes out bit for
// bit as GStrip<F, kRecur3x2> computes it.
template <int F, int R>
struct GMStrip {
    float2 a[F][R];  // g_i (XC, XS) of realization r
    float2 w1[F];    // g_i (C, S)
    float2 w2[F];    // (CC', CS')

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) {
            w1[i] = w2[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) a[i][r] = make_float2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ float value(int i, int r, double n) const {
        const float g = ((i >> 1) & 1) ? -1.f : 1.f;
        return gls_value(g * a[i][r].x, g * a[i][r].y, g * w1[i].x, g * w1[i].y, w2[i].x, w2[i].y, n);
    }

    __device__ __forceinline__ void acc(int i, const float2 (&xp)[R], float2 qp, float2 y) {
#pragma unroll
        for (int r = 0; r < R; ++r) a[i][r] = __ffma2_rn(xp[r], y, a[i][r]);
        w1[i] = __ffma2_rn(qp, y, w1[i]);
        w2[i] = __ffma2_rn(make_float2(y.x, y.x), y, w2[i]);
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, const float (&x)[R], float q, uint32_t k0) {
        const uint32_t p = top_phase_hi(A, k0);
        const float C = B.y, S = B.z, C2 = B.w;
        float s, c;
        __sincosf(phase_to_angle(p), &s, &c);
        c *= q;
        s *= q;
        float2 xp[R];
#pragma unroll
        for (int r = 0; r < R; ++r) xp[r] = make_float2(x[r], x[r]);
        const float2 qp = make_float2(q, q);
        const float2 cp2 = make_float2(C2, C2), cn2 = make_float2(-C2, -C2);
        float2 y0 = make_float2(c, s);
        acc(0, xp, qp, y0);
        if (F == 1) return;
        float2 y1 = make_float2(fmaf(c, C, -s * S), fmaf(s, C, c * S));
        acc(1, xp, qp, y1);
#pragma unroll
        for (int i = 2; i < F; ++i) {
            const float2 y2 = __ffma2_rn(((i - 1) & 1) ? cn2 : cp2, y1, y0);
            acc(i, xp, qp, y2);
            y0 = y1;
            y1 = y2;
        }
    }
};

// Tile of the floating-mean realization groups: the two records, the R
// realizations' x of a sample side by side (one 128-bit load for R = 4) and
// the sqrt-weight q.
template <int R, int TILE>
struct GTileX {
    uint4 A[2][TILE];
    float4 B[2][TILE];
    float X[2][TILE][R];
    float Q[2][TILE];
};

// Persistent kernel over (curve, group of up to R realizations starting at
// w.real, frequency block) items (w.pad = the group's size) of a floating-mean
// Monte Carlo: x of realization r from row r of xr (stride `total`), P of
// realization r at P_out[r P_total + P_off[c] + k], its maximum at
// maxkey[r n_curves + c].
template <int F, int R, int TILE>
__global__ void __launch_bounds__(kGlsBatchThreads)
gls_mrhs_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                const int64_t* __restrict__ off, const int64_t* __restrict__ nf, const uint4* __restrict__ recA,
                const float4* __restrict__ recB, const float* __restrict__ q, float* __restrict__ P_out,
                const int64_t* __restrict__ P_off, unsigned long long* __restrict__ maxkey,
                const float* __restrict__ xr, int64_t total, int64_t P_total, int n_curves) {
    __shared__ __align__(16) GTileX<R, TILE> sm;
    __shared__ int s_item;
    static_assert(kGlsBatchThreads == 32, "the maxima are reduced within one warp");
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const int64_t b = off[w.curve], e = off[w.curve + 1];
        const int64_t N_f = nf[w.curve];
        const int nr = w.pad;
        const uint32_t k0 = (uint32_t)w.fblock * (kGlsBatchThreads * F) + (uint32_t)threadIdx.x * F;
        GMStrip<F, R> st;
        st.zero();
        const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
        const float* x0 = xr + (size_t)w.real * (size_t)total;
        const int ntiles = e > b ? (int)((e - b + TILE - 1) / TILE) : 0;
        auto stage = [&](int buf, int64_t jt) {
            const int n = (int)min((int64_t)TILE, e - jt);
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                cp_async16(&sm.A[buf][i], recA + jt + i);
                cp_async16(&sm.B[buf][i], recB + jt + i);
                cp_async4(&sm.Q[buf][i], q + jt + i);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < nr)
                        cp_async4(&sm.X[buf][i][r], x0 + (size_t)r * (size_t)total + jt + i);
                    else
                        sm.X[buf][i][r] = 0.f;  // missing realizations of the last group add nothing
                }
            }
        };
        if (ntiles > 0) stage(0, b);
        cp_async_commit();
        for (int t = 0; t < ntiles; ++t) {
            const int64_t jt = b + (int64_t)t * TILE;
            if (t + 1 < ntiles) stage((t + 1) & 1, jt + TILE);
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            const int n = (int)min((int64_t)TILE, e - jt);
            if (live) {
                const int bf = t & 1;
#pragma unroll 2
                for (int j = 0; j < n; ++j) {
                    float x[R];
                    if constexpr (R % 4 == 0) {
#pragma unroll
                        for (int u = 0; u < R / 4; ++u) {
                            const float4 v = reinterpret_cast<const float4*>(sm.X[bf][j])[u];
                            x[4 * u] = v.x;
                            x[4 * u + 1] = v.y;
                            x[4 * u + 2] = v.z;
                            x[4 * u + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < R; ++r) x[r] = sm.X[bf][j][r];
                    }
                    st.add(sm.A[bf][j], sm.B[bf][j], x, sm.Q[bf][j], k0);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r >= nr) break;
            float* P = P_out ? P_out + (size_t)(w.real + r) * (size_t)P_total + P_off[w.curve] : nullptr;
            unsigned long long best = 0ull;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                const uint32_t k = k0 + i;
                if (k < (uint32_t)N_f) {
                    const float p = st.value(i, r, (double)(e - b));
                    if (P) P[k] = p;
                    best = umax64(best, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(~k));
                }
            }
            for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_down_sync(0xffffffffu, best, o));
            if (threadIdx.x == 0 && best)
                atomicMax(&maxkey[(size_t)(w.real + r) * (size_t)n_curves + w.curve], best);
        }
    }
}

using GlsBatchFn = void (*)(const BatchItem*, int, unsigned*, const int64_t*, const int64_t*, const uint4*,
                            const float4*, const float*, float*, const int64_t*, unsigned long long*, const float*,
                            int64_t, int64_t, int);

// Measured curves: every mode at F = 16 and 8, and the bounded packed form.
// Noise realizations (xrow): the packed mode only, F = 16 (both forms) and 8.
GlsBatchFn gls_batch_fn(int mode, int F, bool packed, bool xrow) {
    if (xrow) {
        if (mode != kRecur3x2) return nullptr;
        if (packed) return F == 16 ? gls_batch_kernel<16, kRecur3x2, 16, true> : nullptr;
        return F == 16 ? gls_batch_kernel<16, kRecur3x2, 1, true> : F == 8 ? gls_batch_kernel<8, kRecur3x2, 1, true>
                                                                           : nullptr;
    }
    if (packed) return F == 16 && mode == kRecur3x2 ? gls_batch_kernel<16, kRecur3x2, 16, false> : nullptr;
    if (F == 16) {
        switch (mode) {
            case kMufu: return gls_batch_kernel<16, kMufu, 1, false>;
            case kRecur: return gls_batch_kernel<16, kRecur, 1, false>;
            case kRecur3: return gls_batch_kernel<16, kRecur3, 1, false>;
            case kRecur3x2: return gls_batch_kernel<16, kRecur3x2, 1, false>;
            default: return nullptr;
        }
    }
    if (F == 8) {
        switch (mode) {
            case kMufu: return gls_batch_kernel<8, kMufu, 1, false>;
            case kRecur: return gls_batch_kernel<8, kRecur, 1, false>;
            case kRecur3: return gls_batch_kernel<8, kRecur3, 1, false>;
            case kRecur3x2: return gls_batch_kernel<8, kRecur3x2, 1, false>;
            default: return nullptr;
        }
    }
    return nullptr;
}

using GlsFn = void (*)(const uint4*, const float4*, const float*, int64_t, int64_t, int, int64_t, float*, float*);

template <int MODE>
GlsFn gls_fn_f(int F) {
    switch (F) {
        case 8: return gls_main_kernel<8, MODE>;
        case 12: return gls_main_kernel<12, MODE>;
        case 16: return gls_main_kernel<16, MODE>;
        default: return nullptr;
    }
}

GlsFn gls_fn(int mode, int F) {
    switch (mode) {
        case kMufu: return gls_fn_f<kMufu>(F);
        case kRecur: return gls_fn_f<kRecur>(F);
        case kRecur3: return gls_fn_f<kRecur3>(F);
        case kRecur3x2: return gls_fn_f<kRecur3x2>(F);
        default: return nullptr;
    }
}

}  // namespace

int gls_occupancy(int mode, int F) {
    const GlsFn fn = gls_fn(mode, F);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kGlsThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_gls(const MainShape& s, const uint4* recA, const float4* recB, const float* q, int64_t N,
                       int64_t N_f, float* part, float* P_out, cudaStream_t st) {
    const GlsFn fn = gls_fn(s.mode, s.F);
    if (!fn) return cudaErrorInvalidValue;
    dim3 grid((unsigned)s.nfb, (unsigned)s.split);
    fn<<<grid, kGlsThreads, 0, st>>>(recA, recB, q, N, s.chunk, (int)N_f, s.nf_pad, part,
                                      s.split == 1 ? P_out : nullptr);
    return cudaGetLastError();
}

using GlsMrhsFn = GlsBatchFn;

GlsMrhsFn gls_mrhs_fn(int F, int R) {
    if (F == 8 && R == 4) return gls_mrhs_kernel<8, 4, kGlsBatchTile>;
    if (F == 4 && R == 8) return gls_mrhs_kernel<4, 8, 64>;
    if (F == 8 && R == 2) return gls_mrhs_kernel<8, 2, kGlsBatchTile>;
    return nullptr;
}

int gls_mrhs_occupancy(int F, int R) {
    const GlsMrhsFn fn = gls_mrhs_fn(F, R);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kGlsBatchThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_gls_mrhs(int F, int R, int grid, const BatchItem* items, int n_items, unsigned* head,
                            const int64_t* off, const int64_t* nf, const uint4* recA, const float4* recB,
                            const float* q, float* P_out, const int64_t* P_off, unsigned long long* maxkey,
                            const float* xr, int64_t total, int64_t P_total, int n_curves, cudaStream_t st) {
    const GlsMrhsFn fn = gls_mrhs_fn(F, R);
    if (!fn || !xr) return cudaErrorInvalidValue;
    fn<<<grid, kGlsBatchThreads, 0, st>>>(items, n_items, head, off, nf, recA, recB, q, P_out, P_off, maxkey, xr,
                                          total, P_total, n_curves);
    return cudaGetLastError();
}

int gls_batch_occupancy(int mode, int F, bool packed, bool xrow) {
    const GlsBatchFn fn = gls_batch_fn(mode, F, packed, xrow);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kGlsBatchThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_gls_batch(int mode, int F, bool packed, int grid, const BatchItem* items, int n_items,
                             unsigned* head, const int64_t* off, const int64_t* nf, const uint4* recA,
                             const float4* recB, const float* q, float* P_out, const int64_t* P_off,
                             unsigned long long* maxkey, cudaStream_t st, const float* xr, int64_t total,
                             int64_t P_total, int n_curves) {
    const GlsBatchFn fn = gls_batch_fn(mode, F, packed, xr != nullptr);
    if (!fn) return cudaErrorInvalidValue;
    fn<<<grid, kGlsBatchThreads, 0, st>>>(items, n_items, head, off, nf, recA, recB, q, P_out, P_off, maxkey, xr,
                                          total, P_total, n_curves);
    return cudaGetLastError();
}

cudaError_t launch_gls_finalize(const MainShape& s, const float* part, int64_t N, int64_t N_f, float* P_out,
                                cudaStream_t st) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((N_f + threads - 1) / threads);
    gls_finalize_kernel<<<blocks, threads, 0, st>>>(part, s.split, s.nf_pad, (int)N_f, (double)N, P_out);
    return cudaGetLastError();
}

}  // namespace lsp
