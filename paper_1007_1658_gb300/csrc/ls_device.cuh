// ls_device.cuh -- device-side pieces of the O(N_t N_f) evaluation shared by
// the single-curve kernels (ls_main.cu) and the batched Monte-Carlo kernel
// (batch.cu): phase handling, the per-sample update of one frequency strip
// in each sin/cos mode, the cp.async tile pipeline and Eq. 5-6.
#pragma once

#include <cstdint>

#include "lsp_kernels.cuh"

namespace lsp {
namespace dev {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kThreePi = 9.42477796076937971538f;

// Internal kernel modes (the kMode* values of lsp_kernels.cuh).
enum : int {
    kMufu = kModeMufu,
    kRecur = kModeRecur,
    kNaive = kModeNaive,
    kRecur3 = kModeRecur3,
    kRecur3x2 = kModeRecur3x2
};

// Top 23 bits of a 32-bit turn fraction, offset by half a turn at prep time,
// become a float in [1, 2) by pasting them under the exponent of 1.0; one FMA
// maps that to an angle in [-pi, pi).  No int->float conversion unit is used.
__device__ __forceinline__ float phase_to_angle(uint32_t p) {
    return fmaf(__uint_as_float(0x3F800000u | (p >> 9)), kTwoPi, -kThreePi);
}

// Top 32 bits of the phase v + k u (mod 2^64) of record A at frequency k.
__device__ __forceinline__ uint32_t top_phase(const uint4& A, uint32_t k) {
    const uint64_t u = ((uint64_t)A.y << 32) | A.x;
    const uint64_t v = ((uint64_t)A.w << 32) | A.z;
    return (uint32_t)((v + (uint64_t)k * u) >> 32);
}

// The same word from 32-bit products only: v_hi + k u_hi + hi(k u_lo).  The
// carry of the low word (v_lo + lo(k u_lo)) is left out, so the result is the
// exact top word or one less: an error below 2^-32 turn, far under the
// 2^-23-turn step of the FP32 angle taken from it (the 2^40 rounding offset
// in v sits in the top word and still rounds that step).  Measured faster in
// the six-sum floating-mean strips, slower in the four-sum ones.
__device__ __forceinline__ uint32_t top_phase_hi(const uint4& A, uint32_t k) {
    return __umulhi(k, A.x) + k * A.y + A.w;
}

// round(u / 2^32) of record A: the phase step of one frequency bin in the
// 32-bit turns that top_phase returns (the MUFU strips add it per bin).
__device__ __forceinline__ uint32_t round_top_word(const uint4& A) { return A.y + (A.x >> 31); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Fixed-order compensated (Neumaier) FP32 sum, over the `split` sample
// chunks, of the R partial sums of frequency k (row r of chunk sp at
// part[(sp R + r) nf_pad + k]); leaves the sums in s and their corrections in
// c.  The loads of 8 chunks are issued before any of them is added, so a
// thread waits on memory once per 8 chunks instead of once per chunk; the
// additions keep the chunk order, so the result does not depend on that.
template <int R>
__device__ __forceinline__ void merge_chunks(const float* __restrict__ part, int split, int64_t nf_pad, int k,
                                             float (&s)[R], float (&c)[R]) {
    constexpr int kB = 8;
#pragma unroll
    for (int r = 0; r < R; ++r) s[r] = c[r] = 0.f;
    for (int sp0 = 0; sp0 < split; sp0 += kB) {
        float v[kB][R];
#pragma unroll
        for (int u = 0; u < kB; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[u][r] = sp0 + u < split ? part[((size_t)(sp0 + u) * R + r) * (size_t)nf_pad + k] : 0.f;
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (sp0 + u < split) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float x = v[u][r];
                    const float t = s[r] + x;
                    c[r] += fabsf(s[r]) >= fabsf(x) ? (s[r] - t) + x : (x - t) + s[r];
                    s[r] = t;
                }
            }
        }
    }
}

// Eq. 5 with tau from Eq. 6, in closed form.  With A = CC - SS = 2CC - N,
// B = 2CS and R = |A + iB| = |sum exp(2 i w t_j)|, tan 2wtau = B/A gives
// cos 2wtau = A/R, sin 2wtau = B/R, and the two denominators of Eq. 5 are
// (N + R)/2 and (N - R)/2; the two numerators are (|Z|^2 +- Re(e^{-2iwtau} Z^2))/2
// with Z = XC + i XS.  No trig, and R = 0 (tau undefined) takes wtau = 0.
// A term whose denominator is below N 2^-16 is taken as zero.  A NaN among
// the sums (non-finite data, or data the prep kernels refused) gives NaN: the
// clamps and threshold tests below would otherwise turn it into 0.
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
    const float probe = z2 + R;
    return probe == probe ? 0.5f * P : probe;
}

// The four running sums of Eq. 8 for a strip of F adjacent frequencies
// k0 .. k0+F-1 of one thread.
template <int F, int MODE>
struct Strip {
    float xc[F], xs[F], cc[F], cs[F];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) xc[i] = xs[i] = cc[i] = cs[i] = 0.f;
    }

    __device__ __forceinline__ void get(int i, float& xc_, float& xs_, float& cc_, float& cs_) const {
        xc_ = xc[i];
        xs_ = xs[i];
        cc_ = cc[i];
        cs_ = cs[i];
    }

    __device__ __forceinline__ void acc(int i, float x, float c, float s) {
        xc[i] = fmaf(x, c, xc[i]);
        xs[i] = fmaf(x, s, xs[i]);
        cc[i] = fmaf(c, c, cc[i]);
        cs[i] = fmaf(c, s, cs[i]);
    }

    // Sample with phase record A = {u, v}, B = {x_hat, cos 2 pi u, sin 2 pi u,
    // 2 cos 2 pi u} and normalized value x.  C2_REC takes the recurrence factor
    // from the record, else it is formed as 2 B.y (the same value): which is
    // faster depends on the kernel around the strip, so each kernel picks.
    template <bool C2_REC = true>
    __device__ __forceinline__ void add(const uint4& A, const float4& B, float x, uint32_t k0) {
        uint32_t p = top_phase(A, k0);
        if (MODE == kMufu) {
            const uint32_t du = round_top_word(A);
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float s, c;
                __sincosf(phase_to_angle(p), &s, &c);
                acc(i, x, c, s);
                p += du;
            }
        } else {
            // seed from the exact phase, then step k -> k+1 by the rotation
            // (cos, sin)(2 pi u): RECUR uses the angle-addition formulas at
            // every step; RECUR3 uses them once and then the three-term form
            // z_{i+1} = 2 cos(2 pi u) z_i - z_{i-1}.
            const float C = B.y, S = B.z, C2 = C2_REC ? B.w : 2.f * B.y;
            float s, c;
            __sincosf(phase_to_angle(p), &s, &c);
            float cp = c, sp = s;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                acc(i, x, c, s);
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

// Packed FP32x2 form of the three-term strip for the four-sum kernels: the
// (cos, sin) pair of a frequency sits in the two lanes of an FFMA2, and every
// operation of a term is one FFMA2 -- (XC, XS) with the pair (x, x), (CC, CS)
// with the pair (c, c), and the three-term step -- with no scalar FFMA
// between them.  FFMA2 has no negated addend, so the lanes carry y_i = g_i z_i
// with g = (+, +, -, -, +, +, ...): z_{i+1} = 2C z_i - z_{i-1} becomes
// y_{i+1} = (i odd ? -2C : 2C) y_i + y_{i-1}.  (XC, XS) is kept as g_i times
// the sums (g_i is the same for every sample) and read back through get();
// c c and c s do not see the sign.  Round to nearest is symmetric, so every
// sum is bit for bit Strip<F, kRecur3>'s.
template <int F>
struct Strip<F, kRecur3x2> {
    float2 xcs[F], ccs[F];  // g_i (XC, XS) and (CC, CS) of frequency i

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) xcs[i] = ccs[i] = make_float2(0.f, 0.f);
    }

    __device__ __forceinline__ void get(int i, float& xc, float& xs, float& cc, float& cs) const {
        const bool neg = (i >> 1) & 1;
        xc = neg ? -xcs[i].x : xcs[i].x;
        xs = neg ? -xcs[i].y : xcs[i].y;
        cc = ccs[i].x;
        cs = ccs[i].y;
    }

    __device__ __forceinline__ void acc(int i, float2 xp, float2 y) {
        xcs[i] = __ffma2_rn(xp, y, xcs[i]);
        ccs[i] = __ffma2_rn(make_float2(y.x, y.x), y, ccs[i]);
    }

    template <bool C2_REC = true>
    __device__ __forceinline__ void add(const uint4& A, const float4& B, float x, uint32_t k0) {
        const float C = B.y, S = B.z, C2 = C2_REC ? B.w : 2.f * B.y;
        float s, c;
        __sincosf(phase_to_angle(top_phase(A, k0)), &s, &c);
        const float2 xp = make_float2(x, x);
        float2 y0 = make_float2(c, s);
        acc(0, xp, y0);
        if (F == 1) return;
        // first step by angle addition, as the scalar strip takes it
        float2 y1 = make_float2(fmaf(c, C, -s * S), fmaf(s, C, c * S));
        acc(1, xp, y1);
        const float2 cp2 = make_float2(C2, C2), cn2 = make_float2(-C2, -C2);
#pragma unroll
        for (int i = 2; i < F; ++i) {
            const float2 y2 = __ffma2_rn(((i - 1) & 1) ? cn2 : cp2, y1, y0);
            acc(i, xp, y2);
            y0 = y1;
            y1 = y2;
        }
    }
};

// Multi-right-hand-side strip: R realizations of one sampling pattern share
// the phase, the sin/cos recurrence and the CC, CS sums; each keeps its own
// XC, XS.  Per term and realization: 2 FFMA plus (2 recurrence + 2 CC/CS)/R,
// instead of 6.  The arithmetic of every (frequency, realization) pair is the
// single-realization strip's, in the same order, so results are identical.
// With CCS false the strip leaves CC and CS out (they depend on the sampling
// pattern only, and WStrip computes them once for all groups): 2 + 2/R per
// term and realization, and 2F fewer registers.
template <int F, int R, int MODE, bool CCS = true>
struct MStrip {
    float xc[F][R], xs[F][R], cc[F], cs[F];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) {
            cc[i] = cs[i] = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) xc[i][r] = xs[i][r] = 0.f;
        }
    }

    __device__ __forceinline__ float get_xc(int i, int r) const { return xc[i][r]; }
    __device__ __forceinline__ float get_xs(int i, int r) const { return xs[i][r]; }
    __device__ __forceinline__ float get_cc(int i) const { return cc[i]; }
    __device__ __forceinline__ float get_cs(int i) const { return cs[i]; }

    __device__ __forceinline__ void acc(int i, const float (&x)[R], float c, float s) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            xc[i][r] = fmaf(x[r], c, xc[i][r]);
            xs[i][r] = fmaf(x[r], s, xs[i][r]);
        }
        if (CCS) {
            cc[i] = fmaf(c, c, cc[i]);
            cs[i] = fmaf(c, s, cs[i]);
        }
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, const float (&x)[R], uint32_t k0) {
        uint32_t p = top_phase(A, k0);
        if (MODE == kMufu) {
            const uint32_t du = round_top_word(A);
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float s, c;
                __sincosf(phase_to_angle(p), &s, &c);
                acc(i, x, c, s);
                p += du;
            }
        } else {
            const float C = B.y, S = B.z, C2 = B.w;
            float s, c;
            __sincosf(phase_to_angle(p), &s, &c);
            float cp = c, sp = s;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                acc(i, x, c, s);
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

// Packed form of the multi-realization strip: the (cos, sin) pair of a
// frequency sits in the two lanes of an FFMA2, so (XC, XS) of one realization
// take one FFMA2 per term, (CC, CS) -- when the strip keeps them (CCS) -- one
// FFMA2 with the pair (c, c), and the three-term step one FFMA2 for both
// lanes: the FMA pipe does the same lane operations as the scalar strip in
// half the issue slots, with no scalar FFMA between the packed ones.  FFMA2
// has no negated addend, so the lanes carry y_i = g_i z_i with the signs
// g = (+, +, -, -, +, +, ...) of the other packed strips, and the running sums
// are kept as g_i (XC, XS): g_i is the same for every sample, and round to
// nearest is symmetric, so g_i times the sums is bit for bit
// MStrip<F, R, kRecur3, CCS>'s XC and XS (c c and c s do not see the sign).
template <int F, int R, bool CCS>
struct MStrip<F, R, kRecur3x2, CCS> {
    float2 a[F][R];                // g_i (XC, XS) of frequency i, realization r
    float2 w[CCS ? F : 1];         // (CC, CS) of frequency i

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) {
            if (CCS) w[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) a[i][r] = make_float2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ float get_xc(int i, int r) const { return ((i >> 1) & 1) ? -a[i][r].x : a[i][r].x; }
    __device__ __forceinline__ float get_xs(int i, int r) const { return ((i >> 1) & 1) ? -a[i][r].y : a[i][r].y; }
    __device__ __forceinline__ float get_cc(int i) const { return CCS ? w[i].x : 0.f; }
    __device__ __forceinline__ float get_cs(int i) const { return CCS ? w[i].y : 0.f; }

    __device__ __forceinline__ void acc(int i, const float2 (&xp)[R], float2 y) {
#pragma unroll
        for (int r = 0; r < R; ++r) a[i][r] = __ffma2_rn(xp[r], y, a[i][r]);
        if (CCS) w[i] = __ffma2_rn(make_float2(y.x, y.x), y, w[i]);
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, const float (&x)[R], uint32_t k0) {
        const float C = B.y, S = B.z, C2 = B.w;
        float s, c;
        __sincosf(phase_to_angle(top_phase(A, k0)), &s, &c);
        float2 xp[R];
#pragma unroll
        for (int r = 0; r < R; ++r) xp[r] = make_float2(x[r], x[r]);
        float2 y0 = make_float2(c, s);
        acc(0, xp, y0);
        if (F == 1) return;
        // first step by angle addition, as the scalar strip takes it
        float2 y1 = make_float2(fmaf(c, C, -s * S), fmaf(s, C, c * S));
        acc(1, xp, y1);
        const float2 cp2 = make_float2(C2, C2), cn2 = make_float2(-C2, -C2);
#pragma unroll
        for (int i = 2; i < F; ++i) {
            const float2 y2 = __ffma2_rn(((i - 1) & 1) ? cn2 : cp2, y1, y0);
            acc(i, xp, y2);
            y0 = y1;
            y1 = y2;
        }
    }
};

// The window sums CC = sum cos^2 and CS = sum cos sin of Eq. 8 alone, for a
// strip of F frequencies: the same seed, step and order as MStrip (and Strip)
// of the same F and k0, so the sums are bit for bit theirs.  They do not
// depend on the data, so one pass per sampling pattern serves every group of
// realizations of that pattern.
template <int F, int MODE>
struct WStrip {
    float cc[F], cs[F];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) cc[i] = cs[i] = 0.f;
    }

    __device__ __forceinline__ float get_cc(int i) const { return cc[i]; }
    __device__ __forceinline__ float get_cs(int i) const { return cs[i]; }

    __device__ __forceinline__ void acc(int i, float c, float s) {
        cc[i] = fmaf(c, c, cc[i]);
        cs[i] = fmaf(c, s, cs[i]);
    }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, uint32_t k0) {
        uint32_t p = top_phase(A, k0);
        if (MODE == kMufu) {
            const uint32_t du = round_top_word(A);
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float s, c;
                __sincosf(phase_to_angle(p), &s, &c);
                acc(i, c, s);
                p += du;
            }
        } else {
            const float C = B.y, S = B.z, C2 = B.w;
            float s, c;
            __sincosf(phase_to_angle(p), &s, &c);
            float cp = c, sp = s;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                acc(i, c, s);
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

// Packed form of the window strip: the (cos, sin) pair in the two lanes,
// (CC, CS) one FFMA2 with the pair (c, c) and the three-term step one FFMA2
// per term (signs folded into y as in the other packed strips; c c and c s do
// not see them), bit for bit WStrip<F, kRecur3>'s sums.
template <int F>
struct WStrip<F, kRecur3x2> {
    float2 w[F];  // (CC, CS) of frequency i

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < F; ++i) w[i] = make_float2(0.f, 0.f);
    }

    __device__ __forceinline__ void acc(int i, float2 y) { w[i] = __ffma2_rn(make_float2(y.x, y.x), y, w[i]); }

    __device__ __forceinline__ void add(const uint4& A, const float4& B, uint32_t k0) {
        const float C = B.y, S = B.z, C2 = B.w;
        float s, c;
        __sincosf(phase_to_angle(top_phase(A, k0)), &s, &c);
        float2 y0 = make_float2(c, s);
        acc(0, y0);
        if (F == 1) return;
        float2 y1 = make_float2(fmaf(c, C, -s * S), fmaf(s, C, c * S));
        acc(1, y1);
        const float2 cp2 = make_float2(C2, C2), cn2 = make_float2(-C2, -C2);
#pragma unroll
        for (int i = 2; i < F; ++i) {
            const float2 y2 = __ffma2_rn(((i - 1) & 1) ? cn2 : cp2, y1, y0);
            acc(i, y2);
            y0 = y1;
            y1 = y2;
        }
    }

    __device__ __forceinline__ float get_cc(int i) const { return w[i].x; }
    __device__ __forceinline__ float get_cs(int i) const { return w[i].y; }
};

// One 128-bit shared-memory load of a 16-byte record.  A float4 whose fourth
// word goes unused is split by the compiler into narrower loads: one more
// instruction per sample.
__device__ __forceinline__ uint4 lds128(const void* p) {
    uint4 r;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"(a)
                 : "memory");
    return r;
}

// The samples of one staged tile through a strip, x from the records: each
// record pair with two 128-bit loads, and full tiles (n == TILE) with a
// constant trip count.  Measured with one-warp CTAs: 1.3% faster for the
// single-curve kernel, 14% for the batch kernel (76.6 -> 65.9 ms on the
// 4096-curve Monte Carlo), than float4 loads in a loop over n.
template <int TILE, bool C2_REC = true, class S>
__device__ __forceinline__ void strip_tile(S& st, const uint4* a, const float4* b, int n, uint32_t k0) {
    auto sample = [&](int j) {
        const uint4 A = lds128(a + j);
        const uint4 Bu = lds128(b + j);
        const float4 B = make_float4(__uint_as_float(Bu.x), __uint_as_float(Bu.y), __uint_as_float(Bu.z),
                                     __uint_as_float(Bu.w));
        st.template add<C2_REC>(A, B, B.x, k0);
    };
    if (n == TILE) {
#pragma unroll 2
        for (int j = 0; j < TILE; ++j) sample(j);
    } else {
#pragma unroll 2
        for (int j = 0; j < n; ++j) sample(j);
    }
}

// Double-buffered cp.async pipeline over the samples [j0, j1) in tiles of
// TILE samples (kTile unless a kernel is built for another tile length):
// stages the two 16-byte phase records of every sample and, when `xr` is
// given, the sample values from that array; calls body(a, b, x, n) once per
// tile with the tile in shared memory.  Every thread of the CTA must call it
// (it synchronizes the CTA).  NX rows of x values may come along: row r of a
// tile is xr[r * xstride + j].
template <int NX, int TILE = kTile>
struct TileSmemN {
    uint4 A[2][TILE];
    float4 B[2][TILE];
    float X[2][NX > 0 ? NX : 1][NX > 0 ? TILE : 1];
};

template <bool XARR, int TILE = kTile>
using TileSmem = TileSmemN<XARR ? 1 : 0, TILE>;

template <int NX, int TILE, class Body>
__device__ __forceinline__ void for_each_tile_n(TileSmemN<NX, TILE>& sm, const uint4* __restrict__ recA,
                                                const float4* __restrict__ recB, const float* __restrict__ xr,
                                                int64_t xstride, int nx_valid, int64_t j0, int64_t j1,
                                                Body&& body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + TILE - 1) / TILE) : 0;
    auto stage = [&](int buf, int64_t jt) {
        const int n = (int)min((int64_t)TILE, j1 - jt);
        for (int q = tid; q < n; q += nt) {
            cp_async16(&sm.A[buf][q], recA + jt + q);
            cp_async16(&sm.B[buf][q], recB + jt + q);
#pragma unroll
            for (int r = 0; r < NX; ++r) {
                if (r < nx_valid)
                    cp_async4(&sm.X[buf][r][q], xr + (size_t)r * (size_t)xstride + jt + q);
                else
                    sm.X[buf][r][q] = 0.f;  // missing realizations of the last group add nothing
            }
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
        const int n = (int)min((int64_t)TILE, j1 - jt);
        body(sm.A[it & 1], sm.B[it & 1], sm.X[it & 1], n);
        __syncthreads();
    }
}

template <bool XARR, int TILE, class Body>
__device__ __forceinline__ void for_each_tile(TileSmem<XARR, TILE>& sm, const uint4* __restrict__ recA,
                                              const float4* __restrict__ recB, const float* __restrict__ xr,
                                              int64_t j0, int64_t j1, Body&& body) {
    for_each_tile_n<XARR ? 1 : 0, TILE>(sm, recA, recB, xr, 0, XARR ? 1 : 0, j0, j1,
                                        [&](const uint4* a, const float4* b, const float (*x)[XARR ? TILE : 1],
                                            int n) { body(a, b, XARR ? x[0] : nullptr, n); });
}

}  // namespace dev
}  // namespace lsp
