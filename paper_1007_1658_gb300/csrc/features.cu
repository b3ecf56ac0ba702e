// features.cu -- sampling-pattern features for the learned false-alarm
// surrogate.
//
// The paper's false-alarm probability (Eq. 3) takes the N_f frequencies of a
// periodogram as independent; Sec. 6.2 notes that the exponent should really
// be an empirical number of independent frequencies, which depends on the
// sampling pattern.  The surrogate predicts the noise-peak quantiles from 32
// features of the pattern (definitions in include/lsp.h, lsp_fap_features).
// Two kernels:
//   ls_window_kernel  -- the spectral window W(f) = |sum_j e^{2 pi i f t_j}|^2 / N^2
//                        on f_m = m df, m = 1..floor(f_max / df): the same
//                        persistent tile loop as the batch periodogram, x = 1;
//   features_kernel   -- one CTA per pattern: cadence order statistics (a
//                        bitonic sort of the gaps in shared memory, or for
//                        patterns of more than 32,768 gaps a radix select of
//                        the five ranks over the gaps in global memory), gap
//                        fractions, and the 8 highest window maxima outside
//                        the main lobe (per-thread top-8 lists merged by
//                        warp shuffles).
#include <algorithm>
#include <cfloat>

#include "ls_device.cuh"

namespace lsp {
namespace {

using namespace dev;

constexpr int kFeatThreads = 1024;
constexpr int kSortMaxGaps = 32768;  // gaps sorted in shared memory (128 KB); more are selected

// The five cadence order statistics sorted(gaps)[k[i]] of a pattern too long
// for the shared-memory sort, without sorting: an MSB-first radix select on
// the FP32 bit patterns of the gaps (ordered as the values, gaps being >= 0),
// 8 bits per pass and the five ranks at once, the gaps re-formed from t in
// every pass exactly as the sort forms them.  Each warp adds to the five
// 256-bin histograms once per distinct bin (__match_any_sync), so gaps that
// share their leading bits do not serialize on one counter.  hist holds
// 5 x 256 counters; out[i] receives the value of rank k[i].
__device__ void select_gap_ranks(const double* __restrict__ t, int64_t b, int M, const int (&k)[5],
                                 unsigned* hist, float* out) {
    __shared__ unsigned s_prefix[5], s_rank[5];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    if (tid < 5) {
        s_prefix[tid] = 0u;
        s_rank[tid] = (unsigned)k[tid];
    }
    unsigned mask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 5 * 256; i += nt) hist[i] = 0u;
        __syncthreads();
        unsigned prefix[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) prefix[q] = s_prefix[q];
        // the whole warp steps together so that every lane takes part in the match
        for (int base = tid - lane; base < M; base += nt) {
            const int i = base + lane;
            unsigned key = 0u;
            if (i < M) key = __float_as_uint((float)(t[b + i + 1] - t[b + i]));
            const int bin = (int)((key >> shift) & 255u);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const int mine = (i < M && (key & mask) == prefix[q]) ? bin : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, mine);
                if (mine >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[q * 256 + mine], (unsigned)__popc(peers));
            }
        }
        __syncthreads();
        if (tid < 5) {
            // the bin holding rank s_rank: ranks below it move to the next pass's count
            unsigned r = s_rank[tid], acc = 0u;
            int bin = 0;
            for (; bin < 255; ++bin) {
                const unsigned c = hist[tid * 256 + bin];
                if (acc + c > r) break;
                acc += c;
            }
            s_rank[tid] = r - acc;
            s_prefix[tid] |= (unsigned)bin << shift;
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    if (tid < 5) out[tid] = __uint_as_float(s_prefix[tid]);
    __syncthreads();
}

template <int F>
__global__ void __launch_bounds__(kMainThreads)
ls_window_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                 const int64_t* __restrict__ off, const int64_t* __restrict__ nw, const uint4* __restrict__ recA,
                 const float4* __restrict__ recB, float* __restrict__ W, const int64_t* __restrict__ W_off) {
    __shared__ __align__(16) TileSmem<false> sm;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const int64_t b = off[w.curve], e = off[w.curve + 1];
        const int64_t M = nw[w.curve];
        const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) + (uint32_t)threadIdx.x * F;
        Strip<F, kRecur3x2> st;
        st.zero();
        for_each_tile<false>(sm, recA, recB, nullptr, b, e, [&](const uint4* a, const float4* bb, const float*, int n) {
#pragma unroll 2
            for (int j = 0; j < n; ++j) st.add(a[j], bb[j], 1.f, k0);
        });
        const float inv = 1.f / ((float)(e - b) * (float)(e - b));
        float* out = W + W_off[w.curve];
#pragma unroll
        for (int i = 0; i < F; ++i)
            if (k0 + i < (uint32_t)M) {
                float xc, xs, cc, cs;
                st.get(i, xc, xs, cc, cs);
                out[k0 + i] = (xc * xc + xs * xs) * inv;
            }
    }
}

// (value, bin) ordered by value, then by lower bin.
__device__ __forceinline__ bool better(float v, int m, float v2, int m2) { return v > v2 || (v == v2 && m < m2); }

__device__ __forceinline__ void top8_insert(float (&v)[8], int (&m)[8], float x, int mi) {
    if (!better(x, mi, v[7], m[7])) return;
    int p = 7;
    while (p > 0 && better(x, mi, v[p - 1], m[p - 1])) {
        v[p] = v[p - 1];
        m[p] = m[p - 1];
        --p;
    }
    v[p] = x;
    m[p] = mi;
}

// One CTA per pattern.  Dynamic shared memory: the gaps, padded to a power of
// two, for patterns of up to kSortMaxGaps gaps; the select's histograms for longer ones.
__global__ void __launch_bounds__(kFeatThreads)
features_kernel(const double* __restrict__ t, const int64_t* __restrict__ off, const double* __restrict__ f0a,
                const double* __restrict__ dfa, const int64_t* __restrict__ nfa, const float* __restrict__ W,
                const int64_t* __restrict__ W_off, const int64_t* __restrict__ nw, float* __restrict__ feat,
                int* __restrict__ status) {
    extern __shared__ float gaps[];
    __shared__ double red[33];
    __shared__ float wv[32 * 8];
    __shared__ int wm[32 * 8];
    __shared__ int unsorted;
    __shared__ float qsel[5];
    const int c = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t b = off[c], e = off[c + 1];
    const int n = (int)(e - b), M = n - 1;
    const double ps[5] = {0.05, 0.25, 0.5, 0.75, 0.95};
    int P2 = 1;
    while (P2 < M) P2 <<= 1;
    const bool sorted_in_smem = M <= kSortMaxGaps;
    if (tid == 0) unsorted = 0;
    __syncthreads();
    const double T = t[e - 1] - t[b];
    if (!sorted_in_smem) {
        int k[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) k[i] = (int)floor(ps[i] * (double)(M - 1));
        select_gap_ranks(t, b, M, k, (unsigned*)gaps, qsel);
        for (int i = tid; i < M; i += nt)
            if (t[b + i + 1] - t[b + i] < 0.0) unsorted = 1;
    }
    for (int i = tid; sorted_in_smem && i < P2; i += nt) {
        if (i < M) {
            const double d = t[b + i + 1] - t[b + i];
            if (d < 0.0) unsorted = 1;
            gaps[i] = (float)d;
        } else {
            gaps[i] = FLT_MAX;
        }
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; sorted_in_smem && k <= P2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P2; i += nt) {
                const int l = i ^ j;
                if (l > i) {
                    const float a = gaps[i], bb = gaps[l];
                    const bool up = (i & k) == 0;
                    if ((a > bb) == up) {
                        gaps[i] = bb;
                        gaps[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // q(ps[i]) = sorted(gaps)[floor(ps[i] (M - 1))]; the median is q(1/2)
    auto q = [&](int i) { return sorted_in_smem ? gaps[(int)floor(ps[i] * (double)(M - 1))] : qsel[i]; };
    const double med = (double)q(2);
    // gap sums over dt > c med (1 + 1e-6): the margin keeps exact multiples of
    // the cadence (one dropped sample on an even grid) out of the gaps
    double s2 = 0.0, s10 = 0.0, s100 = 0.0, cnt2 = 0.0, mx = 0.0;
    for (int i = tid; i < M; i += nt) {
        const double d = t[b + i + 1] - t[b + i];
        const double r = d / med;
        if (r > 2.0 * (1.0 + 1e-6)) {
            s2 += d;
            cnt2 += 1.0;
        }
        if (r > 10.0 * (1.0 + 1e-6)) s10 += d;
        if (r > 100.0 * (1.0 + 1e-6)) s100 += d;
        mx = fmax(mx, d);
    }
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        double r = tid < (nt >> 5) ? red[tid] : 0.0;
        if (tid < 32)
            for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (tid == 0) red[32] = r;
        __syncthreads();
        return red[32];
    };
    auto bmax = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        double r = tid < (nt >> 5) ? red[tid] : 0.0;
        if (tid < 32)
            for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
        if (tid == 0) red[32] = r;
        __syncthreads();
        return red[32];
    };
    s2 = bsum(s2);
    s10 = bsum(s10);
    s100 = bsum(s100);
    cnt2 = bsum(cnt2);
    mx = bmax(mx);

    // window maxima outside the main lobe: interior m with W[m] > W[m-1], W[m] >= W[m+1], f_m T >= 1
    const double df = dfa[c], f0 = f0a[c];
    const int64_t nf = nfa[c];
    const double f_max = f0 + (double)(nf - 1) * df;
    const int64_t mw = nw[c];
    const float* Wc = W + W_off[c];
    float tv[8];
    int tm[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        tv[r] = -1.f;
        tm[r] = 0x7fffffff;
    }
    for (int64_t i = 1 + tid; i + 1 < mw; i += nt) {
        const float w = Wc[i];
        if (w > Wc[i - 1] && w >= Wc[i + 1] && (double)(i + 1) * df * T >= 1.0) top8_insert(tv, tm, w, (int)i);
    }
    // warp merge: eight rounds of "best head in the warp wins"
    const int lane = tid & 31, warp = tid >> 5;
    int headp = 0;
    for (int r = 0; r < 8; ++r) {
        float bv = headp < 8 ? tv[headp] : -1.f;
        int bm = headp < 8 ? tm[headp] : 0x7fffffff;
        int bl = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int om = __shfl_xor_sync(0xffffffffu, bm, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (better(ov, om, bv, bm)) {
                bv = ov;
                bm = om;
                bl = ol;
            }
        }
        if (lane == bl) ++headp;
        if (lane == 0) {
            wv[warp * 8 + r] = bv;
            wm[warp * 8 + r] = bm;
        }
    }
    __syncthreads();
    if (tid == 0) {
        float fv[8];
        int fm[8];
        for (int r = 0; r < 8; ++r) {
            fv[r] = -1.f;
            fm[r] = 0x7fffffff;
        }
        for (int i = 0; i < (nt >> 5) * 8; ++i)
            if (wv[i] >= 0.f) top8_insert(fv, fm, wv[i], wm[i]);
        float* o = feat + (size_t)c * 32;
        const float nanv = __int_as_float(0x7fc00000);
        if (unsorted || !(T > 0.0) || M < 1) {
            for (int i = 0; i < 32; ++i) o[i] = nanv;
            atomicOr(status, kStatusNonFinite);
            return;
        }
        const double meanGap = T / (double)M;
        o[0] = (float)log((double)n);
        o[1] = (float)log(T);
        o[2] = (float)log((double)nf);
        o[3] = (float)log(1.0 / (df * T));
        o[4] = (float)log(f_max * T / (double)n);
        o[5] = (float)log1p(f0 / df);
        for (int i = 0; i < 5; ++i) o[6 + i] = (float)log(fmax((double)q(i), 1e-12 * T) / meanGap);
        o[11] = (float)(s2 / T);
        o[12] = (float)(s10 / T);
        o[13] = (float)(s100 / T);
        o[14] = (float)(mx / T);
        o[15] = (float)(cnt2 / (double)M);
        for (int r = 0; r < 8; ++r) {
            const bool ok = fv[r] >= 0.f;
            o[16 + r] = ok ? fv[r] : 0.f;
            o[24 + r] = ok ? (float)((double)(fm[r] + 1) * df / f_max) : 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_window(int F, int grid, const BatchItem* items, int n_items, unsigned* head, const int64_t* off,
                          const int64_t* nw, const uint4* recA, const float4* recB, float* W, const int64_t* W_off,
                          cudaStream_t st) {
    switch (F) {
        case 8: ls_window_kernel<8><<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nw, recA, recB, W, W_off); break;
        case 16: ls_window_kernel<16><<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nw, recA, recB, W, W_off); break;
        case 24: ls_window_kernel<24><<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nw, recA, recB, W, W_off); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int window_occupancy(int F) {
    const void* fn = F == 8 ? (const void*)ls_window_kernel<8> : F == 16 ? (const void*)ls_window_kernel<16>
                                                                           : (const void*)ls_window_kernel<24>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kMainThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

size_t features_smem_bytes(int64_t max_n) {
    int64_t P2 = 1;
    while (P2 < max_n - 1 && P2 < kSortMaxGaps) P2 <<= 1;
    return std::max((size_t)P2 * sizeof(float), (size_t)5 * 256 * sizeof(unsigned));
}

cudaError_t launch_features(int n_patterns, int64_t max_n, const double* t, const int64_t* off, const double* f0,
                            const double* df, const int64_t* nf, const float* W, const int64_t* W_off,
                            const int64_t* nw, float* feat, int* status, cudaStream_t st) {
    const size_t smem = features_smem_bytes(max_n);
    cudaError_t e = cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    features_kernel<<<n_patterns, kFeatThreads, smem, st>>>(t, off, f0, df, nf, W, W_off, nw, feat, status);
    return cudaGetLastError();
}

}  // namespace lsp
