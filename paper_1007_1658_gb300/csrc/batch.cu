// batch.cu -- many periodograms in one persistent kernel (lsp_batch).
//
// Sec. 6.2 of the paper points at Monte-Carlo simulation of periodogram
// statistics (e.g. the number of independent frequencies behind Eq. 3) as a
// natural use of a GPU: many noise periodograms of the same sampling
// pattern.  Here a batch of curves with uneven N_t and N_f (CSR layout), each
// with one or many noise realizations, is evaluated by one persistent kernel:
// CTAs take work items -- (realization, curve, block of kMainThreads*F
// frequencies) -- from an atomic ticket in the order the host sorted them
// (longest curve first, so the tail of the run is made of the shortest items),
// run the same tile loop as the single-curve kernel over all samples of the
// curve, finish Eq. 5-6 in registers, write P if asked, and fold the block's
// largest P into the curve's maximum with one 64-bit atomicMax on
// (bits of P) << 32 | ~k, which keeps the lowest k on ties.  Nothing ever
// waits on another CTA: a CTA with no ticket left simply exits.
#include "ls_device.cuh"

namespace lsp {
namespace {

using namespace dev;

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Strip length of the tail items: the frequencies of a curve left over after
// its full blocks of kMainThreads*F run in blocks of kMainThreads*kTailF, so
// at most kMainThreads*kTailF - 1 slots per curve are padding.
constexpr int kTailF = kBatchTailF;

// One work item with strips of FF frequencies starting at k0: the tile loop
// over all samples of the curve, Eq. 5-6, P written if asked; returns this
// thread's largest (P bits << 32 | ~k) key.
template <int FF, int MODE, bool XREC, class SM>
__device__ __forceinline__ unsigned long long batch_item(SM& sm, uint32_t k0, int64_t b, int64_t e, int64_t N_f,
                                                        const uint4* __restrict__ recA,
                                                        const float4* __restrict__ recB, const float* x,
                                                        float* P) {
    Strip<FF, MODE> st;
    st.zero();
    if constexpr (XREC) {
        // the single-curve kernel's loop: x from the records
        for_each_tile<false>(sm, recA, recB, nullptr, b, e, [&](const uint4* a, const float4* bb, const float*, int n) {
#pragma unroll 2
            for (int j = 0; j < n; ++j) {
                const float4 B = bb[j];
                st.add(a[j], B, B.x, k0);
            }
        });
    } else {
        for_each_tile<true>(sm, recA, recB, x, b, e, [&](const uint4* a, const float4* bb, const float* xs, int n) {
#pragma unroll 2
            for (int j = 0; j < n; ++j) st.add(a[j], bb[j], xs[j], k0);
        });
    }
    const float n = (float)(e - b);
    unsigned long long best = 0ull;
#pragma unroll
    for (int i = 0; i < FF; ++i) {
        const uint32_t k = k0 + i;
        if (k < (uint32_t)N_f) {
            float xc, xs, cc, cs;
            st.get(i, xc, xs, cc, cs);
            const float p = periodogram_value(xc, xs, cc, cs, n);
            if (P) P[k] = p;
            best = umax64(best, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(~k));
        }
    }
    return best;
}

template <int F, int MODE, bool XREC>
__global__ void __launch_bounds__(kMainThreads)
ls_batch_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                const int64_t* __restrict__ off, const int64_t* __restrict__ nf, int64_t total, int n_curves,
                const uint4* __restrict__ recA, const float4* __restrict__ recB, const float* __restrict__ xr,
                float* __restrict__ P_out, const int64_t* __restrict__ P_off, int64_t P_total,
                unsigned long long* __restrict__ maxkey) {
    __shared__ __align__(16) TileSmem<!XREC> sm;
    __shared__ int s_item;
    __shared__ unsigned long long s_red[kMainThreads / 32];
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const int64_t b = off[w.curve], e = off[w.curve + 1];
        const int64_t N_f = nf[w.curve];
        const float* x = xr + (size_t)w.real * (size_t)total;
        float* P = P_out ? P_out + (size_t)w.real * (size_t)P_total + P_off[w.curve] : nullptr;
        unsigned long long best;
        if (F > kTailF && w.pad < 0) {
            // tail item: sub-block (-1 - pad) of kMainThreads*kTailF after fblock full blocks
            const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) +
                                (uint32_t)(-1 - w.pad) * (kMainThreads * kTailF) + (uint32_t)threadIdx.x * kTailF;
            best = batch_item<kTailF, MODE, XREC>(sm, k0, b, e, N_f, recA, recB, x, P);
        } else {
            const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) + (uint32_t)threadIdx.x * F;
            best = batch_item<F, MODE, XREC>(sm, k0, b, e, N_f, recA, recB, x, P);
        }
        for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_down_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = s_red[0];
            for (int q = 1; q < kMainThreads / 32; ++q) m = umax64(m, s_red[q]);
            if (m) atomicMax(&maxkey[(size_t)w.real * n_curves + w.curve], m);
        }
    }
}

// Multi-RHS variant for many realizations of the same patterns: an item is
// (curve, frequency block, group of up to R realizations starting at
// w.real; w.pad = group size), and the group shares the phase, the
// recurrence and CC/CS (MStrip).  Per (frequency, realization) the result is
// the single-realization kernel's, bit for bit.
template <int F, int R, int MODE>
__global__ void __launch_bounds__(kMainThreads)
ls_mrhs_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
               const int64_t* __restrict__ off, const int64_t* __restrict__ nf, int64_t total, int n_curves,
               const uint4* __restrict__ recA, const float4* __restrict__ recB, const float* __restrict__ xr,
               float* __restrict__ P_out, const int64_t* __restrict__ P_off, int64_t P_total,
               unsigned long long* __restrict__ maxkey) {
    __shared__ __align__(16) TileSmemN<R> sm;
    __shared__ int s_item;
    __shared__ unsigned long long s_red[R][kMainThreads / 32];
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
        const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) + (uint32_t)threadIdx.x * F;
        MStrip<F, R, MODE> st;
        st.zero();
        for_each_tile_n<R>(sm, recA, recB, xr + (size_t)w.real * (size_t)total, total, nr, b, e,
                           [&](const uint4* a, const float4* bb, const float (*xs)[kTile], int n) {
                               for (int j = 0; j < n; ++j) {
                                   float x[R];
#pragma unroll
                                   for (int r = 0; r < R; ++r) x[r] = xs[r][j];
                                   st.add(a[j], bb[j], x, k0);
                               }
                           });
        const float n = (float)(e - b);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            unsigned long long best = 0ull;
            float* P = (P_out && r < nr) ? P_out + (size_t)(w.real + r) * (size_t)P_total + P_off[w.curve] : nullptr;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                const uint32_t k = k0 + i;
                if (k < (uint32_t)N_f && r < nr) {
                    const float p = periodogram_value(st.xc[i][r], st.xs[i][r], st.cc[i], st.cs[i], n);
                    if (P) P[k] = p;
                    best = umax64(best, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(~k));
                }
            }
            for (int o = 16; o > 0; o >>= 1) best = umax64(best, __shfl_down_sync(0xffffffffu, best, o));
            if ((threadIdx.x & 31) == 0) s_red[r][threadIdx.x >> 5] = best;
        }
        __syncthreads();
        if (threadIdx.x < R && (int)threadIdx.x < nr) {
            const int r = threadIdx.x;
            unsigned long long m = s_red[r][0];
            for (int q = 1; q < kMainThreads / 32; ++q) m = umax64(m, s_red[r][q]);
            if (m) atomicMax(&maxkey[(size_t)(w.real + r) * n_curves + w.curve], m);
        }
    }
}

// maxkey -> (max P, argmax k); a curve with no frequency gets (0, -1).
__global__ void unpack_max_kernel(const unsigned long long* __restrict__ maxkey, int64_t n, float* __restrict__ maxP,
                                  int32_t* __restrict__ argmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long key = maxkey[i];
    if (maxP) maxP[i] = key ? __uint_as_float((uint32_t)(key >> 32)) : 0.f;
    if (argmax) argmax[i] = key ? (int32_t)(~(uint32_t)key) : -1;
}

using BatchFn = void (*)(const BatchItem*, int, unsigned*, const int64_t*, const int64_t*, int64_t, int,
                         const uint4*, const float4*, const float*, float*, const int64_t*, int64_t,
                         unsigned long long*);

template <int MODE, bool XREC>
BatchFn batch_fn_f(int F) {
    switch (F) {
        case 4: return ls_batch_kernel<4, MODE, XREC>;
        case 8: return ls_batch_kernel<8, MODE, XREC>;
        case 12: return ls_batch_kernel<12, MODE, XREC>;
        case 16: return ls_batch_kernel<16, MODE, XREC>;
        case 20: return MODE == kMufu ? nullptr : ls_batch_kernel<20, MODE, XREC>;
        case 24: return ls_batch_kernel<24, MODE, XREC>;
        case 28: return MODE == kMufu ? nullptr : ls_batch_kernel<28, MODE, XREC>;
        default: return nullptr;
    }
}

template <bool XREC>
BatchFn batch_fn_x(int mode, int F) {
    switch (mode) {
        case kMufu: return batch_fn_f<kMufu, XREC>(F);
        case kRecur: return batch_fn_f<kRecur, XREC>(F);
        case kRecur3: return batch_fn_f<kRecur3, XREC>(F);
        case kRecur3x2: return batch_fn_f<kRecur3x2, XREC>(F);
        default: return nullptr;
    }
}

BatchFn batch_fn(int mode, int F, bool xrec) { return xrec ? batch_fn_x<true>(mode, F) : batch_fn_x<false>(mode, F); }

using MrhsFn = BatchFn;

// Multi-RHS shapes: F frequencies x R realizations per thread.
template <int MODE>
MrhsFn mrhs_fn_f(int F, int R) {
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, MODE>;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, MODE>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, MODE>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, MODE>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, MODE>;
    return nullptr;
}

MrhsFn mrhs_fn(int mode, int F, int R) {
    switch (mode) {
        case kMufu: return mrhs_fn_f<kMufu>(F, R);
        case kRecur: return mrhs_fn_f<kRecur>(F, R);
        case kRecur3:
        case kRecur3x2: return mrhs_fn_f<kRecur3>(F, R);  // shared-recurrence strips use the scalar form
        default: return nullptr;
    }
}

}  // namespace

int mrhs_occupancy(int mode, int F, int R) {
    MrhsFn fn = mrhs_fn(mode, F, R);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kMainThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_mrhs(int mode, int F, int R, int grid, const BatchItem* items, int n_items, unsigned* head,
                        const int64_t* off, const int64_t* nf, int64_t total, int n_curves, const uint4* recA,
                        const float4* recB, const float* xr, float* P_out, const int64_t* P_off, int64_t P_total,
                        unsigned long long* maxkey, cudaStream_t st) {
    MrhsFn fn = mrhs_fn(mode, F, R);
    if (!fn) return cudaErrorInvalidValue;
    fn<<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nf, total, n_curves, recA, recB, xr, P_out, P_off,
                                      P_total, maxkey);
    return cudaGetLastError();
}

int batch_occupancy(int mode, int F, bool x_in_records) {
    BatchFn fn = batch_fn(mode, F, x_in_records);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kMainThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

cudaError_t launch_batch(int mode, int F, bool x_in_records, int grid, const BatchItem* items, int n_items,
                         unsigned* head, const int64_t* off, const int64_t* nf, int64_t total, int n_curves,
                         const uint4* recA, const float4* recB, const float* xr, float* P_out, const int64_t* P_off,
                         int64_t P_total, unsigned long long* maxkey, cudaStream_t st) {
    BatchFn fn = batch_fn(mode, F, x_in_records);
    if (!fn) return cudaErrorInvalidValue;
    fn<<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nf, total, n_curves, recA, recB, xr, P_out, P_off,
                                      P_total, maxkey);
    return cudaGetLastError();
}

cudaError_t launch_unpack_max(const unsigned long long* maxkey, int64_t n, float* maxP, int32_t* argmax,
                              cudaStream_t st) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((n + threads - 1) / threads);
    unpack_max_kernel<<<blocks, threads, 0, st>>>(maxkey, n, maxP, argmax);
    return cudaGetLastError();
}

}  // namespace lsp
