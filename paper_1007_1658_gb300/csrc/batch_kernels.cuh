// batch_kernels.cuh -- the persistent kernels of lsp_batch as templates.
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
// The templates are instantiated in several translation units (by sin/cos
// mode and shape), each exporting a lookup from the runtime shape to its
// kernels, so that the library compiles in parallel.
#pragma once

#include "ls_device.cuh"

namespace lsp {

using BatchFn = void (*)(const BatchItem*, int, unsigned*, const int64_t*, const int64_t*, int64_t, int,
                         const uint4*, const float4*, const float*, float*, const int64_t*, int64_t,
                         unsigned long long*);

// Kernel of a single-realization shape (nullptr when it is not built):
// defaults (tail strips of 8 for F > 8, tiles of kTile) for every mode and
// strip length, and for the three-term recurrence (scalar and packed) at
// F = 16 and 24 with x in the records also tail strips of 0, 4, 8 and tiles
// of 128, 256, 512.
BatchFn batch_fn_mufu(int F, bool xrec);
BatchFn batch_fn_recur(int F, bool xrec);
BatchFn batch_fn_recur3(int F, bool xrec, int tailF, int tile);
BatchFn batch_fn_recur3x2(int F, bool xrec, int tailF, int tile);
// Multi-realization kernels take two more arguments: the window sums (CC, CS)
// of every frequency of every curve, curve c's at win[woff[c] + k], which the
// kernels built with win = true read instead of accumulating (the others
// ignore both).
using MrhsFn = void (*)(const BatchItem*, int, unsigned*, const int64_t*, const int64_t*, int64_t, int,
                        const uint4*, const float4*, const float*, float*, const int64_t*, int64_t,
                        unsigned long long*, const float2*, const int64_t*);
// Multi-realization shapes (F, R) in {(8, 4), (12, 4), (8, 2), (16, 2), (4, 8), (8, 8)},
// tiles of kTile; the three-term recurrence at (12, 4) and (8, 4) also with
// tiles of 256 and 512; each with and without the window sums from WStrip.
MrhsFn mrhs_fn_recur3(int F, int R, int tile, bool win);
MrhsFn mrhs_fn_other(int mode, int F, int R, bool win);
// The same with the three-term recurrence in packed FP32x2 (MStrip<F, R,
// kRecur3x2, !win>), for the (F, R) shapes of the scalar kernels and tiles of
// kTile.
MrhsFn mrhs_fn_recur3x2(int F, int R, int tile, bool win);
// The window pass (ls_window_kernel) for the strip lengths above.
using WindowFn = void (*)(const BatchItem*, int, unsigned*, const int64_t*, const int64_t*, const int64_t*,
                          const uint4*, const float4*, float2*);
WindowFn window_fn(int mode, int F);

namespace {

using namespace dev;

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// The double-buffered cp.async tile loop of for_each_tile for a realization
// whose x is not the one the records carry: each sample's second record is
// staged as {x[j], cos 2 pi u, sin 2 pi u, 2 cos 2 pi u}, x taken from the
// realization's row, so the strip reads it exactly as it reads the records'
// own x.  Reading x with a load of its own instead measured 0.63 against 0.81
// of the FMA roof (ncu: dispatch stalls 1.33 against 0.19 per issue).
template <int TILE, class Body>
__device__ __forceinline__ void for_each_tile_xb(TileSmem<false, TILE>& sm, const uint4* __restrict__ recA,
                                                 const float4* __restrict__ recB, const float* __restrict__ x,
                                                 int64_t j0, int64_t j1, Body&& body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + TILE - 1) / TILE) : 0;
    auto stage = [&](int buf, int64_t jt) {
        const int n = (int)min((int64_t)TILE, j1 - jt);
        for (int q = tid; q < n; q += nt) {
            cp_async16(&sm.A[buf][q], recA + jt + q);
            float* dst = reinterpret_cast<float*>(&sm.B[buf][q]);
            const float* src = reinterpret_cast<const float*>(recB + jt + q);
            cp_async4(dst, x + jt + q);
            cp_async4(dst + 1, src + 1);
            cp_async8(dst + 2, src + 2);
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
        body(sm.A[it & 1], sm.B[it & 1], (int)min((int64_t)TILE, j1 - jt));
        __syncthreads();
    }
}

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
    // a strip that lies wholly beyond the grid (the padding of the item's last
    // block) only helps stage the tiles: its warp, when all of it is padding,
    // leaves its issue slots to the other CTAs on the SM
    const bool live = k0 < (uint32_t)N_f;
    if constexpr (XREC) {
        // the single-curve kernel's loop: x from the records
        constexpr int T = sizeof(sm.A[0]) / sizeof(uint4);  // the tile length of this kernel
        for_each_tile<false>(sm, recA, recB, nullptr, b, e, [&](const uint4* a, const float4* bb, const float*, int n) {
            if (live) strip_tile<T, false>(st, a, bb, n, k0);
        });
    } else {
        // x of this realization staged into the records' x slot
        constexpr int T = sizeof(sm.A[0]) / sizeof(uint4);
        for_each_tile_xb(sm, recA, recB, x, b, e, [&](const uint4* a, const float4* bb, int n) {
            if (live) strip_tile<T, false>(st, a, bb, n, k0);
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

// TAILF: strip length of the tail items (0: none).  The frequencies of a curve
// left over after its full blocks of kMainThreads*F run in blocks of
// kMainThreads*TAILF, so at most kMainThreads*TAILF - 1 slots per curve are
// padding.  TILE: samples per shared-memory tile.
template <int F, int MODE, bool XREC, int TAILF, int TILE>
__global__ void __launch_bounds__(kMainThreads)
ls_batch_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                const int64_t* __restrict__ off, const int64_t* __restrict__ nf, int64_t total, int n_curves,
                const uint4* __restrict__ recA, const float4* __restrict__ recB, const float* __restrict__ xr,
                float* __restrict__ P_out, const int64_t* __restrict__ P_off, int64_t P_total,
                unsigned long long* __restrict__ maxkey) {
    __shared__ __align__(16) TileSmem<false, TILE> sm;
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
        unsigned long long best = 0ull;
        bool tail = false;
        if constexpr (TAILF > 0 && F > TAILF) {
            if (w.pad < 0) {
                // tail item: sub-block (-1 - pad) of kMainThreads*TAILF after fblock full blocks
                const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) +
                                    (uint32_t)(-1 - w.pad) * (kMainThreads * TAILF) + (uint32_t)threadIdx.x * TAILF;
                best = batch_item<TAILF, MODE, XREC>(sm, k0, b, e, N_f, recA, recB, x, P);
                tail = true;
            }
        }
        if (!tail) {
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

// The shapes that lsp_autotune_batch may pick for single-realization batches
// with x in the records besides the default pair (tail 8, tiles of kTile):
// strips of 16 or 24, tail strips of 0, 4 or 8, tiles of 128, 256 or 512.
template <int MODE>
BatchFn batch_fn_tuned(int F, int tailF, int tile) {
    if (F == 16 && tailF == 0 && tile == 128) return ls_batch_kernel<16, MODE, true, 0, 128>;
    if (F == 16 && tailF == 0 && tile == 256) return ls_batch_kernel<16, MODE, true, 0, 256>;
    if (F == 16 && tailF == 0 && tile == 512) return ls_batch_kernel<16, MODE, true, 0, 512>;
    if (F == 16 && tailF == 4 && tile == 128) return ls_batch_kernel<16, MODE, true, 4, 128>;
    if (F == 16 && tailF == 4 && tile == 256) return ls_batch_kernel<16, MODE, true, 4, 256>;
    if (F == 16 && tailF == 4 && tile == 512) return ls_batch_kernel<16, MODE, true, 4, 512>;
    if (F == 16 && tailF == 8 && tile == 256) return ls_batch_kernel<16, MODE, true, 8, 256>;
    if (F == 16 && tailF == 8 && tile == 512) return ls_batch_kernel<16, MODE, true, 8, 512>;
    if (F == 24 && tailF == 0 && tile == 128) return ls_batch_kernel<24, MODE, true, 0, 128>;
    if (F == 24 && tailF == 0 && tile == 256) return ls_batch_kernel<24, MODE, true, 0, 256>;
    if (F == 24 && tailF == 0 && tile == 512) return ls_batch_kernel<24, MODE, true, 0, 512>;
    if (F == 24 && tailF == 4 && tile == 128) return ls_batch_kernel<24, MODE, true, 4, 128>;
    if (F == 24 && tailF == 4 && tile == 256) return ls_batch_kernel<24, MODE, true, 4, 256>;
    if (F == 24 && tailF == 4 && tile == 512) return ls_batch_kernel<24, MODE, true, 4, 512>;
    if (F == 24 && tailF == 8 && tile == 256) return ls_batch_kernel<24, MODE, true, 8, 256>;
    if (F == 24 && tailF == 8 && tile == 512) return ls_batch_kernel<24, MODE, true, 8, 512>;
    return nullptr;
}

// Multi-RHS variant for many realizations of the same patterns: an item is
// (curve, frequency block, group of up to R realizations starting at
// w.real; w.pad = group size), and the group shares the phase, the
// recurrence and CC/CS (MStrip).  Per (frequency, realization) the result is
// the single-realization kernel's, bit for bit.
// Tile of the multi-realization kernel: the records as in TileSmemN, and the
// x values of a sample's R realizations side by side (X[buf][j][0..R-1]), so
// that R = 4 realizations come in one 128-bit load.  Measured with one-warp
// CTAs: 156.1 -> 148.2 ms for 256 patterns x 64 realizations at R = 4 (with
// four-warp CTAs the same layout had measured slower).
template <int R, int TILE>
struct TileSmemX {
    uint4 A[2][TILE];
    float4 B[2][TILE];
    float X[2][TILE][R];
};

// The double-buffered cp.async pipeline of for_each_tile_n for TileSmemX:
// realization r of sample j comes from xr[r * xstride + j]; realizations
// r >= nx_valid (the last group's missing ones) read as 0.
template <int R, int TILE, class Body>
__device__ __forceinline__ void for_each_tile_x(TileSmemX<R, TILE>& sm, const uint4* __restrict__ recA,
                                                const float4* __restrict__ recB, const float* __restrict__ xr,
                                                int64_t xstride, int nx_valid, int64_t j0, int64_t j1, Body&& body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntiles = j1 > j0 ? (int)((j1 - j0 + TILE - 1) / TILE) : 0;
    auto stage = [&](int buf, int64_t jt) {
        const int n = (int)min((int64_t)TILE, j1 - jt);
        for (int q = tid; q < n; q += nt) {
            cp_async16(&sm.A[buf][q], recA + jt + q);
            cp_async16(&sm.B[buf][q], recB + jt + q);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nx_valid)
                    cp_async4(&sm.X[buf][q][r], xr + (size_t)r * (size_t)xstride + jt + q);
                else
                    sm.X[buf][q][r] = 0.f;
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

template <int F, int R, int MODE, int TILE, bool WIN>
__global__ void __launch_bounds__(kMainThreads)
ls_mrhs_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
               const int64_t* __restrict__ off, const int64_t* __restrict__ nf, int64_t total, int n_curves,
               const uint4* __restrict__ recA, const float4* __restrict__ recB, const float* __restrict__ xr,
               float* __restrict__ P_out, const int64_t* __restrict__ P_off, int64_t P_total,
               unsigned long long* __restrict__ maxkey, const float2* __restrict__ win,
               const int64_t* __restrict__ woff) {
    __shared__ __align__(16) TileSmemX<R, TILE> sm;
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
        MStrip<F, R, MODE, !WIN> st;
        st.zero();
        const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
        for_each_tile_x<R, TILE>(sm, recA, recB, xr + (size_t)w.real * (size_t)total, total, nr, b, e,
                                 [&](const uint4* a, const float4* bb, const float (*xs)[R], int n) {
                                     if (!live) return;
                                     auto sample = [&](int j) {
                                         float x[R];
                                         if constexpr (R % 4 == 0) {  // R/4 128-bit loads
#pragma unroll
                                             for (int q = 0; q < R / 4; ++q) {
                                                 const float4 v = reinterpret_cast<const float4*>(xs[j])[q];
                                                 x[4 * q] = v.x;
                                                 x[4 * q + 1] = v.y;
                                                 x[4 * q + 2] = v.z;
                                                 x[4 * q + 3] = v.w;
                                             }
                                         } else {
#pragma unroll
                                             for (int r = 0; r < R; ++r) x[r] = xs[j][r];
                                         }
                                         st.add(a[j], bb[j], x, k0);
                                     };
                                     // unrolled twice when the window sums free the registers
                                     // for it (0.6 % at (12, 4)); with its own CC/CS the
                                     // strip has no room and measured slower unrolled
                                     if constexpr (WIN) {
#pragma unroll 2
                                         for (int j = 0; j < n; ++j) sample(j);
                                     } else {
                                         for (int j = 0; j < n; ++j) sample(j);
                                     }
                                 });
        const float n = (float)(e - b);
        const float2* wc = WIN ? win + woff[w.curve] : nullptr;  // the pattern's window sums
#pragma unroll
        for (int r = 0; r < R; ++r) {
            unsigned long long best = 0ull;
            float* P = (P_out && r < nr) ? P_out + (size_t)(w.real + r) * (size_t)P_total + P_off[w.curve] : nullptr;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                const uint32_t k = k0 + i;
                if (k < (uint32_t)N_f && r < nr) {
                    float cc_k, cs_k;
                    if constexpr (WIN) {
                        const float2 w2 = wc[k];
                        cc_k = w2.x;
                        cs_k = w2.y;
                    } else {
                        cc_k = st.get_cc(i);
                        cs_k = st.get_cs(i);
                    }
                    const float p = periodogram_value(st.get_xc(i, r), st.get_xs(i, r), cc_k, cs_k, n);
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

// Window pass: CC and CS of Eq. 8 at every frequency of every curve, win[woff[c] + k]
// = (CC, CS), by the strips of F frequencies that the multi-realization kernel of
// the same F uses (k0 a multiple of F), so its groups read the sums they would have
// accumulated, bit for bit.  Persistent over (curve, block of kMainThreads F
// frequencies) items like the batch kernels.
template <int F, int MODE>
__global__ void __launch_bounds__(kMainThreads)
ls_window_kernel(const BatchItem* __restrict__ items, int n_items, unsigned* __restrict__ head,
                 const int64_t* __restrict__ off, const int64_t* __restrict__ nf, const int64_t* __restrict__ woff,
                 const uint4* __restrict__ recA, const float4* __restrict__ recB, float2* __restrict__ win) {
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
        const int64_t N_f = nf[w.curve];
        const uint32_t k0 = (uint32_t)w.fblock * (kMainThreads * F) + (uint32_t)threadIdx.x * F;
        WStrip<F, MODE> st;
        st.zero();
        const bool live = k0 < (uint32_t)N_f;  // padding strips only help stage the tiles
        for_each_tile<false>(sm, recA, recB, nullptr, b, e,
                             [&](const uint4* a, const float4* bb, const float*, int n) {
                                 if (!live) return;
#pragma unroll 2
                                 for (int j = 0; j < n; ++j) st.add(a[j], bb[j], k0);
                             });
        float2* out = win + woff[w.curve];
#pragma unroll
        for (int i = 0; i < F; ++i)
            if (k0 + i < (uint32_t)N_f) out[k0 + i] = make_float2(st.get_cc(i), st.get_cs(i));
    }
}

}  // namespace
}  // namespace lsp
