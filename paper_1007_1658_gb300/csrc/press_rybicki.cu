// press_rybicki.cu -- the fast approximate periodogram of Press & Rybicki
// (1989), the O(N log N) alternative the paper's introduction cites: the data
// are "extirpolated" onto a uniform periodic grid and one FFT gives the sums
// of Eq. 5-8 at every grid frequency.
//
// Grid: n_fft nodes (a power of two) spanning one period 1/df, so FFT bin K
// is the frequency K df.  Sample j sits at g = frac(t'_j df) n_fft for the
// sums over x and at g2 = frac(2 t'_j df) n_fft for the sums over the doubled
// angle; each is spread onto the macc nodes around it with the Lagrange
// weights that would interpolate a function from those nodes to g.  The two
// real grids travel as one complex array z = grid_x + i grid_1; one FFT with
// the e^{+2 pi i K m / n} sign gives Z, and the transforms of the two real
// grids are (Z[K] + conj Z[n-K]) / 2 and (Z[K] - conj Z[n-K]) / 2i.  With
// XC + i XS = sum x e^{i w t'} and CC - SS + 2i CS = sum e^{2 i w t'}, Eq. 5-6
// follow in the closed form of periodogram_value.
//
// Kernels: spread (FP64 positions, FP32 Lagrange weights, FP64 atomics into a
// double2 grid), Stockham passes of radix 16 (radix 2 and/or 4 first for the
// remainder of log2 n_fft modulo 4; the first pass reads the FP64 grid and
// rounds it to FP32), and a finalize pass over the requested bins.
#include "ls_device.cuh"

namespace lsp {
namespace {

constexpr int kPrThreads = 256;

constexpr int kMaxMacc = 16;

// Lagrange weights of the macc nodes lo .. lo+macc-1 for a position d = g - lo
// in [macc/2 - 1, macc/2): w_i = prod_{l != i} (d - l) / prod_{l != i} (i - l),
// numerators from prefix and suffix products, denominators 1 / (i! (macc-1-i)!)
// with the sign (-1)^(macc-1-i).  FP32 (d is small; the FFT is FP32 too).
__device__ __forceinline__ void lagrange_weights(float d, int macc, float* w) {
    float pre = 1.f;
    for (int i = 0; i < macc; ++i) {
        w[i] = pre;
        pre *= d - (float)i;
    }
    float suf = 1.f;
    for (int i = macc - 1; i >= 0; --i) {
        float den = 1.f;
        for (int l = 0; l < macc; ++l)
            if (l != i) den *= (float)(i - l);
        w[i] *= suf / den;
        suf *= d - (float)i;
    }
}

__global__ void __launch_bounds__(kPrThreads)
pr_spread_kernel(const double* __restrict__ t, const double* __restrict__ X, int64_t n,
                 const CurveStats* __restrict__ stats, double df, int64_t n_fft, int macc,
                 double2* __restrict__ acc) {
    const CurveStats st = stats[0];
    const double nd = (double)n_fft;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double tt = t[j] - st.t_ref;
        const double x = (X[j] - st.mean) * st.inv_sd;
#pragma unroll 1
        for (int which = 0; which < 2; ++which) {
            // position in FP64 (node choice exact), offset from the first node in FP32
            const double p = (which ? 2.0 * tt : tt) * df;
            const double g = (p - floor(p)) * nd;
            const int64_t lo = (int64_t)floor(g) - (macc / 2 - 1);
            float w[kMaxMacc];
            lagrange_weights((float)(g - (double)lo), macc, w);
            for (int i = 0; i < macc; ++i) {
                const int64_t m = (lo + i) & (n_fft - 1);  // periodic grid, n_fft a power of two
                if (which == 0)
                    atomicAdd(&acc[m].x, (double)w[i] * x);
                else
                    atomicAdd(&acc[m].y, (double)w[i]);
            }
        }
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// e^{+2 pi i f / den} for integer f, den a power of two (f reduced exactly
// to [-den/2, den/2) first, so the FP32 argument of sincospif is small).
__device__ __forceinline__ float2 twiddle(int64_t f, int64_t den) {
    f &= den - 1;
    if (f >= den / 2) f -= den;
    float s, c;
    sincospif(2.0f * (float)f / (float)den, &s, &c);
    return make_float2(c, s);
}

template <class T>
__device__ __forceinline__ float2 load_c(const T* p, int64_t i);
template <>
__device__ __forceinline__ float2 load_c<float2>(const float2* p, int64_t i) {
    return p[i];
}
template <>
__device__ __forceinline__ float2 load_c<double2>(const double2* p, int64_t i) {
    const double2 v = p[i];
    return make_float2((float)v.x, (float)v.y);
}

// One radix-2 Stockham pass with Ns = 1 (only used first, when log2 n is odd).
template <class T>
__global__ void __launch_bounds__(kPrThreads)
fft_radix2_first(const T* __restrict__ in, float2* __restrict__ out, int64_t n) {
    const int64_t h = n >> 1;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < h; j += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = load_c(in, j), b = load_c(in, j + h);
        out[2 * j] = make_float2(a.x + b.x, a.y + b.y);
        out[2 * j + 1] = make_float2(a.x - b.x, a.y - b.y);
    }
}

// One radix-4 Stockham pass: sub-transforms of length Ns become length 4 Ns.
// Element j (of n/4) takes in[j + q n/4], q = 0..3, twiddles them by
// e^{+2 pi i r q / (4 Ns)} with r = j mod Ns, applies the 4-point DFT
// (e^{+2 pi i / 4} = i) and writes out[(j - r) 4 + r + q Ns].
template <class T>
__global__ void __launch_bounds__(kPrThreads)
fft_radix4_pass(const T* __restrict__ in, float2* __restrict__ out, int64_t n, int64_t Ns) {
    const int64_t quarter = n >> 2;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < quarter;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = j & (Ns - 1);
        float2 v0 = load_c(in, j), v1 = load_c(in, j + quarter), v2 = load_c(in, j + 2 * quarter),
               v3 = load_c(in, j + 3 * quarter);
        if (Ns > 1) {
            v1 = cmul(v1, twiddle(r, 4 * Ns));
            v2 = cmul(v2, twiddle(2 * r, 4 * Ns));
            v3 = cmul(v3, twiddle(3 * r, 4 * Ns));
        }
        const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y);
        const float2 a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
        const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y);
        const float2 a3 = make_float2(-(v1.y - v3.y), v1.x - v3.x);  // i (v1 - v3)
        const int64_t d = ((j - r) << 2) + r;
        out[d] = make_float2(a0.x + a2.x, a0.y + a2.y);
        out[d + Ns] = make_float2(a1.x + a3.x, a1.y + a3.y);
        out[d + 2 * Ns] = make_float2(a0.x - a2.x, a0.y - a2.y);
        out[d + 3 * Ns] = make_float2(a1.x - a3.x, a1.y - a3.y);
    }
}

// In-place 4-point DFT with the e^{+2 pi i / 4} = i kernel.
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    const float2 a0 = make_float2(x0.x + x2.x, x0.y + x2.y);
    const float2 a1 = make_float2(x0.x - x2.x, x0.y - x2.y);
    const float2 a2 = make_float2(x1.x + x3.x, x1.y + x3.y);
    const float2 a3 = make_float2(-(x1.y - x3.y), x1.x - x3.x);
    x0 = make_float2(a0.x + a2.x, a0.y + a2.y);
    x1 = make_float2(a1.x + a3.x, a1.y + a3.y);
    x2 = make_float2(a0.x - a2.x, a0.y - a2.y);
    x3 = make_float2(a1.x - a3.x, a1.y - a3.y);
}

// One radix-16 Stockham pass (sub-transforms of length Ns become 16 Ns).  The
// 16-point DFT runs as 4 x 4: with q = 4a + b and k = c + 4d,
// X[c + 4d] = sum_b i^{bd} w^{bc} sum_a v[4a + b] i^{ac}, w = e^{+2 pi i / 16}.
template <class T>
__global__ void __launch_bounds__(kPrThreads)
fft_radix16_pass(const T* __restrict__ in, float2* __restrict__ out, int64_t n, int64_t Ns) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
    const int64_t m = n >> 4;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = j & (Ns - 1);
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = load_c(in, j + q * m);
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < 16; ++q) v[q] = cmul(v[q], twiddle(q * r, 16 * Ns));
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) dft4(v[b], v[4 + b], v[8 + b], v[12 + b]);  // v[4c + b] = Y_b[c]
        // inner twiddles w^{bc}
        v[5] = cmul(v[5], make_float2(c1, s1));    // b = 1, c = 1
        v[6] = cmul(v[6], make_float2(h, h));      // b = 2, c = 1
        v[7] = cmul(v[7], make_float2(s1, c1));    // b = 3, c = 1
        v[9] = cmul(v[9], make_float2(h, h));      // b = 1, c = 2
        v[10] = make_float2(-v[10].y, v[10].x);    // b = 2, c = 2: w^4 = i
        v[11] = cmul(v[11], make_float2(-h, h));   // b = 3, c = 2
        v[13] = cmul(v[13], make_float2(s1, c1));  // b = 1, c = 3
        v[14] = cmul(v[14], make_float2(-h, h));   // b = 2, c = 3
        v[15] = cmul(v[15], make_float2(-c1, -s1));  // b = 3, c = 3: w^9
#pragma unroll
        for (int c = 0; c < 4; ++c) dft4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);  // v[4c + d] = X[c + 4d]
        const int64_t d0 = ((j - r) << 4) + r;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int d = 0; d < 4; ++d) out[d0 + (c + 4 * d) * Ns] = v[4 * c + d];
    }
}

__global__ void __launch_bounds__(kPrThreads)
pr_finalize_kernel(const float2* __restrict__ Z, int64_t n_fft, int64_t j0, int64_t N_f, float n,
                   float* __restrict__ P_out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N_f; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t K = j0 + k;
        const float2 a = Z[K & (n_fft - 1)];
        const float2 b = Z[(n_fft - K) & (n_fft - 1)];
        // transform of the x grid: (a + conj b) / 2; of the unit grid: (a - conj b) / 2i
        const float XC = 0.5f * (a.x + b.x), XS = 0.5f * (a.y - b.y);
        const float A2 = 0.5f * (a.y + b.y), B2 = -0.5f * (a.x - b.x);
        P_out[k] = dev::periodogram_value(XC, XS, 0.5f * (n + A2), 0.5f * B2, n);
    }
}

unsigned blocks_for(int64_t work) {
    int64_t b = (work + kPrThreads - 1) / kPrThreads;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int64_t pr_fft_size(int64_t k_hi, int macc) {
    const int64_t need = 2 * (int64_t)macc * (k_hi + 1);
    int64_t n = 1;
    while (n < need) n <<= 1;
    return n;
}

cudaError_t launch_pr(const double* t, const double* X, int64_t N, const CurveStats* stats, double df, int64_t j0,
                      int64_t N_f, int macc, int64_t n_fft, double2* acc, float2* z0, float2* z1, float* P_out,
                      int* launches, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)n_fft * sizeof(double2), st);
    if (e != cudaSuccess) return e;
    pr_spread_kernel<<<blocks_for(N), kPrThreads, 0, st>>>(t, X, N, stats, df, n_fft, macc, acc);
    int nl = 1;
    int L = 0;
    while ((int64_t(1) << L) < n_fft) ++L;
    // radix 2 and/or 4 first for the remainder of log2 n_fft modulo 4, then
    // radix 16; the first pass reads the FP64 grid
    float2* cur = z0;
    float2* nxt = z1;
    int64_t Ns = 1;
    const int rem = L & 3;
    bool first = true;
    auto flip = [&]() {
        if (!first) {
            float2* tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        first = false;
        ++nl;
    };
    if (rem == 1 || rem == 3) {
        fft_radix2_first<double2><<<blocks_for(n_fft / 2), kPrThreads, 0, st>>>(acc, cur, n_fft);
        Ns = 2;
        flip();
    }
    if (rem >= 2) {
        if (first)
            fft_radix4_pass<double2><<<blocks_for(n_fft / 4), kPrThreads, 0, st>>>(acc, cur, n_fft, Ns);
        else
            fft_radix4_pass<float2><<<blocks_for(n_fft / 4), kPrThreads, 0, st>>>(cur, nxt, n_fft, Ns);
        Ns *= 4;
        flip();
    }
    for (; Ns < n_fft; Ns <<= 4) {
        if (first)
            fft_radix16_pass<double2><<<blocks_for(n_fft / 16), kPrThreads, 0, st>>>(acc, cur, n_fft, Ns);
        else
            fft_radix16_pass<float2><<<blocks_for(n_fft / 16), kPrThreads, 0, st>>>(cur, nxt, n_fft, Ns);
        flip();
    }
    pr_finalize_kernel<<<blocks_for(N_f), kPrThreads, 0, st>>>(cur, n_fft, j0, N_f, (float)N, P_out);
    ++nl;
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace lsp
