// batch.cu -- launchers of the persistent batch kernels (batch_kernels.cuh,
// instantiated in batch_k_*.cu) and the unpacking of the per-curve maxima.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

// maxkey -> (max P, argmax k); a curve with no frequency gets (0, -1).
__global__ void unpack_max_kernel(const unsigned long long* __restrict__ maxkey, int64_t n, float* __restrict__ maxP,
                                  int32_t* __restrict__ argmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long key = maxkey[i];
    if (maxP) maxP[i] = key ? __uint_as_float((uint32_t)(key >> 32)) : 0.f;
    if (argmax) argmax[i] = key ? (int32_t)(~(uint32_t)key) : -1;
}

BatchFn batch_fn(int mode, int F, bool xrec, int tailF, int tile) {
    switch (mode) {
        case kModeMufu: return tailF == (F > kBatchTailF ? kBatchTailF : 0) && tile == kTile ? batch_fn_mufu(F, xrec) : nullptr;
        case kModeRecur: return tailF == (F > kBatchTailF ? kBatchTailF : 0) && tile == kTile ? batch_fn_recur(F, xrec) : nullptr;
        case kModeRecur3: return batch_fn_recur3(F, xrec, tailF, tile);
        case kModeRecur3x2: return batch_fn_recur3x2(F, xrec, tailF, tile);
        default: return nullptr;
    }
}

MrhsFn mrhs_fn(int mode, int F, int R, int tile, bool win) {
    switch (mode) {
        case kModeRecur3: return mrhs_fn_recur3(F, R, tile, win);
        case kModeRecur3x2: return mrhs_fn_recur3x2(F, R, tile, win);
        case kModeMufu:
        case kModeRecur: return tile == kTile ? mrhs_fn_other(mode, F, R, win) : nullptr;
        default: return nullptr;
    }
}

template <class Fn>
int occupancy_of(Fn fn) {
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)fn, kMainThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace

int batch_default_tail(int F) { return F > kBatchTailF ? kBatchTailF : 0; }

int mrhs_occupancy(int mode, int F, int R, int tile, bool win) {
    return occupancy_of(mrhs_fn(mode, F, R, tile, win));
}

cudaError_t launch_mrhs(int mode, int F, int R, int tile, int grid, const BatchItem* items, int n_items,
                        unsigned* head, const int64_t* off, const int64_t* nf, int64_t total, int n_curves,
                        const uint4* recA, const float4* recB, const float* xr, float* P_out, const int64_t* P_off,
                        int64_t P_total, unsigned long long* maxkey, const float2* win, const int64_t* woff,
                        cudaStream_t st) {
    MrhsFn fn = mrhs_fn(mode, F, R, tile, win != nullptr);
    if (!fn || (win && !woff)) return cudaErrorInvalidValue;
    fn<<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nf, total, n_curves, recA, recB, xr, P_out, P_off,
                                      P_total, maxkey, win, woff);
    return cudaGetLastError();
}

int window_occupancy(int mode, int F) { return occupancy_of(window_fn(mode, F)); }

cudaError_t launch_window(int mode, int F, int grid, const BatchItem* items, int n_items, unsigned* head,
                          const int64_t* off, const int64_t* nf, const int64_t* woff, const uint4* recA,
                          const float4* recB, float2* win, cudaStream_t st) {
    WindowFn fn = window_fn(mode, F);
    if (!fn) return cudaErrorInvalidValue;
    fn<<<grid, kMainThreads, 0, st>>>(items, n_items, head, off, nf, woff, recA, recB, win);
    return cudaGetLastError();
}

int batch_occupancy(int mode, int F, bool x_in_records, int tailF, int tile) {
    return occupancy_of(batch_fn(mode, F, x_in_records, tailF, tile));
}

cudaError_t launch_batch(int mode, int F, bool x_in_records, int tailF, int tile, int grid, const BatchItem* items,
                         int n_items, unsigned* head, const int64_t* off, const int64_t* nf, int64_t total,
                         int n_curves, const uint4* recA, const float4* recB, const float* xr, float* P_out,
                         const int64_t* P_off, int64_t P_total, unsigned long long* maxkey, cudaStream_t st) {
    BatchFn fn = batch_fn(mode, F, x_in_records, tailF, tile);
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
