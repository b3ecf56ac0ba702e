// batch_k_recur3x2.cu -- single-realization batch kernels, packed three-term recurrence (the default shapes).
#include "batch_kernels.cuh"

namespace lsp {

// The tuned shapes (the other tail strips and tiles of 256 or 512) live in
// batch_k_recur3x2_tuned.cu.
BatchFn batch_fn_recur3x2_tuned(int F, int tailF, int tile);

BatchFn batch_fn_recur3x2(int F, bool xrec, int tailF, int tile) {
    using namespace dev;
    if (tailF != (F > kBatchTailF ? kBatchTailF : 0) || tile != kTile)
        return xrec ? batch_fn_recur3x2_tuned(F, tailF, tile) : nullptr;
    switch (F) {
        case 4: return xrec ? (BatchFn)ls_batch_kernel<4, kRecur3x2, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<4, kRecur3x2, false, 0, kTile>;
        case 8: return xrec ? (BatchFn)ls_batch_kernel<8, kRecur3x2, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<8, kRecur3x2, false, 0, kTile>;
        case 12: return xrec ? (BatchFn)ls_batch_kernel<12, kRecur3x2, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<12, kRecur3x2, false, 8, kTile>;
        case 16: return xrec ? (BatchFn)ls_batch_kernel<16, kRecur3x2, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<16, kRecur3x2, false, 8, kTile>;
        case 20: return xrec ? (BatchFn)ls_batch_kernel<20, kRecur3x2, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<20, kRecur3x2, false, 8, kTile>;
        case 24: return xrec ? (BatchFn)ls_batch_kernel<24, kRecur3x2, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<24, kRecur3x2, false, 8, kTile>;
        case 28: return xrec ? (BatchFn)ls_batch_kernel<28, kRecur3x2, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<28, kRecur3x2, false, 8, kTile>;
        default: return nullptr;
    }
}

}  // namespace lsp
