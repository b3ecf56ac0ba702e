// batch_k_recur.cu -- single-realization batch kernels, angle-addition recurrence.
#include "batch_kernels.cuh"

namespace lsp {

BatchFn batch_fn_recur(int F, bool xrec) {
    using namespace dev;
    switch (F) {
        case 4: return xrec ? (BatchFn)ls_batch_kernel<4, kRecur, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<4, kRecur, false, 0, kTile>;
        case 8: return xrec ? (BatchFn)ls_batch_kernel<8, kRecur, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<8, kRecur, false, 0, kTile>;
        case 12: return xrec ? (BatchFn)ls_batch_kernel<12, kRecur, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<12, kRecur, false, 8, kTile>;
        case 16: return xrec ? (BatchFn)ls_batch_kernel<16, kRecur, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<16, kRecur, false, 8, kTile>;
        case 20: return xrec ? (BatchFn)ls_batch_kernel<20, kRecur, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<20, kRecur, false, 8, kTile>;
        case 24: return xrec ? (BatchFn)ls_batch_kernel<24, kRecur, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<24, kRecur, false, 8, kTile>;
        case 28: return xrec ? (BatchFn)ls_batch_kernel<28, kRecur, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<28, kRecur, false, 8, kTile>;
        default: return nullptr;
    }
}

}  // namespace lsp
