// batch_k_mufu.cu -- single-realization batch kernels, hardware sin/cos.
#include "batch_kernels.cuh"

namespace lsp {

BatchFn batch_fn_mufu(int F, bool xrec) {
    using namespace dev;
    switch (F) {
        case 4: return xrec ? (BatchFn)ls_batch_kernel<4, kMufu, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<4, kMufu, false, 0, kTile>;
        case 8: return xrec ? (BatchFn)ls_batch_kernel<8, kMufu, true, 0, kTile>
                         : (BatchFn)ls_batch_kernel<8, kMufu, false, 0, kTile>;
        case 12: return xrec ? (BatchFn)ls_batch_kernel<12, kMufu, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<12, kMufu, false, 8, kTile>;
        case 16: return xrec ? (BatchFn)ls_batch_kernel<16, kMufu, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<16, kMufu, false, 8, kTile>;
        case 24: return xrec ? (BatchFn)ls_batch_kernel<24, kMufu, true, 8, kTile>
                         : (BatchFn)ls_batch_kernel<24, kMufu, false, 8, kTile>;
        default: return nullptr;
    }
}

}  // namespace lsp
