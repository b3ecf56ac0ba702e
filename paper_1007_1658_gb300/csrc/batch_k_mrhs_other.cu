// batch_k_mrhs_other.cu -- multi-realization batch kernels, hardware sin/cos and angle-addition recurrence.
#include "batch_kernels.cuh"

namespace lsp {

BatchFn mrhs_fn_other(int mode, int F, int R) {
    using namespace dev;
    if (mode == kMufu) {
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kMufu, kTile>;
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kMufu, kTile>;
        if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kMufu, kTile>;
        if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kMufu, kTile>;
        if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kMufu, kTile>;
    }
    if (mode == kRecur) {
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur, kTile>;
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur, kTile>;
        if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur, kTile>;
        if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur, kTile>;
        if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur, kTile>;
    }
    return nullptr;
}

}  // namespace lsp
