// batch_k_mrhs_win.cu -- multi-realization batch kernels, scalar three-term
// recurrence, groups that read CC and CS from the window pass.
#include "batch_kernels.cuh"

namespace lsp {

MrhsFn mrhs_fn_recur3_win(int F, int R, int tile) {
    using namespace dev;
    if (tile == kTile) {
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, kTile, true>;
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, kTile, true>;
        if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur3, kTile, true>;
        if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur3, kTile, true>;
        if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur3, kTile, true>;
        if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur3, kTile, true>;
        return nullptr;
    }
    if (tile == 256) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 256, true>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 256, true>;
    }
    if (tile == 512) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 512, true>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 512, true>;
    }
    return nullptr;
}

}  // namespace lsp
