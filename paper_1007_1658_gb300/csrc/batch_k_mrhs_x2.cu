// batch_k_mrhs_x2.cu -- multi-realization batch kernels with the window sums,
// three-term recurrence in packed FP32x2 (the (cos, sin) pair in the two lanes).
#include "batch_kernels.cuh"

namespace lsp {

MrhsFn mrhs_fn_recur3x2(int F, int R, int tile) {
    using namespace dev;
    if (tile != kTile) return nullptr;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3x2, kTile, true>;
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3x2, kTile, true>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur3x2, kTile, true>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur3x2, kTile, true>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur3x2, kTile, true>;
    if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur3x2, kTile, true>;
    return nullptr;
}

}  // namespace lsp
