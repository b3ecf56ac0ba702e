// batch_k_mrhs_x2.cu -- multi-realization batch kernels, three-term recurrence
// in packed FP32x2 (the (cos, sin) pair in the two lanes), with and without
// the window sums.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

template <bool WIN>
MrhsFn pick_recur3x2(int F, int R) {
    using namespace dev;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3x2, kTile, WIN>;
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3x2, kTile, WIN>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur3x2, kTile, WIN>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur3x2, kTile, WIN>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur3x2, kTile, WIN>;
    if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur3x2, kTile, WIN>;
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_recur3x2(int F, int R, int tile, bool win) {
    if (tile != kTile) return nullptr;
    return win ? pick_recur3x2<true>(F, R) : pick_recur3x2<false>(F, R);
}

}  // namespace lsp
