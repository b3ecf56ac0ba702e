// batch_k_mrhs_rot.cu -- multi-realization batch kernels, angle-addition recurrence.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

template <bool WIN>
MrhsFn pick_rot(int F, int R) {
    using namespace dev;
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur, kTile, WIN>;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur, kTile, WIN>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur, kTile, WIN>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur, kTile, WIN>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur, kTile, WIN>;
    if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur, kTile, WIN>;
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_rot(int F, int R, bool win) { return win ? pick_rot<true>(F, R) : pick_rot<false>(F, R); }

}  // namespace lsp
