// batch_k_mrhs_other.cu -- multi-realization batch kernels, hardware sin/cos and angle-addition recurrence.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

template <int MODE, bool WIN>
MrhsFn pick_other(int F, int R) {
    using namespace dev;
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, MODE, kTile, WIN>;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, MODE, kTile, WIN>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, MODE, kTile, WIN>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, MODE, kTile, WIN>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, MODE, kTile, WIN>;
    if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, MODE, kTile, WIN>;
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_other(int mode, int F, int R, bool win) {
    using namespace dev;
    if (mode == kMufu) return win ? pick_other<kMufu, true>(F, R) : pick_other<kMufu, false>(F, R);
    if (mode == kRecur) return win ? pick_other<kRecur, true>(F, R) : pick_other<kRecur, false>(F, R);
    return nullptr;
}

}  // namespace lsp
