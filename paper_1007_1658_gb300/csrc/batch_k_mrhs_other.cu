// batch_k_mrhs_other.cu -- multi-realization batch kernels, hardware sin/cos
// (the angle-addition recurrence's are in batch_k_mrhs_rot.cu).
#include "batch_kernels.cuh"

namespace lsp {

MrhsFn mrhs_fn_rot(int F, int R, bool win);

namespace {

template <bool WIN>
MrhsFn pick_mufu(int F, int R) {
    using namespace dev;
    if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kMufu, kTile, WIN>;
    if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kMufu, kTile, WIN>;
    if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kMufu, kTile, WIN>;
    if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kMufu, kTile, WIN>;
    if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kMufu, kTile, WIN>;
    if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kMufu, kTile, WIN>;
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_other(int mode, int F, int R, bool win) {
    using namespace dev;
    if (mode == kMufu) return win ? pick_mufu<true>(F, R) : pick_mufu<false>(F, R);
    if (mode == kRecur) return mrhs_fn_rot(F, R, win);
    return nullptr;
}

}  // namespace lsp
