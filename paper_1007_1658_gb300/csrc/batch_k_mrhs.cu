// batch_k_mrhs.cu -- multi-realization batch kernels, three-term recurrence.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

template <bool WIN>
MrhsFn pick_recur3(int F, int R, int tile) {
    using namespace dev;
    if (tile == kTile) {
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, kTile, WIN>;
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, kTile, WIN>;
        if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur3, kTile, WIN>;
        if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur3, kTile, WIN>;
        if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur3, kTile, WIN>;
        if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur3, kTile, WIN>;
        return nullptr;
    }
    if (tile == 256) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 256, WIN>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 256, WIN>;
    }
    if (tile == 512) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 512, WIN>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 512, WIN>;
    }
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_recur3(int F, int R, int tile, bool win) {
    return win ? pick_recur3<true>(F, R, tile) : pick_recur3<false>(F, R, tile);
}

}  // namespace lsp
