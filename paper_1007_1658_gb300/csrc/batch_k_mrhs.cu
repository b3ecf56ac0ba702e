// batch_k_mrhs.cu -- multi-realization batch kernels, scalar three-term
// recurrence, groups that keep their own CC and CS (the window-sum forms are
// in batch_k_mrhs_win.cu: two translation units so that the library compiles
// in parallel).
#include "batch_kernels.cuh"

namespace lsp {

MrhsFn mrhs_fn_recur3_win(int F, int R, int tile);

namespace {

MrhsFn pick_recur3_own(int F, int R, int tile) {
    using namespace dev;
    if (tile == kTile) {
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, kTile, false>;
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, kTile, false>;
        if (F == 8 && R == 2) return ls_mrhs_kernel<8, 2, kRecur3, kTile, false>;
        if (F == 16 && R == 2) return ls_mrhs_kernel<16, 2, kRecur3, kTile, false>;
        if (F == 4 && R == 8) return ls_mrhs_kernel<4, 8, kRecur3, kTile, false>;
        if (F == 8 && R == 8) return ls_mrhs_kernel<8, 8, kRecur3, kTile, false>;
        return nullptr;
    }
    if (tile == 256) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 256, false>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 256, false>;
    }
    if (tile == 512) {
        if (F == 12 && R == 4) return ls_mrhs_kernel<12, 4, kRecur3, 512, false>;
        if (F == 8 && R == 4) return ls_mrhs_kernel<8, 4, kRecur3, 512, false>;
    }
    return nullptr;
}

}  // namespace

MrhsFn mrhs_fn_recur3(int F, int R, int tile, bool win) {
    return win ? mrhs_fn_recur3_win(F, R, tile) : pick_recur3_own(F, R, tile);
}

}  // namespace lsp
