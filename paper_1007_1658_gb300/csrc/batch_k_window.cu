// batch_k_window.cu -- the window pass (CC, CS per frequency and curve) of the
// multi-realization batches, for each mode and multi-realization strip length.
#include "batch_kernels.cuh"

namespace lsp {
namespace {

template <int MODE>
WindowFn pick_window(int F) {
    using namespace dev;
    switch (F) {
        case 4: return ls_window_kernel<4, MODE>;
        case 8: return ls_window_kernel<8, MODE>;
        case 12: return ls_window_kernel<12, MODE>;
        case 16: return ls_window_kernel<16, MODE>;
        default: return nullptr;
    }
}

}  // namespace

WindowFn window_fn(int mode, int F) {
    using namespace dev;
    switch (mode) {
        case kMufu: return pick_window<kMufu>(F);
        case kRecur: return pick_window<kRecur>(F);
        case kRecur3: return pick_window<kRecur3>(F);
        case kRecur3x2: return pick_window<kRecur3x2>(F);  // the same sums, bit for bit
        default: return nullptr;
    }
}

}  // namespace lsp
