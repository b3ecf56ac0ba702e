// batch_k_recur3_tuned.cu -- tuning variants of the three-term-recurrence batch kernel.
#include "batch_kernels.cuh"

namespace lsp {

// Shapes that lsp_autotune_batch may pick for single-realization batches
// with x in the records: strips of 16 or 24, tail strips of 0, 4 or 8, tiles
// of 128, 256 or 512 samples (the default pair, tail 8 and tiles of kTile =
// 128, is in batch_k_recur3.cu).
BatchFn batch_fn_recur3_tuned(int F, int tailF, int tile) {
    using namespace dev;
    if (F == 16 && tailF == 0 && tile == 128) return ls_batch_kernel<16, kRecur3, true, 0, 128>;
    if (F == 16 && tailF == 0 && tile == 256) return ls_batch_kernel<16, kRecur3, true, 0, 256>;
    if (F == 16 && tailF == 0 && tile == 512) return ls_batch_kernel<16, kRecur3, true, 0, 512>;
    if (F == 16 && tailF == 4 && tile == 128) return ls_batch_kernel<16, kRecur3, true, 4, 128>;
    if (F == 16 && tailF == 4 && tile == 256) return ls_batch_kernel<16, kRecur3, true, 4, 256>;
    if (F == 16 && tailF == 4 && tile == 512) return ls_batch_kernel<16, kRecur3, true, 4, 512>;
    if (F == 16 && tailF == 8 && tile == 256) return ls_batch_kernel<16, kRecur3, true, 8, 256>;
    if (F == 16 && tailF == 8 && tile == 512) return ls_batch_kernel<16, kRecur3, true, 8, 512>;
    if (F == 24 && tailF == 0 && tile == 128) return ls_batch_kernel<24, kRecur3, true, 0, 128>;
    if (F == 24 && tailF == 0 && tile == 256) return ls_batch_kernel<24, kRecur3, true, 0, 256>;
    if (F == 24 && tailF == 0 && tile == 512) return ls_batch_kernel<24, kRecur3, true, 0, 512>;
    if (F == 24 && tailF == 4 && tile == 128) return ls_batch_kernel<24, kRecur3, true, 4, 128>;
    if (F == 24 && tailF == 4 && tile == 256) return ls_batch_kernel<24, kRecur3, true, 4, 256>;
    if (F == 24 && tailF == 4 && tile == 512) return ls_batch_kernel<24, kRecur3, true, 4, 512>;
    if (F == 24 && tailF == 8 && tile == 256) return ls_batch_kernel<24, kRecur3, true, 8, 256>;
    if (F == 24 && tailF == 8 && tile == 512) return ls_batch_kernel<24, kRecur3, true, 8, 512>;
    return nullptr;
}

}  // namespace lsp
