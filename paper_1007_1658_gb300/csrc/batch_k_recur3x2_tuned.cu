// batch_k_recur3x2_tuned.cu -- tuning variants of the packed three-term-recurrence batch kernel.
#include "batch_kernels.cuh"

namespace lsp {

// The tuned shapes of batch_fn_tuned (batch_kernels.cuh); the default pair,
// tail 8 and tiles of kTile = 128, is in batch_k_recur3x2.cu.
BatchFn batch_fn_recur3x2_tuned(int F, int tailF, int tile) { return batch_fn_tuned<dev::kRecur3x2>(F, tailF, tile); }

}  // namespace lsp
