// batch_k_recur3_tuned.cu -- tuning variants of the scalar three-term-recurrence batch kernel.
#include "batch_kernels.cuh"

namespace lsp {

// The tuned shapes of batch_fn_tuned (batch_kernels.cuh); the default pair,
// tail 8 and tiles of kTile = 128, is in batch_k_recur3.cu.
BatchFn batch_fn_recur3_tuned(int F, int tailF, int tile) { return batch_fn_tuned<dev::kRecur3>(F, tailF, tile); }

}  // namespace lsp
