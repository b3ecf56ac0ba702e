/*
 * lsp_testing.h -- hooks that the library's own tests use to reach error
 * paths without a failing GPU.  Nothing here is needed in normal use, and
 * nothing here computes any part of the periodogram (the paper has no
 * counterpart: these exist for failure detection, as a test harness's fault
 * injection on the host).
 */
#ifndef LSP_TESTING_H
#define LSP_TESTING_H

#include <stdint.h>

#include "lsp.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * The library's decision on where a caller's array lives, from the two
 * fields of its CUDA pointer attributes that decide it: memory_type (the
 * cudaMemoryType value: 0 unregistered host, 1 host, 2 device, 3 managed) and
 * pointer_device (the device that owns the memory), against `device` (the
 * context's device, or the current device for lsp_periodogram_noalloc).
 * Returns 0 for host memory (the library stages it through copies), 1 for
 * memory used in place (device memory of `device`, or managed memory), and
 * 2 for device memory of another GPU, which every entry point refuses with
 * LSP_ERR_INVALID_ARG.  Host arithmetic only; needs no GPU.
 */
int32_t lsp_test_pointer_kind(int32_t memory_type, int32_t pointer_device, int32_t device);

/*
 * Make the n-th workspace allocation of `ctx` from now fail as if cudaMalloc
 * had run out of memory (n = 0 cancels).  The failing call returns
 * LSP_ERR_OOM and leaves the context usable: a later call allocates again.
 * Errors: INVALID_ARG (null context, n < 0).
 */
lsp_status lsp_test_fail_allocation(lsp_ctx *ctx, int32_t n);

/*
 * Launch shape of the context's last lsp_batch plan: shape[0..4] = kernel
 * mode (1 hardware sin/cos, 2 angle-addition recurrence, 4 three-term
 * recurrence, 5 its packed form), strip length F, realizations per pass R,
 * tail-strip length (0: none) and samples per shared-memory tile.
 * Errors: INVALID_ARG (null arguments, or no batch planned yet).
 */
lsp_status lsp_test_last_batch_shape(const lsp_ctx *ctx, int32_t shape[5]);

#ifdef __cplusplus
}
#endif

#endif /* LSP_TESTING_H */
