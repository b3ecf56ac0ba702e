// philox.cuh -- the Philox-4x32-10 counter-based generator (Salmon, Moraes,
// Dror & Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3"): ten
// rounds of two 32x32->64-bit multiplies and a Feistel-like swap of the four
// counter words, with the two key words bumped by Weyl constants between
// rounds.  Device code; every draw is a pure function of (counter, key).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lsp {
namespace dev {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c0, c1, c2, c3, k0, k1);
    }
    return make_uint4(c0, c1, c2, c3);
}

}  // namespace dev
}  // namespace lsp
