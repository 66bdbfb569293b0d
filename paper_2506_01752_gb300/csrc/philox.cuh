// philox.cuh -- counter-based random words for the device kernels.
//
// Philox4x32 with 10 rounds, written from the definition in Salmon, Moraes,
// Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): each
// round multiplies counter words 0 and 2 by the two round multipliers, mixes
// the high halves with counter words 1 and 3 and the key, and the key is
// bumped by the two Weyl constants between rounds.
//
// Stream layout used by every kernel (key = seed):
//   per individual i and node v:  counter (v, i / 4, g, stage), word i % 4
//   per child i (selection):      counter (w / 4, i, g, kStageSelect), word w % 4
#pragma once

#include <stdint.h>

namespace mocd {

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1)
{
    const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kMul0, ctr.x), lo0 = kMul0 * ctr.x;
        const uint32_t hi1 = __umulhi(kMul1, ctr.z), lo1 = kMul1 * ctr.z;
        ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return ctr;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &r, int k)
{
    return k == 0 ? r.x : k == 1 ? r.y : k == 2 ? r.z : r.w;
}

// Integer pick in [0, k): floor(u * k / 2^32).
__device__ __forceinline__ uint32_t pick_index(uint32_t u, uint32_t k)
{
    return __umulhi(u, k);
}

}  // namespace mocd
