// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), written from its
// published definition.  One round maps (X0, X1, X2, X3) under key (K0, K1) to
//   (hi(M1 X2) ^ X1 ^ K0,  lo(M1 X2),  hi(M0 X0) ^ X3 ^ K1,  lo(M0 X0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
// (0x9E3779B9, 0xBB67AE85) after every round; ten rounds in all.
#pragma once

#include <stdint.h>

namespace esim {

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, x.x);
        const uint32_t lo0 = 0xD2511F53u * x.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x.z);
        const uint32_t lo1 = 0xCD9E8D57u * x.z;
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

}  // namespace esim
