// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), written from its
// published definition.  One round maps (X0, X1, X2, X3) under key (K0, K1) to
//   (hi(M1 X2) ^ X1 ^ K0,  lo(M1 X2),  hi(M0 X0) ^ X3 ^ K1,  lo(M0 X0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
// (0x9E3779B9, 0xBB67AE85) after every round; ten rounds in all.
#pragma once

#include <stdint.h>

namespace esim {

// The ten round keys of one seed, computed once on the host and passed as a
// kernel parameter, so each round reads its key from the constant bank instead
// of holding twenty key registers per thread.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        K.k0[i] = k0;
        K.k1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const PhiloxKeys& K) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * x.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * x.z;
        x = make_uint4((uint32_t)(p1 >> 32) ^ x.y ^ K.k0[i], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ x.w ^ K.k1[i],
                       (uint32_t)p0);
    }
    return x;
}

}  // namespace esim
