// The two-step walk distribution of one node, built by one warp in a shared-memory hash
// table, and the sum of its squares (Lemma 5's l' = 2 terms).
//
// With h_1 = (P^T)(k, .) = 1/din(k) on I(k) (a graph without repeated in-edges) and
// h_2 = (P^T)^2(k, .), the table holds, in unsigned fixed point with 63 fraction bits
// (2^63 = probability 1),
//   H_2(q) = sum over q' in I(k) with q in I(q') of floor(2^63 / (din(k) din(q'))).
// These are the integers of two probe steps that divide by din with truncation, since
// floor(floor(x / a) / b) = floor(x / (a b)) for positive integers; integer atomics make
// the table exact and independent of the lanes' order.  The result is
//   sum_q floor(H_2(q)^2 / 2^63)
// in the same fixed point.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esim {

constexpr unsigned long long kTwoHopOne = 1ull << 63;
constexpr unsigned long long kTwoHopTooLarge = ~0ull;  // a real sum never exceeds 2^63

// floor(H^2 / 2^63) for H <= 2^63
__device__ __forceinline__ unsigned long long twohop_sq(unsigned long long H) {
    return (__umul64hi(H, H) << 1) | ((H * H) >> 63);
}

// All 32 lanes of a warp call it with the same k; K and V are the warp's kTable slots
// (kTable a power of two).  Returns the sum above (0 when din(k) = 0), or
// kTwoHopTooLarge when the two-hop multiset (sum of din(q') over q' in I(k)) exceeds
// half the slots.  T receives sum over q' in I(k) with din(q') > 0 of 1/din(q') (FP64,
// fixed lane order) and dk din(k), in every lane.
template <int kTable>
__device__ unsigned long long twohop_sq_sum(int32_t k, const uint32_t* __restrict__ rp,
                                            const int32_t* __restrict__ col, int32_t* K, unsigned long long* V,
                                            double& T, uint32_t& dk) {
    const int lane = threadIdx.x & 31;
    const uint32_t kb = rp[k], ke = rp[k + 1];
    dk = ke - kb;
    T = 0.0;
    if (dk == 0) return 0ull;  // no in-neighbour: the walks stop at once
    unsigned long long e1 = 0;
    for (uint32_t p = kb + lane; p < ke; p += 32) {
        const int32_t q1 = col[p];
        const uint32_t d1 = rp[q1 + 1] - rp[q1];
        e1 += d1;
        if (d1) T += 1.0 / (double)d1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        T += __shfl_xor_sync(0xffffffffu, T, o);
    }
    if (e1 > (unsigned long long)(kTable / 2)) return kTwoHopTooLarge;
    for (int s = lane; s < kTable; s += 32) {
        K[s] = -1;
        V[s] = 0ull;
    }
    __syncwarp();
    for (uint32_t p1 = kb; p1 < ke; ++p1) {  // q' in I(k), then its in-neighbours across the lanes
        const int32_t q1 = col[p1];
        const uint32_t b1 = rp[q1], e1r = rp[q1 + 1];
        if (b1 == e1r) continue;
        const unsigned long long w = kTwoHopOne / ((unsigned long long)dk * (unsigned long long)(e1r - b1));
        for (uint32_t p2 = b1 + lane; p2 < e1r; p2 += 32) {
            const int32_t q = col[p2];
            uint32_t slot = ((uint32_t)q * 2654435761u) & (kTable - 1);
            for (;;) {  // at most half the slots are taken: a free or matching slot exists
                const int32_t prev = atomicCAS(&K[slot], -1, q);
                if (prev == -1 || prev == q) break;
                slot = (slot + 1) & (kTable - 1);
            }
            atomicAdd(&V[slot], w);
        }
    }
    __syncwarp();
    unsigned long long sq = 0;
    for (int s = lane; s < kTable; s += 32) sq += twohop_sq(V[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    __syncwarp();  // the table is free for the warp's next node
    return sq;
}

}  // namespace esim
