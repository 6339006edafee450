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
//
// A table keeps the list of the slots it has used, so that its sums, its scans and its
// reset touch those slots only: a node costs in proportion to its neighbourhood, not to
// the table.  Between nodes every slot is free (key -1, value 0) and the list is empty.
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

// A hash table of kT slots (a power of two) in shared memory, shared by the threads of one
// warp (or of one block: the callers synchronise accordingly).  K: keys (-1 free), V:
// fixed-point values, U: the used slots in insertion order (kT / 2 entries), n: their
// count.  Callers insert at most kT / 2 distinct keys.
template <int kT>
struct SlotTable {
    int32_t* K;
    unsigned long long* V;
    uint16_t* U;
    unsigned int* n;

    // every slot free and the list empty; threads t of nthreads share the work
    __device__ void clear_all(int t, int nthreads) {
        for (int s = t; s < kT; s += nthreads) {
            K[s] = -1;
            V[s] = 0ull;
        }
        if (t == 0) *n = 0u;
    }

    __device__ __forceinline__ void add(int32_t key, unsigned long long w) {
        uint32_t slot = ((uint32_t)key * 2654435761u) & (kT - 1);
        for (;;) {  // at most half the slots are taken: a free or matching slot exists
            const int32_t prev = atomicCAS(&K[slot], -1, key);
            if (prev == -1) {
                U[atomicAdd(n, 1u)] = (uint16_t)slot;
                break;
            }
            if (prev == key) break;
            slot = (slot + 1) & (kT - 1);
        }
        atomicAdd(&V[slot], w);
    }

    // this thread's share of sum over used slots of floor(V^2 / 2^63)
    __device__ unsigned long long sq_part(int t, int nthreads) const {
        const unsigned int cnt = *n;
        unsigned long long s = 0;
        for (unsigned int i = (unsigned int)t; i < cnt; i += (unsigned int)nthreads) s += twohop_sq(V[U[i]]);
        return s;
    }

    // frees the used slots (the callers synchronise before and after)
    __device__ void reset(int t, int nthreads) {
        const unsigned int cnt = *n;
        for (unsigned int i = (unsigned int)t; i < cnt; i += (unsigned int)nthreads) {
            K[U[i]] = -1;
            V[U[i]] = 0ull;
        }
    }
};

// Per-warp scratch of push_batch.
struct PushScratch {
    uint32_t excl[32];
    uint32_t beg[32];
    unsigned long long w[32];
};

// floor(H / d) for 1 <= d < 2^32, with M = floor((2^64 - 1) / d) (0 for d = 1): the high
// word of H M never exceeds the quotient and falls short of it by at most two, which the
// remainder corrects.
__device__ __forceinline__ unsigned long long floor_div_magic(unsigned long long H, uint32_t d, unsigned long long M) {
    if (d == 1u) return H;
    unsigned long long q = __umul64hi(H, M);
    unsigned long long r = H - q * d;
    while (r >= d) {
        ++q;
        r -= d;
    }
    return q;
}

// All 32 lanes: lane l brings node a_l (-1 for none) and a numerator num_l; every q in
// I(a_l) receives floor(num_l / din(a_l)) in tb.  The (node, in-neighbour) entries of the
// 32 nodes are spread over the lanes (prefix sums of the lengths, then a five-step search
// for each entry's node), so the loads do not wait on one another.
template <class Table>
__device__ void push_batch(int32_t a, unsigned long long num, const uint32_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const unsigned long long* __restrict__ magic, Table& tb,
                           PushScratch& sc) {
    const int lane = threadIdx.x & 31;
    uint32_t b = 0, len = 0;
    unsigned long long w = 0;
    if (a >= 0 && num) {
        b = rp[a];
        len = rp[a + 1] - b;
        if (len) w = floor_div_magic(num, len, magic[a]);
        if (!w) len = 0;
    }
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    sc.excl[lane] = incl - len;
    sc.beg[lane] = b;
    sc.w[lane] = w;
    __syncwarp();
    for (uint32_t f = (uint32_t)lane; f < total; f += 32) {
        int src = 0;  // the last lane whose entries start at or before f: it owns f
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
            if (sc.excl[src + step] <= f) src += step;
        tb.add(col[sc.beg[src] + (f - sc.excl[src])], sc.w[src]);
    }
    __syncwarp();
}

// All 32 lanes of a warp call it with the same k; tb is the warp's table, free on entry.
// Builds H_2 of node k and returns 0, or returns kTwoHopTooLarge (table untouched) when
// the two-hop multiset (sum of din(q') over q' in I(k)) exceeds half the slots.  T
// receives sum over q' in I(k) with din(q') > 0 of 1/din(q') (FP64, fixed lane order)
// and dk din(k), in every lane.  The caller reads the table, then frees it with
// twohop_release.  magic: floor((2^64 - 1) / din) per node (0 where din <= 1).
template <int kT>
__device__ unsigned long long twohop_build(int32_t k, const uint32_t* __restrict__ rp,
                                           const int32_t* __restrict__ col,
                                           const unsigned long long* __restrict__ magic, SlotTable<kT>& tb,
                                           PushScratch& sc, double& T, uint32_t& dk) {
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
    if (e1 > (unsigned long long)(kT / 2)) return kTwoHopTooLarge;
    // every q1 in I(k) holds h_1(q1) = x_0 = floor(2^63 / din(k)) and pushes floor(x_0 / din(q1))
    const unsigned long long x0 = floor_div_magic(kTwoHopOne, dk, magic[k]);
    for (uint32_t base = kb; base < ke; base += 32) {
        const uint32_t p = base + (uint32_t)lane;
        push_batch(p < ke ? col[p] : -1, x0, rp, col, magic, tb, sc);
    }
    return 0ull;
}

// sum over the warp's table of floor(H^2 / 2^63), in every lane
template <int kT>
__device__ unsigned long long warp_sq_sum(const SlotTable<kT>& tb) {
    unsigned long long sq = tb.sq_part(threadIdx.x & 31, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    return sq;
}

// frees the warp's table for its next node
template <int kT>
__device__ void twohop_release(SlotTable<kT>& tb) {
    __syncwarp();
    tb.reset(threadIdx.x & 31, 32);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) *tb.n = 0u;
    __syncwarp();
}

}  // namespace esim
