// Algorithm 3's adaptive depth, as the paper gives it: node k extends walk
// distributions level by level and stops at the level l(k) during which its count of
// explored edges E_k reaches 2 R(k)/sqrt(c), the expected number of steps of its R(k)
// walk pairs ("Local deterministic exploitation for D", Algorithm 3).
//
// At level l the listing extends, for every l' = 0..l and every q' with
// (P^T)^(l-l')(k, q') != 0, the distribution (P^T)^(l')(q', .) by one step: each x in its
// support sends mass to every q in I(x), one explored edge each.  With
//   S_j(q) = supp (P^T)^j(q, .)   and   e_j(q) = sum_{x in S_j(q)} din(x),
// level l adds W_l(k) = sum_{j=0..l} sum_{q' in S_j(k)} e_(l-j)(q'), and l(k) is the
// first l with W_0(k) + ... + W_l(k) >= 2 R(k)/sqrt(c).  Where the listing gives no
// stop, a level that adds no edge ends the exploration (no walk pair can meet later,
// so the Z up to that level give D exactly), and so does the depth cap.
//
// The supports are bit sets, one row of ceil(n/32) words per node: S_0 is the
// identity and S_(j+1)(q) = OR over x in I(q) of S_j(x), a pull over the in-edge CSR.
// A first pass over the levels gives the table e_j(q); a second pass rebuilds S_j and
// adds each still undecided node's terms.  All counts are integers, so the depths
// are exact.  The bit sets take 2 n ceil(n/32) words: the rule is offered for graphs
// whose bit sets fit kPaperBitsBudget.
#include "common.cuh"
#include "internal.h"
#include "twohop.cuh"

#include <algorithm>
#include <vector>

namespace esim {

namespace {

constexpr size_t kPaperBitsBudget = (size_t)4 << 30;  // bytes for the two bit-set levels

int64_t words_of(int64_t n) { return (n + 31) / 32; }

// S_0: row q holds bit q only.
__global__ void bits_identity_kernel(int64_t n, int64_t words, uint32_t* __restrict__ B) {
    const int64_t total = n * words;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / words, w = i - q * words;
        B[i] = (q >> 5) == w ? 1u << (q & 31) : 0u;
    }
}

// S_(j+1)(q) = OR over x in I(q) of S_j(x); one warp per row, lanes over its words.
__global__ void __launch_bounds__(kBlock) bits_step_kernel(int64_t n, int64_t words, const uint32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const uint32_t* __restrict__ Bp, uint32_t* __restrict__ Bn) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < n; q += warps) {
        const uint32_t b = rp[q], e = rp[q + 1];
        for (int64_t w = lane; w < words; w += 32) {
            uint32_t acc = 0;
            for (uint32_t p = b; p < e; ++p) acc |= Bp[(int64_t)col[p] * words + w];
            Bn[q * words + w] = acc;
        }
    }
}

// e(q) = sum of din(x) over the bits x of row q; one warp per row.
__global__ void __launch_bounds__(kBlock) bits_weight_kernel(int64_t n, int64_t words, const uint32_t* __restrict__ B,
                                                            const uint32_t* __restrict__ rp,
                                                            unsigned long long* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < n; q += warps) {
        unsigned long long sum = 0;
        for (int64_t w = lane; w < words; w += 32) {
            uint32_t bits = B[q * words + w];
            while (bits) {
                const int64_t x = w * 32 + (__ffs(bits) - 1);
                sum += rp[x + 1] - rp[x];
                bits &= bits - 1;
            }
        }
        sum = warp_sum_u64(sum);
        if (lane == 0) e[q] = sum;
    }
}

// The undecided nodes to start with: those with R(k) > 0.
__global__ void paper_alive_kernel(int64_t n, const uint64_t* __restrict__ R, int32_t* __restrict__ alive,
                                   unsigned* __restrict__ count) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (R[k] > 0) alive[atomicAdd(count, 1u)] = (int32_t)k;
}

// Level j: W[j+t](k) += sum over q' in S_j(k) of e_t(q'), t = 0..D-j, for the undecided
// nodes; one warp per (node, t).
__global__ void __launch_bounds__(kBlock) paper_level_kernel(int count, const int32_t* __restrict__ alive,
                                                            int64_t n, int64_t words,
                                                            const uint32_t* __restrict__ B,
                                                            const unsigned long long* __restrict__ etab, int j,
                                                            int D, unsigned long long* __restrict__ W) {
    const int lane = threadIdx.x & 31;
    const int terms = D - j + 1;
    const int64_t items = (int64_t)count * terms;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += warps) {
        const int64_t k = alive[it / terms];
        const int t = (int)(it % terms);
        const unsigned long long* et = etab + (int64_t)t * n;
        unsigned long long sum = 0;
        for (int64_t w = lane; w < words; w += 32) {
            uint32_t bits = B[k * words + w];
            while (bits) {
                sum += et[w * 32 + (__ffs(bits) - 1)];
                bits &= bits - 1;
            }
        }
        sum = warp_sum_u64(sum);
        if (lane == 0) W[(int64_t)(j + t) * n + k] += sum;
    }
}

// After level j: node k's count E_k = C(k) + W_j(k); it stops here if E_k reaches
// 2 R(k)/sqrt(c) (compared in FP64, as the oracle does), if level j added no edge, or at
// the cap D.  The others go to the next level's list.
__global__ void paper_decide_kernel(int count, const int32_t* __restrict__ alive, int64_t n, int j, int D,
                                    double sqrt_c, const uint64_t* __restrict__ R,
                                    const unsigned long long* __restrict__ W, unsigned long long* __restrict__ C,
                                    uint8_t* __restrict__ depth, int32_t* __restrict__ next,
                                    unsigned* __restrict__ next_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t k = alive[i];
    const unsigned long long add = W[(int64_t)j * n + k];
    const unsigned long long e = C[k] + add;
    C[k] = e;
    const double T = 2.0 * (double)R[k] / sqrt_c;
    if ((double)e >= T || (j > 0 && add == 0ull) || j == D) {
        depth[k] = (uint8_t)j;
    } else {
        next[atomicAdd(next_count, 1u)] = (int32_t)k;
    }
}

// zsum(k) = Z_1(k) = c sum_{q} ((P^T)(k, q))^2 = c din(k) / din(k)^2 for the nodes of
// depth 1 (a simple graph: each in-neighbour once).
__global__ void paper_z1_kernel(int64_t n, const uint8_t* __restrict__ depth, const uint32_t* __restrict__ rp,
                                double c, double* __restrict__ zsum) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (depth[k] != 1) continue;
        const double d = (double)(rp[k + 1] - rp[k]);
        if (d == 0.0) {  // no in-neighbour: the walks stop at once and never meet
            zsum[k] = 0.0;
            continue;
        }
        const double w = 1.0 / d;
        zsum[k] = c * (d * (w * w));
    }
}

// Depth 2 in closed form.  With h_1 = (P^T)(k, .) (1/din(k) on I(k), a simple graph) and
// h_2 = (P^T)^2(k, .), Lemma 5 gives Z_1(k) = c / din(k) and
//   Z_2(k) = c^2 sum_q h_2(q)^2 - c sum_{q'} Z_1(k, q') sum_q (P^T)(q', q)^2
//          = c^2 (sum_q h_2(q)^2 - (1/din(k)^2) sum_{q' in I(k), din(q') > 0} 1/din(q')).
// One warp per node builds h_2 over the two-hop neighbourhood and sums its squares in
// 63-bit fixed point (twohop.cuh).  A node whose two-hop multiset exceeds half the table
// gets NaN and is left to the one-node Lemma 5 path.
constexpr int kD2Warps = 3;
constexpr int kD2Table = 1024;  // slots per warp (power of two): 3 warps x 13 KB of shared memory

__global__ void __launch_bounds__(kD2Warps * 32) paper_z2_kernel(int count, const int32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ rp,
                                                                 const int32_t* __restrict__ col,
                                                                 const unsigned long long* __restrict__ magic,
                                                                 double c, double* __restrict__ zsum) {
    __shared__ int32_t key[kD2Warps][kD2Table];
    __shared__ unsigned long long val[kD2Warps][kD2Table];
    __shared__ uint16_t used[kD2Warps][kD2Table / 2];
    __shared__ unsigned int nused[kD2Warps];
    __shared__ PushScratch scratch[kD2Warps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SlotTable<kD2Table> tb{key[wid], val[wid], used[wid], &nused[wid]};
    tb.clear_all(lane, 32);
    __syncwarp();
    const int nw = gridDim.x * kD2Warps;
    for (int i = blockIdx.x * kD2Warps + wid; i < count; i += nw) {
        const int32_t k = ids[i];
        double T;
        uint32_t dk;
        const bool large = twohop_build<kD2Table>(k, rp, col, magic, tb, scratch[wid], T, dk) == kTwoHopTooLarge;
        unsigned long long sq = 0;
        if (!large) {
            sq = warp_sq_sum(tb);
            twohop_release(tb);
        }
        if (lane != 0) continue;
        if (dk == 0) zsum[k] = 0.0;  // no in-neighbour: the walks stop at once and never meet
        else if (large) zsum[k] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: the one-node path
        else {
            const double S2 = (double)sq * (1.0 / 9223372036854775808.0);
            const double inv = 1.0 / (double)dk;
            zsum[k] = c * inv + c * c * (S2 - T * inv * inv);
        }
    }
}

// dst[i] = src[ids[i]]
__global__ void gather_f64_kernel(int count, const int32_t* __restrict__ ids, const double* __restrict__ src,
                                  double* __restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) dst[i] = src[ids[i]];
}

int grid_for(const Graph& g, int64_t items_per_warp_rows) {
    const int64_t want = (items_per_warp_rows + (kBlock / 32) - 1) / (kBlock / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g.sm_count * 16));
}

}  // namespace

size_t alg3_paper_bytes(int64_t n, int max_depth) {
    const size_t words = (size_t)words_of(n);
    const size_t bits = 2 * (size_t)n * words * 4;
    const size_t tables = 2 * (size_t)(max_depth + 1) * (size_t)n * 8;  // e table, W table
    const size_t rest = (size_t)n * 8 + 2 * (size_t)n * 4 + 256;        // C, two alive lists, counters
    return bits + tables + rest + 8 * 256;
}

bool alg3_paper_fits(int64_t n) { return 2 * (size_t)n * (size_t)words_of(n) * 4 <= kPaperBitsBudget; }

cudaError_t alg3_paper_depths(const Graph& g, const uint64_t* R, double c, int max_depth, void* ws, uint8_t* depth,
                              int* launches) {
    const int64_t n = g.n, words = words_of(n);
    const int D = max_depth;
    auto align = [](size_t b) { return (b + 255) / 256 * 256; };
    char* p = (char*)ws;
    uint32_t* B0 = (uint32_t*)p;
    p += align((size_t)n * words * 4);
    uint32_t* B1 = (uint32_t*)p;
    p += align((size_t)n * words * 4);
    unsigned long long* etab = (unsigned long long*)p;
    p += align((size_t)(D + 1) * n * 8);
    unsigned long long* W = (unsigned long long*)p;
    p += align((size_t)(D + 1) * n * 8);
    unsigned long long* C = (unsigned long long*)p;
    p += align((size_t)n * 8);
    int32_t* alive[2];
    alive[0] = (int32_t*)p;
    p += align((size_t)n * 4);
    alive[1] = (int32_t*)p;
    p += align((size_t)n * 4);
    unsigned* counts = (unsigned*)p;  // one counter per level list
    cudaStream_t st = g.stream;
    int nl = 0;
    const int ib = (int)std::max<int64_t>(1, std::min<int64_t>((n * words + kBlock - 1) / kBlock,
                                                                (int64_t)g.sm_count * 16));
    const int rb = grid_for(g, n);
    // pass 1: e_j(q) for j = 0..D
    bits_identity_kernel<<<ib, kBlock, 0, st>>>(n, words, B0);
    bits_weight_kernel<<<rb, kBlock, 0, st>>>(n, words, B0, g.in.rp, etab);
    nl += 2;
    uint32_t* cur = B0;
    uint32_t* nxt = B1;
    for (int j = 1; j <= D; ++j) {
        bits_step_kernel<<<rb, kBlock, 0, st>>>(n, words, g.in.rp, g.in.col, cur, nxt);
        bits_weight_kernel<<<rb, kBlock, 0, st>>>(n, words, nxt, g.in.rp, etab + (size_t)j * n);
        std::swap(cur, nxt);
        nl += 2;
    }
    // pass 2: the levels again, the undecided nodes' counts and decisions
    cudaError_t e = cudaMemsetAsync(W, 0, (size_t)(D + 1) * n * 8, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(C, 0, (size_t)n * 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counts, 0, 256, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(depth, 0, (size_t)n, st)) != cudaSuccess) return e;
    paper_alive_kernel<<<rb, kBlock, 0, st>>>(n, R, alive[0], counts);
    bits_identity_kernel<<<ib, kBlock, 0, st>>>(n, words, B0);
    nl += 2;
    cur = B0;
    nxt = B1;
    unsigned count = 0;
    if ((e = cudaMemcpyAsync(&count, counts, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    for (int j = 0; j <= D && count > 0; ++j) {
        if (j > 0) {
            bits_step_kernel<<<rb, kBlock, 0, st>>>(n, words, g.in.rp, g.in.col, cur, nxt);
            std::swap(cur, nxt);
            ++nl;
        }
        const int a = j & 1;
        paper_level_kernel<<<grid_for(g, (int64_t)count * (D - j + 1)), kBlock, 0, st>>>(
            (int)count, alive[a], n, words, cur, etab, j, D, W);
        paper_decide_kernel<<<(count + kBlock - 1) / kBlock, kBlock, 0, st>>>(
            (int)count, alive[a], n, j, D, sqrt(c), R, W, C, depth, alive[a ^ 1], counts + (j + 1));
        nl += 2;
        if ((e = cudaMemcpyAsync(&count, counts + (j + 1), sizeof(unsigned), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

cudaError_t alg3_paper_z2(const Graph& g, const int32_t* ids, int count, double c, double* zsum) {
    if (count <= 0) return cudaSuccess;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((count + kD2Warps - 1) / kD2Warps,
                                                                   (int64_t)g.sm_count * 8));
    paper_z2_kernel<<<blocks, kD2Warps * 32, 0, g.stream>>>(count, ids, g.in.rp, g.in.col, g.din_magic, c, zsum);
    return cudaGetLastError();
}

cudaError_t alg3_gather_f64(const Graph& g, const int32_t* ids, int count, const double* src, double* dst) {
    if (count <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)g.sm_count * 4);
    gather_f64_kernel<<<blocks, 256, 0, g.stream>>>(count, ids, src, dst);
    return cudaGetLastError();
}

cudaError_t alg3_paper_z1(const Graph& g, const uint8_t* depth, double c, double* zsum) {
    paper_z1_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((g.n + kBlock - 1) / kBlock, (int64_t)g.sm_count * 8)),
                      kBlock, 0, g.stream>>>(g.n, depth, g.in.rp, c, zsum);
    return cudaGetLastError();
}

}  // namespace esim
