// Sample allocation, walk-pair sampler and diagonal estimate.
//
//   allocation (Lemma 4, "Sampling according to pi(k)^2"; Algorithm 1 for the
//   basic form): pi(k) = sum_l pi^l(k); R(k) = ceil(R_b * pi(k)^2) or
//   ceil(R_b * pi(k)), at least 1 where pi(k) > 0; off = exclusive prefix sum
//   of R (uint64).
//
//   sampler (Algorithm 2, walk semantics of Eq. scwwalk): R(k) pairs of
//   independent sqrt(c)-walks from each node k; nonmeet(k) counts the pairs that
//   never visit the same node at the same step.  Pair r of node k draws its
//   randomness from Philox-4x32-10 with counter (r_lo, r_hi, k, t) at step t, so
//   the result is independent of how pairs are spread over threads.  In-neighbour
//   choices are exactly uniform (Lemire's multiply-shift with rejection, ACM TOMS
//   2019; rejected words are replaced from a side stream with counter
//   (r_lo, r_hi, k, 2^31 | W 2^30 | j 2^16 | t), W = 0 for walk A, 1 for walk B).
//
//   D^(k) = nonmeet(k) / R(k) (Algorithm 2).
#include "common.cuh"
#include "internal.h"
#include "philox.cuh"
#include "twofloat.cuh"

#include <math.h>

namespace esim {

constexpr int kAllocItems = 8;
constexpr int64_t kAllocTile = (int64_t)kBlock * kAllocItems;
constexpr int kScanThreads = 1024;
constexpr uint32_t kWalkMaxSteps = 65536;

int64_t allocate_blocks(int64_t n) { return (n + kAllocTile - 1) / kAllocTile; }

uint32_t walk_threshold(double c) {
    double v = floor(sqrt(c) * 4294967296.0);
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

// Block-wide exclusive scan of one uint64 per thread; *total gets the block sum.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* smem,
                                                                   unsigned long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < nw ? smem[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem[lane] = w;
    }
    __syncthreads();
    const unsigned long long warp_off = wid ? smem[wid - 1] : 0ull;
    *total = smem[nw - 1];
    __syncthreads();
    return warp_off + x - v;
}

// pi(k) = sum over levels of hist, in level order: FP64 sums for an FP64 history,
// two-float sums (rounded to FP64) for an FP32 history.
__device__ __forceinline__ double level_sum(const double* __restrict__ hist, int64_t n, int64_t k, int32_t L) {
    double p = 0.0;
    for (int32_t l = 0; l <= L; ++l) p += hist[(size_t)l * (size_t)n + (size_t)k];
    return p;
}

__device__ __forceinline__ double level_sum(const float* __restrict__ hist, int64_t n, int64_t k, int32_t L) {
    f2 p = f2{0.f, 0.f};
    for (int32_t l = 0; l <= L; ++l) p = f2_add_f(p, hist[(size_t)l * (size_t)n + (size_t)k]);
    return f2_to_double(p);
}

// pi(k), R(k) per node; per-tile sums of R (exact and in double) and of pi^2.
template <typename H>
__global__ void __launch_bounds__(kBlock) alloc_reduce_kernel(int64_t n, const H* __restrict__ hist, int32_t L,
                                                              double R_b, int mode, const uint32_t* __restrict__ exact_din,
                                                              double* __restrict__ pi_out,
                                                              uint64_t* __restrict__ R_out,
                                                              unsigned long long* __restrict__ part_R,
                                                              double* __restrict__ part_norm,
                                                              double* __restrict__ part_Rd, Status* __restrict__ st) {
    __shared__ unsigned long long red_u[kBlock / 32];
    __shared__ double red_d[kBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kAllocTile;
    unsigned long long sum_r = 0;
    double norm = 0.0, sum_rd = 0.0;
    bool overflow = false;
#pragma unroll 1
    for (int i = 0; i < kAllocItems; ++i) {
        const int64_t k = base + (int64_t)i * kBlock + threadIdx.x;
        if (k >= n) break;
        const double p = level_sum(hist, n, k, L);
        if (pi_out) pi_out[k] = p;
        const double v = mode == 0 ? R_b * (p * p) : R_b * p;
        unsigned long long r = 0;
        if (v >= 9.2e18 || v != v) {
            overflow = true;
        } else {
            r = (unsigned long long)ceil(v);
            if (r == 0ull && p > 0.0) r = 1ull;  // every reached node gets a pair
            // Algorithm 3: D is exact for din <= 1, so those nodes need no pairs
            if (exact_din && exact_din[k + 1] - exact_din[k] <= 1u) r = 0ull;
        }
        R_out[k] = r;
        sum_r += r;
        sum_rd += (double)r;
        norm += p * p;
    }
    if (overflow) atomicOr(&st->err, kErrBudget);
    sum_r = block_sum(sum_r, red_u);
    norm = block_sum(norm, red_d);
    sum_rd = block_sum(sum_rd, red_d);
    if (threadIdx.x == 0) {
        part_R[blockIdx.x] = sum_r;
        part_norm[blockIdx.x] = norm;
        part_Rd[blockIdx.x] = sum_rd;
    }
}

// One block: exclusive scan of the tile sums (in place), totals into the status
// block and off[n]; the budget check.
__global__ void __launch_bounds__(kScanThreads) alloc_partials_kernel(int64_t nblocks, unsigned long long* part_R,
                                                                      const double* __restrict__ part_norm,
                                                                      const double* __restrict__ part_Rd,
                                                                      double budget, uint64_t* __restrict__ off_n,
                                                                      Status* __restrict__ st) {
    __shared__ unsigned long long su[32];
    __shared__ double sd[32];
    const int64_t per = (nblocks + kScanThreads - 1) / kScanThreads;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    const int64_t b1 = b0 + per < nblocks ? b0 + per : nblocks;
    unsigned long long local = 0;
    double nrm = 0.0, rd = 0.0;
    for (int64_t b = b0; b < b1; ++b) {
        local += part_R[b];
        if (part_norm) nrm += part_norm[b];
        rd += part_Rd[b];
    }
    unsigned long long total;
    unsigned long long run = block_exclusive_scan(local, su, &total);
    for (int64_t b = b0; b < b1; ++b) {
        const unsigned long long v = part_R[b];
        part_R[b] = run;
        run += v;
    }
    nrm = block_sum(nrm, sd);
    rd = block_sum(rd, sd);
    if (threadIdx.x == 0) {
        *off_n = total;
        if (st) {  // NULL: an auxiliary scan that records nothing
            st->sum_R = total;
            if (part_norm) st->pi_norm2 = nrm;
            if (rd > budget || rd >= 1.8e19) atomicOr(&st->err, kErrBudget);
        }
    }
}

// off[k] = tile offset + exclusive prefix of R within the tile.
__global__ void __launch_bounds__(kBlock) alloc_scan_kernel(int64_t n, const uint64_t* __restrict__ R,
                                                            const unsigned long long* __restrict__ tile_off,
                                                            uint64_t* __restrict__ off) {
    __shared__ unsigned long long su[32];
    const int64_t base = (int64_t)blockIdx.x * kAllocTile + (int64_t)threadIdx.x * kAllocItems;
    unsigned long long v[kAllocItems];
    unsigned long long local = 0;
#pragma unroll
    for (int i = 0; i < kAllocItems; ++i) {
        const int64_t k = base + i;
        v[i] = k < n ? R[k] : 0ull;
        local += v[i];
    }
    unsigned long long total;
    unsigned long long run = tile_off[blockIdx.x] + block_exclusive_scan(local, su, &total);
#pragma unroll
    for (int i = 0; i < kAllocItems; ++i) {
        const int64_t k = base + i;
        if (k < n) off[k] = run;
        run += v[i];
    }
}

template <typename H>
cudaError_t launch_allocate_t(const Graph& g, const H* hist, int32_t L, double R_b, int mode, double* pi_out,
                              uint64_t* R_out, uint64_t* off) {
    const int64_t nb = allocate_blocks(g.n);
    unsigned long long* part_R = g.scan_part;
    double* part_norm = g.norm_part;
    double* part_Rd = g.norm_part + nb;
    alloc_reduce_kernel<H><<<(unsigned)nb, kBlock, 0, g.stream>>>(g.n, hist, L, R_b, mode,
                                                                  g.alg3 ? g.in.rp : nullptr, pi_out, R_out, part_R,
                                                                  part_norm, part_Rd, g.status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    alloc_partials_kernel<<<1, kScanThreads, 0, g.stream>>>(nb, part_R, part_norm, part_Rd, g.pair_budget,
                                                            off + g.n, g.status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    alloc_scan_kernel<<<(unsigned)nb, kBlock, 0, g.stream>>>(g.n, R_out, part_R, off);
    return cudaGetLastError();
}

cudaError_t launch_allocate(const Graph& g, const double* hist, int32_t L, double R_b, int mode, double* pi_out,
                            uint64_t* R_out, uint64_t* off) {
    return launch_allocate_t<double>(g, hist, L, R_b, mode, pi_out, R_out, off);
}

cudaError_t launch_allocate32(const Graph& g, const float* hist, int32_t L, double R_b, int mode, double* pi_out,
                              uint64_t* R_out, uint64_t* off) {
    return launch_allocate_t<float>(g, hist, L, R_b, mode, pi_out, R_out, off);
}

// Exactly uniform index in [0, d) from word x (Lemire); rejections (probability
// below d / 2^32) redraw from the walk's side stream.
__device__ __forceinline__ uint32_t pick_redraw(uint32_t d, unsigned long long m, uint32_t rlo, uint32_t rhi, uint32_t k,
                                             uint32_t tag, const PhiloxKeys& K) {
    const uint32_t thr = (0u - d) % d;
    uint32_t l = (uint32_t)m;
    uint32_t j = 0;
    int used = 4;
    uint4 z = make_uint4(0, 0, 0, 0);
    while (l < thr) {
        if (used == 4) {
            if (j == (1u << 14)) break;
            z = philox4x32_10(make_uint4(rlo, rhi, k, tag | (j << 16)), K);
            ++j;
            used = 0;
        }
        const uint32_t x = used == 0 ? z.x : (used == 1 ? z.y : (used == 2 ? z.z : z.w));
        ++used;
        m = (unsigned long long)x * d;
        l = (uint32_t)m;
    }
    return (uint32_t)(m >> 32);
}

// Walks shared across the columns of a batch: segment s covers pairs
// [rbase[s], rbase[s] + len) of node s / B (node-major, B segments per node).
struct SharedSegs {
    int B;                  // 0: segments are (column, node) = (s / n, s % n)
    const uint64_t* rbase;  // first pair index of each segment (NULL unless shared)
};

__device__ __forceinline__ uint32_t segment_node(unsigned long long seg, unsigned long long n_nodes,
                                                 const SharedSegs& sh) {
    if (sh.B) return (uint32_t)(seg / (unsigned long long)sh.B);
    return (uint32_t)(seg < n_nodes ? seg : seg % n_nodes);
}

// State of one walk pair stream: the thread's current node k, pair r of R(k)
// (rk), the two walk positions, the step t, and the pairs still to run.
// A segment is the run of pairs of one (column, node): in a single query segment k
// is node k; in a batch of B columns segment q*n + k is node k of column q.
struct PairState {
    unsigned long long r, rk, left, cnt, g_end, seg;
    uint32_t k, xa, xb, t, d;  // d: Algorithm 3 depth of node k (0: Algorithm 2)
};

// One step of the current pair (branch-free apart from the rare Lemire
// rejection and the change of node): both walks' rows and chosen in-neighbours
// are loaded whether or not the walks move (an index into a row without
// in-edges is clamped to entry 0), and the outcome is applied with selects.
__device__ __forceinline__ void pair_step(PairState& S, const uint2* __restrict__ row,
                                          const int32_t* __restrict__ col, const uint64_t* __restrict__ off,
                                          uint32_t T, const PhiloxKeys& K, unsigned long long* __restrict__ nonmeet,
                                          unsigned long long& steps, unsigned long long n_nodes,
                                          const uint8_t* __restrict__ depth, const SharedSegs& sh) {
    const uint32_t rlo = (uint32_t)S.r, rhi = (uint32_t)(S.r >> 32);
    const uint4 w = philox4x32_10(make_uint4(rlo, rhi, S.k, S.t), K);
    const uint2 ra = __ldg(row + S.xa), rb = __ldg(row + S.xb);  // (first in-edge, din)
    // Algorithm 3's special pairs move without the continuation draw for their first d steps
    const bool forced = S.t < S.d;
    const bool cont = (forced | ((w.x < T) & (w.z < T))) & (ra.y != 0u) & (rb.y != 0u);
    const unsigned long long ma = (unsigned long long)w.y * ra.y;
    const unsigned long long mb = (unsigned long long)w.w * rb.y;
    uint32_t ia = (uint32_t)(ma >> 32), ib = (uint32_t)(mb >> 32);
    if (__builtin_expect(cont & (((uint32_t)ma < ra.y) | ((uint32_t)mb < rb.y)), 0)) {
        if ((uint32_t)ma < ra.y) ia = pick_redraw(ra.y, ma, rlo, rhi, S.k, 0x80000000u | S.t, K);
        if ((uint32_t)mb < rb.y) ib = pick_redraw(rb.y, mb, rlo, rhi, S.k, 0xC0000000u | S.t, K);
    }
    const uint32_t na = (uint32_t)__ldg(col + (ra.y ? ra.x + ia : 0u));
    const uint32_t nb = (uint32_t)__ldg(col + (rb.y ? rb.x + ib : 0u));
    const bool meet = cont & (na == nb);
    const bool ended = !cont | meet | (S.t + 1u >= kWalkMaxSteps);
    S.xa = ended ? S.k : na;
    S.xb = ended ? S.k : nb;
    if (!ended) {
        ++S.t;
        return;
    }
    steps += S.t + 1u;
    // Algorithm 2 counts pairs that never meet; Algorithm 3 counts pairs that first
    // meet after their d forced steps
    S.cnt += S.d ? ((meet & (S.t >= S.d)) ? 1ull : 0ull) : (meet ? 0ull : 1ull);
    S.t = 0;
    if (--S.left == 0) {
        if (S.cnt) atomicAdd(nonmeet + S.seg, S.cnt);
        S.cnt = 0;
        return;
    }
    if (++S.r == S.rk) {  // segment done: flush and move to the next segment with pairs
        if (S.cnt) atomicAdd(nonmeet + S.seg, S.cnt);
        S.cnt = 0;
        const unsigned long long g = S.g_end - S.left;
        do {
            ++S.seg;
            if (sh.B) {  // shared layout: a node's empty intervals are its last ones; skip them at once
                const unsigned long long i = S.seg % (unsigned long long)sh.B;
                if (i != 0 && __ldg(off + S.seg + 1) == __ldg(off + S.seg)) S.seg += (unsigned long long)sh.B - 1 - i;
            }
        } while (__ldg(off + S.seg + 1) <= g);
        S.r = sh.rbase ? __ldg(sh.rbase + S.seg) : 0ull;
        S.rk = S.r + (__ldg(off + S.seg + 1) - __ldg(off + S.seg));
        S.k = segment_node(S.seg, n_nodes, sh);
        S.d = depth ? depth[S.k] : 0u;
        S.xa = S.xb = S.k;
    }
}

// Persistent walk-pair sampler.  Thread t takes a contiguous run of global pair
// indices (about total / #threads of them) and advances its current pair by one
// step per loop iteration, so a lane whose pair ended starts its next pair at
// once and lanes stay busy.  Counts stay in registers while the node does not
// change and are flushed with one atomic add per (thread, node).
__global__ void __launch_bounds__(kBlock, 6) sample_pairs_kernel(int64_t n, int64_t nseg, const uint2* __restrict__ row,
                                                                 const int32_t* __restrict__ col,
                                                                 const uint64_t* __restrict__ off, uint32_t T,
                                                                 const __grid_constant__ PhiloxKeys K, double budget,
                                                                 unsigned long long* __restrict__ nonmeet,
                                                                 unsigned long long* __restrict__ steps_out,
                                                                 Status* __restrict__ st,
                                                                 const uint8_t* __restrict__ depth,
                                                                 const SharedSegs sh) {
    __shared__ unsigned long long red[kBlock / 32];
    const unsigned long long total = off[nseg];
    if ((double)total > budget || (st->err & kErrBudget)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&st->err, kErrBudget);
        return;
    }
    const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long per = total / nthreads, rem = total % nthreads;
    const unsigned long long g0 = tid * per + (tid < rem ? tid : rem);
    const unsigned long long g1 = g0 + per + (tid < rem ? 1ull : 0ull);
    PairState S;
    S.left = g1 - g0;
    S.g_end = g1;
    S.cnt = 0;
    S.t = 0;
    unsigned long long steps = 0;
    if (S.left) {
        int64_t lo = 0, hi = nseg;  // segment of pair g0: off[seg] <= g0 < off[seg+1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(off + mid) <= g0) lo = mid; else hi = mid;
        }
        S.seg = (unsigned long long)lo;
        S.k = segment_node(S.seg, (unsigned long long)n, sh);
        S.d = depth ? depth[S.k] : 0u;
        const unsigned long long rb = sh.rbase ? __ldg(sh.rbase + S.seg) : 0ull;
        S.r = rb + (g0 - __ldg(off + S.seg));
        S.rk = rb + (__ldg(off + S.seg + 1) - __ldg(off + S.seg));
        S.xa = S.xb = S.k;
        for (;;) {
            if (!S.left) break;
            pair_step(S, row, col, off, T, K, nonmeet, steps, (unsigned long long)n, depth, sh);
        }
    }
    steps = block_sum(steps, red);
    if (threadIdx.x == 0 && steps) atomicAdd(steps_out, steps);
}

__global__ void dhat_kernel(int64_t n, const uint64_t* __restrict__ nonmeet, const uint64_t* __restrict__ off,
                            double* __restrict__ dhat) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t R = off[k + 1] - off[k];
        dhat[k] = R ? (double)nonmeet[k] / (double)R : 0.0;
    }
}

__global__ void fill_kernel(int64_t n, double value, double* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = value;
}

__global__ void mask_R_kernel(int64_t n, const uint64_t* __restrict__ R, const uint8_t* __restrict__ keep,
                              uint8_t want_mask, uint64_t* __restrict__ R_out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        R_out[k] = ((want_mask >> keep[k]) & 1u) ? R[k] : 0ull;
}

__global__ void merge_counts_kernel(int64_t n, const uint8_t* __restrict__ cand, const uint64_t* __restrict__ side,
                                    uint64_t* __restrict__ counts) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (cand[k] != 1) counts[k] = side[k];
}

__global__ void plan_scatter_kernel(const PlanEntry* __restrict__ plan, int count, uint64_t* __restrict__ R,
                                    uint8_t* __restrict__ depth, uint8_t* __restrict__ cand) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const PlanEntry e = plan[i];
        if (e.depth) {
            R[e.k] = e.R;
            depth[e.k] = e.depth;
        }
        if (e.early) cand[e.k] = 2;
    }
}

__global__ void mark_kernel(const int32_t* __restrict__ ids, int count, uint8_t* __restrict__ mark) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) mark[ids[i]] = 1u;
}

static int eb_cap(const Graph& g, int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    if (b > (int64_t)g.sm_count * 8) b = (int64_t)g.sm_count * 8;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_mask_R(const Graph& g, const uint64_t* R, const uint8_t* keep, uint8_t want_mask, uint64_t* R_out) {
    mask_R_kernel<<<eb_cap(g, g.n), kBlock, 0, g.stream>>>(g.n, R, keep, want_mask, R_out);
    return cudaGetLastError();
}

cudaError_t launch_merge_counts(const Graph& g, const uint8_t* cand, const uint64_t* side, uint64_t* counts) {
    merge_counts_kernel<<<eb_cap(g, g.n), kBlock, 0, g.stream>>>(g.n, cand, side, counts);
    return cudaGetLastError();
}

cudaError_t launch_plan_scatter(const Graph& g, const PlanEntry* plan, int count, uint64_t* R, uint8_t* depth,
                                uint8_t* cand) {
    if (count <= 0) return cudaSuccess;
    plan_scatter_kernel<<<1, kBlock, 0, g.stream>>>(plan, count, R, depth, cand);
    return cudaGetLastError();
}

cudaError_t launch_mark(const Graph& g, const int32_t* ids, int count, uint8_t* mark) {
    mark_kernel<<<1, kBlock, 0, g.stream>>>(ids, count, mark);
    return cudaGetLastError();
}

static int g_sample_blocks_per_sm = 0;

cudaError_t launch_sample(const Graph& g, const uint64_t* off, double c, uint64_t seed, uint64_t* nonmeet,
                          uint64_t* pair_steps, const uint8_t* depth) {
    return launch_sample_segments(g, g.n, off, c, seed, nonmeet, pair_steps, depth);
}

cudaError_t launch_sample_segments(const Graph& g, int64_t nseg, const uint64_t* off, double c, uint64_t seed,
                                   uint64_t* nonmeet, uint64_t* pair_steps, const uint8_t* depth, int shared_B,
                                   const uint64_t* rbase, bool zero_counts) {
    cudaError_t e = cudaSuccess;
    if (zero_counts && (e = cudaMemsetAsync(nonmeet, 0, sizeof(uint64_t) * (size_t)nseg, g.stream)) != cudaSuccess)
        return e;
    unsigned long long* steps = pair_steps ? (unsigned long long*)pair_steps : &g.status->pair_steps;
    if (pair_steps) {
        e = cudaMemsetAsync(pair_steps, 0, sizeof(uint64_t), g.stream);
        if (e != cudaSuccess) return e;
    }
    if (g_sample_blocks_per_sm == 0) {
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sample_pairs_kernel, kBlock, 0);
        if (e != cudaSuccess) return e;
        g_sample_blocks_per_sm = b > 0 ? b : 1;
    }
    const int per_sm = g.sample_block_cap > 0 && g.sample_block_cap < g_sample_blocks_per_sm ? g.sample_block_cap
                                                                                              : g_sample_blocks_per_sm;
    const unsigned blocks = (unsigned)(g.sm_count * per_sm);
    sample_pairs_kernel<<<blocks, kBlock, 0, g.stream>>>(g.n, nseg, g.in.info, g.in.col, off, walk_threshold(c),
                                                         philox_keys(seed), g.pair_budget,
                                                         (unsigned long long*)nonmeet, steps, g.status, depth,
                                                         SharedSegs{rbase ? shared_B : 0, rbase});
    return cudaGetLastError();
}

cudaError_t launch_dhat(const Graph& g, const uint64_t* nonmeet, const uint64_t* off, double* dhat) {
    return launch_dhat_segments(g, g.n, nonmeet, off, dhat);
}

cudaError_t launch_fill(const Graph& g, int64_t n, double value, double* out) {
    int64_t b = (n + kBlock - 1) / kBlock;
    if (b > (int64_t)g.sm_count * 8) b = (int64_t)g.sm_count * 8;
    fill_kernel<<<(unsigned)(b < 1 ? 1 : b), kBlock, 0, g.stream>>>(n, value, out);
    return cudaGetLastError();
}

cudaError_t launch_dhat_segments(const Graph& g, int64_t nseg, const uint64_t* nonmeet, const uint64_t* off,
                                 double* dhat) {
    int64_t b = (nseg + kBlock - 1) / kBlock;
    if (b > (int64_t)g.sm_count * 8) b = (int64_t)g.sm_count * 8;
    dhat_kernel<<<(unsigned)(b < 1 ? 1 : b), kBlock, 0, g.stream>>>(nseg, nonmeet, off, dhat);
    return cudaGetLastError();
}

// Scan of a ready R array of N segments (batches): tile sums, tile offsets, off[].
__global__ void __launch_bounds__(kBlock) tile_sums_kernel(int64_t N, const uint64_t* __restrict__ R,
                                                           unsigned long long* __restrict__ part_R,
                                                           double* __restrict__ part_Rd) {
    __shared__ unsigned long long red_u[kBlock / 32];
    __shared__ double red_d[kBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kAllocTile;
    unsigned long long su = 0;
    double sd = 0.0;
    for (int i = 0; i < kAllocItems; ++i) {
        const int64_t k = base + (int64_t)i * kBlock + threadIdx.x;
        if (k < N) {
            su += R[k];
            sd += (double)R[k];
        }
    }
    su = block_sum(su, red_u);
    sd = block_sum(sd, red_d);
    if (threadIdx.x == 0) {
        part_R[blockIdx.x] = su;
        part_Rd[blockIdx.x] = sd;
    }
}

cudaError_t launch_scan_R(const Graph& g, int64_t N, const uint64_t* R, uint64_t* off, unsigned long long* part_R,
                          double* part_norm, double* part_Rd, bool record) {
    const int64_t nb = allocate_blocks(N);
    (void)part_norm;  // the scan of a ready R leaves the recorded ||pi||^2 as it is
    tile_sums_kernel<<<(unsigned)nb, kBlock, 0, g.stream>>>(N, R, part_R, part_Rd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    alloc_partials_kernel<<<1, kScanThreads, 0, g.stream>>>(nb, part_R, nullptr, part_Rd, g.pair_budget, off + N,
                                                            record ? g.status : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    alloc_scan_kernel<<<(unsigned)nb, kBlock, 0, g.stream>>>(N, R, part_R, off);
    return cudaGetLastError();
}

}  // namespace esim
