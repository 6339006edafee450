// Algorithm 3 ("Improved method for estimating D(k,k)"): exact first-meeting
// probabilities Z_1..Z_d of node k by Lemma 5, for any depth d <= kAlg3MaxDepth,
// the supports that choose d, and the diagonal estimate that combines the Z with the
// tail walk pairs.
//
// Notation: h_l = (P^T)^l(k, .), the distribution of a non-stop walk from k after l
// steps (FP64 storage; pull sweeps over the out-edge CSR with no decay, on the warp-tile
// kernel with two-float sums); Zv_l the vector Z_l(k, .) of Lemma 5; P~ the transition
// matrix with squared entries.
// Lemma 5 reads, for each target level j,
//   Zv_j = c^j h_j^2 - c P~ Zv_{j-1} - sum_{l'=2}^{j-1} c^{l'} sum_{q'} Zv_{j-l'}(q') ((P^T)^{l'}(q', .))^2
// (the l' = 1 term is one squared-weight sweep, because (P^T)(q', q)^2 = 1/din(q')^2
// for q in I(q')).  The l' >= 2 terms need the walk distributions of every q' in
// the support of h_{j-l'}: the "probes".  Probes run in blocks of 32 columns (one
// warp lane each), up to kGroupMax blocks per launch.  A probe step maps the
// block's x = h/din to h_next = P x; its epilogue subtracts
// sum_col c^{l'} Zv_i(q'_col) h^{q'_col}_{l'}(q)^2 from Zv_{i+l'}(q) for a level below
// d, or adds h^2 to per-column sums for level d itself (only Z_d's total is needed).
// The last two probe levels run one warp (or one block) per node over hash tables of
// its two- and three-hop neighbourhood instead, with the same integers.
// Z_j = sum_q Zv_j(q) by fixed-order block partials.  Every accumulation that crosses
// blocks or threads is an integer one or has a fixed order, so the result is
// deterministic.
#include "common.cuh"
#include "internal.h"
#include "twohop.cuh"
#include "f2conv.cuh"
#include "twofloat.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace esim {

namespace {

constexpr int kDotBlocks = 1024;
constexpr int kProbeW = 32;      // probe columns per block (one warp lane each)
constexpr int kGroupMax = 8;     // probe blocks per launch
constexpr int kPushChunk = 64;   // in-edges per push work item
constexpr size_t kProbeBudget = (size_t)2 << 30;  // device bytes for the probe groups

// ---------------------------------------------------------------- dense FP64 helpers

// partial[block] of sum_i a(i)^2 (kind 0) or sum_i a(i) (kind 2)
__global__ void __launch_bounds__(kBlock) wsum_kernel(int64_t n, const double* __restrict__ a, int kind,
                                                      double* __restrict__ partial) {
    __shared__ double red[kBlock / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        acc += kind == 2 ? v : v * v;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void sum_partials_kernel(int count, const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    const int per = (count + blockDim.x - 1) / blockDim.x;
    for (int i = threadIdx.x * per; i < (int)((threadIdx.x + 1) * per) && i < count; ++i) acc += partial[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

// Supports of the walk distributions of up to 32 nodes at once, as bit sets: bit c
// of B_l(i) says (P^T)^l(k_c, i) != 0.  B_{l+1}(i) = OR over j in Out(i) of B_l(j)
// (a pull over the out-edge CSR, one warp per row), and lane c of each warp counts
// the rows with bit c set; one integer atomic per column and block gives
// |supp h_l| for each of the 32 nodes.
__global__ void reach_init_kernel(const int32_t* __restrict__ ks, int count, uint32_t* __restrict__ Bm) {
    if ((int)threadIdx.x < count) atomicOr(Bm + ks[threadIdx.x], 1u << threadIdx.x);
}

__global__ void __launch_bounds__(kBlock) reach_step_kernel(int64_t n, const uint32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const uint32_t* __restrict__ Bcur,
                                                            uint32_t* __restrict__ Bnext,
                                                            unsigned long long* __restrict__ counts) {
    constexpr int kWarps = kBlock / 32;
    __shared__ unsigned long long red[kWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    unsigned long long cnt = 0ull;
    for (int64_t row = (int64_t)blockIdx.x * kWarps + wib; row < n; row += nw) {
        const uint32_t b = __ldg(rp + row), e = __ldg(rp + row + 1);
        uint32_t acc = 0u;
        for (uint32_t p = b + lane; p < e; p += 32) acc |= Bcur[__ldg(col + p)];
        acc = __reduce_or_sync(0xffffffffu, acc);
        if (lane == 0) Bnext[row] = acc;
        cnt += (acc >> lane) & 1u;
    }
    red[wib][lane] = cnt;
    __syncthreads();
    if (wib == 0) {
        unsigned long long t = 0ull;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += red[w][lane];
        if (t) atomicAdd(counts + lane, t);
    }
}

// flag(i) = h(i) != 0, as the uint64 counts of the offset scan
__global__ void flag_kernel(int64_t n, const double* __restrict__ h, uint64_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = h[i] != 0.0 ? 1ull : 0ull;
}

// ids[off(i)] = i for the flagged i: the support in ascending order
__global__ void scatter_ids_kernel(int64_t n, const uint64_t* __restrict__ flag, const uint64_t* __restrict__ off,
                                   int32_t* __restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) ids[off[i]] = (int32_t)i;
}

// x = v / din^2 as a two-float: the input of the squared-transition sweep P~ v
__global__ void sq_scale_kernel(int64_t n, const double* __restrict__ v, const double* __restrict__ inv_din,
                                float2* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = inv_din[i];
        const f2 t = double_to_f2_bits(v[i] * (w * w));
        x[i] = make_float2(t.hi, t.lo);
    }
}

// Probe terms of the levels below d are summed in signed two-word fixed point (integer
// atomics: exact, order-free): each term t is split into the nearest multiple of 2^-58
// (the hi word) and the remainder in units of 2^-98 (the lo word), so that no term is
// lost however small it is and the result does not depend on the order of the terms.
// A row's total over all columns is at most c^2 < 1 in magnitude, so the hi words do not
// overflow; a lo term is at most 2^39 in magnitude.
constexpr double kZOne = 288230376151711744.0;  // 2^58
constexpr double kZLo = 1099511627776.0;        // 2^40: lo units per hi unit

// t = (hi + lo 2^-40) 2^-58 to within 2^-99, for |t| < 1
__device__ __forceinline__ void zacc_split(double t, long long& hi, long long& lo) {
    const double s = t * kZOne;            // exact: a power-of-two scale
    hi = __double2ll_rn(s);
    lo = __double2ll_rn((s - (double)hi) * kZLo);  // s - hi is exact (|s - hi| <= 1/2)
}

// Zv_j = c^j h_j^2 - c T + (probe terms), T = P~ Zv_{j-1} (T = NULL at j = 1)
__global__ void zv_finalize_kernel(int64_t n, double cj, double c, const double* __restrict__ h,
                                   const double* __restrict__ T, const long long* __restrict__ zhi,
                                   const long long* __restrict__ zlo, double* __restrict__ zv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double hv = h[i];
        double z = cj * (hv * hv);
        if (T) z -= c * T[i];
        zv[i] = z + ((double)zhi[i] * (1.0 / kZOne) + (double)zlo[i] * (1.0 / (kZOne * kZLo)));
    }
}

// ---------------------------------------------------------------- probes
//
// A probe value is a probability in [0, 1]; probes carry it in unsigned 64-bit fixed
// point with 63 fraction bits (kOne = 2^63).  FP64 issue on GB300 is a small fraction
// of its integer rate, and the probe sweeps add one value per edge and column, so the
// sums run on the integer pipe: exact additions (no overflow: a row sum of x = h/din
// over out-neighbours never exceeds the total mass 1), truncating divisions by din
// and truncating squares.  The truncations cost at most 2^-63 each, far below the
// FP64 rounding of the rest of the computation.
constexpr unsigned long long kOne = 1ull << 63;
constexpr double kInvOne = 1.0 / 9223372036854775808.0;  // 2^-63



// Direction-optimising steps.  A block starts from 32 single nodes, so its first
// steps touch few rows.  While the frontier F_s (the rows of x_s that may be
// non-zero) has few in-edges, a step pushes x_s(j) to the rows i in I(j) with
// integer atomics into an n x 32 accumulator (exact, so the order of the atomics does
// not matter) and processes only the touched rows; once the frontier's in-edges
// exceed (m + n) / alg3_push_div (default 4) the step and all later ones of the block
// run the dense pull.
// Both forms give the same integers, so the switch changes no bit of the result.
// The frontier, its in-edge count and the work list of 64-entry chunks live on the
// device; the kernels of a step read the same counters, so all agree on the form
// without a host round trip.
struct ProbeStepCnt {
    unsigned int fcount;      // rows in F_s
    unsigned int wcount;      // push work items of F_s (64-entry chunks of in-rows)
    unsigned long long push;  // in-edges of F_s
};

struct ProbeCtl {
    ProbeStepCnt st[kAlg3MaxDepth + 2];
    int dense_plus1;  // 0: sparse so far; s + 1: dense from step s on
    int pad;
};

__device__ __forceinline__ bool probe_dense_at(const ProbeCtl* ctl, int s, unsigned long long thr) {
    const int d = *(volatile const int*)&ctl->dense_plus1;
    return (d != 0 && d - 1 <= s) || ctl->st[s].push > thr;
}

// The buffers of a probe group: block b (blockIdx.y) owns slice b of each.
struct ProbeGroup {
    unsigned long long* X[2];   // x ping-pong, 32 n each
    unsigned long long* Hn;     // push accumulator, 32 n (zero between steps)
    uint32_t* mark;             // n (zero between steps)
    int32_t* F[2];              // frontiers, n each
    int2* W[2];                 // push work items, nw each
    unsigned long long* ppart;  // dense long-row partials, 32 nseg
    ProbeCtl* ctl;              // one per block
    double* coef;               // 32 per block
    unsigned long long* colsum; // 32 per block
    size_t nx, nw, np;          // slice strides of X/Hn, W, ppart
    int64_t n;
};

// What a step does with h_{s+1}: mode 0 nothing, 1 subtract the row terms from a level
// below d (zfx), 2 add h^2 to the column sums (level d).
struct ProbeStepArgs {
    const uint32_t* in_rp;
    const int32_t* in_col;
    const unsigned long long* magic;  // floor((2^64 - 1) / din) per node (division by din)
    int s;               // step index (h_{s+1} is produced)
    int src;             // which X buffer holds x_s
    int mode;
    int last;            // no further step: x_{s+1} is not needed
    long long* zfx;      // mode 1 target: hi words of the level
    long long* zlo;      // and its lo words
    unsigned long long thr;
};

// Row `row` of h_{s+1} is H (fixed point) in lane = column.  All 32 lanes of the warp
// call it.  Writes x_{s+1} (unless last); returns this lane's h^2 for mode 2.
__device__ __forceinline__ unsigned long long probe_row_out(int64_t row, unsigned long long H, int lane,
                                                            const ProbeStepArgs& a, unsigned long long* xnext,
                                                            const double* coef) {
    if (!a.last) {
        const uint32_t d = __ldg(a.in_rp + row + 1) - __ldg(a.in_rp + row);
        xnext[(size_t)row * kProbeW + lane] = (d && H) ? floor_div_magic(H, d, __ldg(a.magic + row)) : 0ull;
    }
    if (a.mode == 2) return twohop_sq(H);  // floor(H^2 / 2^63)
    if (a.mode == 1 && __any_sync(0xffffffffu, H != 0ull)) {
        // each column's term is rounded to fixed point on its own and the integers are
        // added, so the result does not depend on which columns share a block
        const double h = (double)H * kInvOne;
        long long hi, lo;
        zacc_split(coef[lane] * (h * h), hi, lo);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hi += __shfl_xor_sync(0xffffffffu, hi, o);
            lo += __shfl_xor_sync(0xffffffffu, lo, o);
        }
        if (lane == 0 && hi != 0) atomicAdd((unsigned long long*)(a.zfx + row), (unsigned long long)(-hi));
        if (lane == 0 && lo != 0) atomicAdd((unsigned long long*)(a.zlo + row), (unsigned long long)(-lo));
    }
    return 0ull;
}

// Column sums of mode 2: lane sums of the block's warps, then one integer atomic per
// column (order-free, so exact and deterministic).
__device__ __forceinline__ void probe_flush_colsum(unsigned long long v, unsigned long long* colsum) {
    constexpr int kWarps = kBlock / 32;
    __shared__ unsigned long long red[kWarps][kProbeW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    red[wib][lane] = v;
    __syncthreads();
    if (wib == 0) {
        unsigned long long t = 0ull;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += red[w][lane];
        if (t) atomicAdd(colsum + lane, t);
    }
}

// Group start (one warp per block): x_0 = e_{q'} / din(q') per column, F_0 = the
// sources, their work items, fresh counters and column sums.
__global__ void probe_init_kernel(ProbeGroup G, const int32_t* __restrict__ ids, int count,
                                  const uint32_t* __restrict__ in_rp) {
    const int b = blockIdx.y, lane = threadIdx.x;
    ProbeCtl* ctl = G.ctl + b;
    uint32_t* z = (uint32_t*)ctl;
    for (int i = lane; i < (int)(sizeof(ProbeCtl) / 4); i += 32) z[i] = 0u;
    __syncwarp();
    const int left = count - b * kProbeW;
    const int cnt = left < kProbeW ? left : kProbeW;
    int32_t q = -1;
    uint32_t d = 0;
    if (lane < cnt) {
        q = ids[b * kProbeW + lane];
        d = in_rp[q + 1] - in_rp[q];
        G.X[0][(size_t)b * G.nx + (size_t)q * kProbeW + lane] = d ? kOne / d : 0ull;
        G.F[0][(size_t)b * G.n + lane] = q;
    }
    const unsigned int nch = (d + kPushChunk - 1) / kPushChunk;
    unsigned int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned int base = incl - nch;
    for (unsigned int ch = 0; ch < nch; ++ch) G.W[0][(size_t)b * G.nw + base + ch] = make_int2(q, (int)ch);
    unsigned long long dsum = d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    if (lane == 0) {
        ctl->st[0].fcount = (unsigned int)cnt;
        ctl->st[0].wcount = total;
        ctl->st[0].push = dsum;
    }
    G.colsum[(size_t)b * kProbeW + lane] = 0ull;
}

// coef(b, col) = c^{l'} Zv_i(q'_col); 0 for unused columns
__global__ void probe_coef_kernel(ProbeGroup G, const int32_t* __restrict__ ids, int count,
                                  const double* __restrict__ zv_src, double cl) {
    const int i = blockIdx.y * kProbeW + threadIdx.x;
    G.coef[i] = i < count ? cl * zv_src[ids[i]] : 0.0;
}

// Push step (one warp per work item): every entry i of the chunk receives x_s(j) in
// all 32 columns; each lane marks one entry's row and the new rows are appended to
// F_{s+1} with one atomic per warp.
__global__ void __launch_bounds__(kBlock) probe_push_kernel(ProbeGroup G, ProbeStepArgs a) {
    const int b = blockIdx.y;
    ProbeCtl* ctl = G.ctl + b;
    if (probe_dense_at(ctl, a.s, a.thr)) return;
    const int lane = threadIdx.x & 31;
    const unsigned long long* X = G.X[a.src] + (size_t)b * G.nx;
    unsigned long long* Hn = G.Hn + (size_t)b * G.nx;
    uint32_t* mark = G.mark + (size_t)b * G.n;
    const int2* W = G.W[a.s & 1] + (size_t)b * G.nw;
    int32_t* Fnext = G.F[(a.s + 1) & 1] + (size_t)b * G.n;
    const unsigned int items = ctl->st[a.s].wcount;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (int64_t)items; w += nwarps) {
        const int2 it = W[w];
        const int32_t j = it.x;
        const unsigned long long xv = X[(size_t)j * kProbeW + lane];
        if (!__any_sync(0xffffffffu, xv != 0ull)) continue;  // adds nothing, touches nothing
        const uint32_t rb = __ldg(a.in_rp + j), re = __ldg(a.in_rp + j + 1);
        const uint32_t beg = rb + (uint32_t)it.y * kPushChunk;
        const uint32_t end = beg + kPushChunk < re ? beg + kPushChunk : re;
        for (uint32_t p0 = beg; p0 < end; p0 += 32) {
            const uint32_t p = p0 + lane;
            const int32_t mine = p < end ? __ldg(a.in_col + p) : -1;
            bool fresh = false;
            unsigned long long din_new = 0;
            if (mine >= 0) {
                fresh = atomicExch(mark + mine, 1u) == 0u;
                if (fresh) din_new = __ldg(a.in_rp + mine + 1) - __ldg(a.in_rp + mine);
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            if (fm) {
                unsigned long long dsum = din_new;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                unsigned int base = 0;
                if (lane == 0) {
                    base = atomicAdd(&ctl->st[a.s + 1].fcount, (unsigned int)__popc(fm));
                    atomicAdd(&ctl->st[a.s + 1].push, dsum);
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                if (fresh) Fnext[base + __popc(fm & ((1u << lane) - 1u))] = mine;
            }
            const int cnt = (int)(end - p0 < 32 ? end - p0 : 32);  // warp-uniform
            for (int t = 0; t < cnt; ++t) {
                const int32_t i = __shfl_sync(0xffffffffu, mine, t);
                if (xv) atomicAdd(Hn + (size_t)i * kProbeW + lane, xv);
            }
        }
    }
}

// Sparse epilogue: the rows of F_{s+1} (h_{s+1} from the accumulator, which is
// cleared), the next step's work items; then x_s is cleared on F_s.
__global__ void __launch_bounds__(kBlock) probe_sparse_epi_kernel(ProbeGroup G, ProbeStepArgs a) {
    const int b = blockIdx.y;
    ProbeCtl* ctl = G.ctl + b;
    if (probe_dense_at(ctl, a.s, a.thr)) return;
    const int lane = threadIdx.x & 31;
    unsigned long long* Hn = G.Hn + (size_t)b * G.nx;
    uint32_t* mark = G.mark + (size_t)b * G.n;
    const int32_t* Fnext = G.F[(a.s + 1) & 1] + (size_t)b * G.n;
    const int32_t* Fcur = G.F[a.s & 1] + (size_t)b * G.n;
    unsigned long long* Xcur = G.X[a.src] + (size_t)b * G.nx;
    unsigned long long* Xnext = G.X[a.src ^ 1] + (size_t)b * G.nx;
    int2* Wnext = G.W[(a.s + 1) & 1] + (size_t)b * G.nw;
    const double* coef = G.coef + (size_t)b * kProbeW;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned int nf = ctl->st[a.s + 1].fcount;
    unsigned long long nacc = 0ull;
    for (int64_t r = w0; r < (int64_t)nf; r += nwarps) {
        const int32_t i = Fnext[r];
        const size_t at = (size_t)i * kProbeW + lane;
        const unsigned long long H = Hn[at];
        Hn[at] = 0ull;
        if (lane == 0) {
            mark[i] = 0u;
            const uint32_t d = __ldg(a.in_rp + i + 1) - __ldg(a.in_rp + i);
            if (!a.last && d) {
                const unsigned int nch = (d + kPushChunk - 1) / kPushChunk;
                const unsigned int base = atomicAdd(&ctl->st[a.s + 1].wcount, nch);
                for (unsigned int ch = 0; ch < nch; ++ch) Wnext[base + ch] = make_int2(i, (int)ch);
            }
        }
        nacc += probe_row_out(i, H, lane, a, Xnext, coef);
    }
    const unsigned int nc = ctl->st[a.s].fcount;
    for (int64_t r = w0; r < (int64_t)nc; r += nwarps) Xcur[(size_t)Fcur[r] * kProbeW + lane] = 0ull;
    if (a.mode == 2) probe_flush_colsum(nacc, G.colsum + (size_t)b * kProbeW);
}

// Sum of X(col[p], lane) over entries [b, e), eight gathers in flight (integer adds).
__device__ __forceinline__ unsigned long long probe_range(const int32_t* __restrict__ col,
                                                          const unsigned long long* __restrict__ X, uint32_t b,
                                                          uint32_t e, int lane) {
    unsigned long long acc = 0ull;
    uint32_t p = b;
    for (; p + 8 <= e; p += 8) {
        int32_t j[8];
        unsigned long long v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) j[t] = __ldg(col + p + t);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = X[(size_t)j[t] * kProbeW + lane];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc += v[t];
    }
    for (; p < e; ++p) acc += X[(size_t)__ldg(col + p) * kProbeW + lane];
    return acc;
}

// Dense step: h(i, col) = sum_{j in Out(i)} x_s(j, col), a pull over the out-edge CSR
// for 32 columns at once.  Short rows: one warp per row, lane = column.  Long rows:
// one block per 4096-entry segment, each warp adding a contiguous eighth of it into
// the segment's partial; probe_long_rows_kernel adds a row's partials.
__global__ void __launch_bounds__(kBlock) probe_rows_kernel(ProbeGroup G, ProbeStepArgs a,
                                                            const uint32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col, uint32_t long_min,
                                                            int64_t nseg, const Segment* __restrict__ seg,
                                                            int short_blocks) {
    constexpr int kWarps = kBlock / 32;
    const int b = blockIdx.y;
    ProbeCtl* ctl = G.ctl + b;
    if (!probe_dense_at(ctl, a.s, a.thr)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&ctl->dense_plus1, 0, a.s + 1);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned long long* X = G.X[a.src] + (size_t)b * G.nx;
    if ((int)blockIdx.x >= short_blocks) {
        __shared__ unsigned long long red[kWarps][kProbeW];
        unsigned long long* partial = G.ppart + (size_t)b * G.np;
        const int64_t nsb = (int64_t)gridDim.x - short_blocks;
        for (int64_t s = (int64_t)blockIdx.x - short_blocks; s < nseg; s += nsb) {  // uniform per block
            const Segment sg = seg[s];
            const uint32_t per = (sg.end - sg.beg + kWarps - 1) / kWarps;
            uint32_t bb = sg.beg + (uint32_t)wib * per;
            if (bb > sg.end) bb = sg.end;
            const uint32_t e = bb + per < sg.end ? bb + per : sg.end;
            red[wib][lane] = probe_range(col, X, bb, e, lane);
            __syncthreads();
            if (wib == 0) {
                unsigned long long t = 0ull;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) t += red[w][lane];
                partial[(size_t)s * kProbeW + lane] = t;
            }
            __syncthreads();
        }
        return;
    }
    unsigned long long* Xnext = G.X[a.src ^ 1] + (size_t)b * G.nx;
    const double* coef = G.coef + (size_t)b * kProbeW;
    unsigned long long nacc = 0ull;
    const int64_t nw = (int64_t)short_blocks * kWarps;
    for (int64_t row = (int64_t)blockIdx.x * kWarps + wib; row < G.n; row += nw) {
        const uint32_t rb = __ldg(rp + row), re = __ldg(rp + row + 1);
        if (re - rb >= long_min) continue;  // warp-uniform: a long row
        nacc += probe_row_out(row, probe_range(col, X, rb, re, lane), lane, a, Xnext, coef);
    }
    if (a.mode == 2) probe_flush_colsum(nacc, G.colsum + (size_t)b * kProbeW);
}

__global__ void __launch_bounds__(kBlock) probe_long_rows_kernel(ProbeGroup G, ProbeStepArgs a, int64_t nlong,
                                                                 const int32_t* __restrict__ long_rows,
                                                                 const int32_t* __restrict__ long_first) {
    const int b = blockIdx.y;
    if (!probe_dense_at(G.ctl + b, a.s, a.thr)) return;
    const int lane = threadIdx.x & 31;
    const unsigned long long* partial = G.ppart + (size_t)b * G.np;
    unsigned long long* Xnext = G.X[a.src ^ 1] + (size_t)b * G.nx;
    const double* coef = G.coef + (size_t)b * kProbeW;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long nacc = 0ull;
    if (w < nlong) {  // warp-uniform
        unsigned long long acc = 0ull;
        for (int32_t s = long_first[w]; s < long_first[w + 1]; ++s) acc += partial[(size_t)s * kProbeW + lane];
        nacc = probe_row_out(long_rows[w], acc, lane, a, Xnext, coef);
    }
    if (a.mode == 2) probe_flush_colsum(nacc, G.colsum + (size_t)b * kProbeW);
}

// Group end: zlast += the sum over blocks and columns, in order, of
// c^{steps} Zv_i(q'_col) colsum(b, col); blocks that went dense clear both x buffers.
__global__ void probe_end_kernel(ProbeGroup G, const int32_t* __restrict__ ids, int count,
                                 const double* __restrict__ zv_src, double cl, double* __restrict__ zlast,
                                 const int32_t* __restrict__ pos, unsigned long long* __restrict__ colsum_out) {
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        if (colsum_out) {  // the caller sums the terms: hand over the column sums
            for (int i = threadIdx.x; i < count; i += blockDim.x) colsum_out[pos[i]] = G.colsum[i];
        } else if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < count; ++i) t += (cl * zv_src[ids[i]]) * ((double)G.colsum[i] * kInvOne);
            *zlast += t;
        }
    }
    const int b = blockIdx.y;
    if (G.ctl[b].dense_plus1 == 0) return;
    unsigned long long* xa = G.X[0] + (size_t)b * G.nx;
    unsigned long long* xb = G.X[1] + (size_t)b * G.nx;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.nx; i += (size_t)gridDim.x * blockDim.x) {
        xa[i] = 0ull;
        xb[i] = 0ull;
    }
}

// The last probe level (probes of length 2 from the support of h_{d-2}) needs of each
// node q' only g_2(q') = sum_q ((P^T)^2(q', .))(q)^2, its column sum.  One warp per node
// computes it from the two-hop hash table (twohop.cuh: the same integers as the dense
// probe's two steps); a node whose two-hop multiset is too large for the table is
// appended to (big_ids, big_pos) for the dense probes, which write its column sum at
// big_pos.  The order of the appends does not matter: each column sum is exact.
constexpr int kG2Warps = 3;
constexpr int kG2Table = 1024;  // slots per warp: 3 warps x 13 KB of shared memory

__global__ void __launch_bounds__(kG2Warps * 32) probe_g2_kernel(const uint64_t* __restrict__ count_dev,
                                                                 const int32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ rp,
                                                                 const int32_t* __restrict__ col,
                                                                 const unsigned long long* __restrict__ magic,
                                                                 unsigned long long* __restrict__ colsum,
                                                                 int32_t* __restrict__ big_ids,
                                                                 int32_t* __restrict__ big_pos,
                                                                 unsigned int* __restrict__ nbig) {
    __shared__ int32_t key[kG2Warps][kG2Table];
    __shared__ unsigned long long val[kG2Warps][kG2Table];
    __shared__ uint16_t used[kG2Warps][kG2Table / 2];
    __shared__ unsigned int nused[kG2Warps];
    __shared__ PushScratch scratch[kG2Warps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SlotTable<kG2Table> tb{key[wid], val[wid], used[wid], &nused[wid]};
    tb.clear_all(lane, 32);
    __syncwarp();
    const int64_t count = (int64_t)*count_dev;
    const int64_t nw = (int64_t)gridDim.x * kG2Warps;
    for (int64_t i = (int64_t)blockIdx.x * kG2Warps + wid; i < count; i += nw) {
        double T;
        uint32_t dk;
        const bool large = twohop_build<kG2Table>(ids[i], rp, col, magic, tb, scratch[wid], T, dk) == kTwoHopTooLarge;
        unsigned long long sq = 0;
        if (!large) {
            sq = warp_sq_sum(tb);
            twohop_release(tb);
        }
        if (lane != 0) continue;
        if (large) {
            const unsigned int slot = atomicAdd(nbig, 1u);
            big_ids[slot] = ids[i];
            big_pos[slot] = (int32_t)i;
            colsum[i] = 0ull;
        } else {
            colsum[i] = sq;
        }
    }
}

// The level below the last (probes of length 3 from the support of h_{d-3}) needs of each
// node q' its second step's row terms, c^2 Zv(q') h_2^{q'}(q)^2 subtracted from level d-1,
// and its third step's column sum g_3(q') = sum_q h_3^{q'}(q)^2.  One warp per node:
// the two-hop table (twohop.cuh) holds H_2 over the two-hop neighbourhood; its entries
// give the row terms (two-word fixed point, as the dense epilogue);
// then x_2 = floor(H_2 / din) is pushed one more step into a second table, keyed by the
// three-hop nodes, whose squares give g_3.  These are the dense probe's integers (the
// same truncating divisions and sums, each row term rounded to fixed point on its own),
// so a node gives the same terms on either path.  A node whose two- or three-hop
// multiset is too large for the tables is appended to (big_ids, big_pos) for the dense
// probes, before it emits anything.
constexpr int kG3Warps = 4;
constexpr int kG3Table1 = 1024;  // two-hop slots per warp
constexpr int kG3Table2 = 1024;  // three-hop slots per warp
constexpr size_t kG3WarpBytes = (size_t)(kG3Table1 + kG3Table2) * (sizeof(int32_t) + sizeof(unsigned long long)) +
                                (size_t)(kG3Table1 + kG3Table2) / 2 * sizeof(uint16_t) + 16 + sizeof(PushScratch);
constexpr size_t kG3Smem = (size_t)kG3Warps * kG3WarpBytes;

// the shared memory of one warp: values, keys, used-slot lists, counts
template <int kT1, int kT2>
__device__ __forceinline__ void carve_tables(unsigned char* base, SlotTable<kT1>& t1, SlotTable<kT2>& t2) {
    t1.V = (unsigned long long*)base;
    t2.V = t1.V + kT1;
    t1.K = (int32_t*)(t2.V + kT2);
    t2.K = t1.K + kT1;
    t1.U = (uint16_t*)(t2.K + kT2);
    t2.U = t1.U + kT1 / 2;
    t1.n = (unsigned int*)(((uintptr_t)(t2.U + kT2 / 2) + 7) & ~(uintptr_t)7);
    t2.n = t1.n + 1;
}

// The third step of a node from its two-hop table t1 into t2 (all lanes of the warp):
// H_3(r) = sum over two-hop keys a with r in I(a) of floor(H_2(a) / din(a)).
template <int kT1, int kT2>
__device__ void warp_third_step(const SlotTable<kT1>& t1, SlotTable<kT2>& t2, const uint32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const unsigned long long* __restrict__ magic,
                                PushScratch& sc) {
    const int lane = threadIdx.x & 31;
    const unsigned int cnt = *t1.n;
    for (unsigned int i0 = 0; i0 < cnt; i0 += 32) {
        const unsigned int i = i0 + (unsigned int)lane;
        const int slot = i < cnt ? (int)t1.U[i] : -1;
        push_batch(slot >= 0 ? t1.K[slot] : -1, slot >= 0 ? t1.V[slot] : 0ull, rp, col, magic, t2, sc);
    }
}

__global__ void __launch_bounds__(kG3Warps * 32) probe_g3_kernel(const uint64_t* __restrict__ count_dev,
                                                                 const int32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ rp,
                                                                 const int32_t* __restrict__ col,
                                                                 const unsigned long long* __restrict__ magic,
                                                                 const double* __restrict__ zv_src, double c2,
                                                                 long long* __restrict__ zhi_next,
                                                                 long long* __restrict__ zlo_next,
                                                                 unsigned long long* __restrict__ colsum,
                                                                 int32_t* __restrict__ big_ids,
                                                                 int32_t* __restrict__ big_pos,
                                                                 unsigned int* __restrict__ nbig) {
    extern __shared__ __align__(16) unsigned char g3_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    SlotTable<kG3Table1> t1;
    SlotTable<kG3Table2> t2;
    unsigned char* mine = g3_smem + (size_t)wid * kG3WarpBytes;
    PushScratch& sc = *(PushScratch*)mine;
    carve_tables(mine + sizeof(PushScratch), t1, t2);
    t1.clear_all(lane, 32);
    t2.clear_all(lane, 32);
    __syncwarp();
    const int64_t count = (int64_t)*count_dev;
    const int64_t nw = (int64_t)gridDim.x * kG3Warps;
    for (int64_t i = (int64_t)blockIdx.x * kG3Warps + wid; i < count; i += nw) {
        const int32_t q = ids[i];
        double T;
        uint32_t dk;
        const bool built = twohop_build<kG3Table1>(q, rp, col, magic, t1, sc, T, dk) != kTwoHopTooLarge;
        bool big = !built;
        if (built && dk) {  // the three-hop multiset: sum of din over the two-hop keys
            const unsigned int cnt = *t1.n;
            unsigned long long e2 = 0;
            for (unsigned int u = (unsigned int)lane; u < cnt; u += 32) {
                const int32_t a = t1.K[t1.U[u]];
                e2 += rp[a + 1] - rp[a];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            big = e2 > (unsigned long long)(kG3Table2 / 2);
        }
        if (big) {
            if (built) twohop_release(t1);
            if (lane == 0) {
                const unsigned int slot = atomicAdd(nbig, 1u);
                big_ids[slot] = q;
                big_pos[slot] = (int32_t)i;
                colsum[i] = 0ull;
            }
            continue;
        }
        if (dk == 0) {  // no walk leaves q: no terms
            if (lane == 0) colsum[i] = 0ull;
            continue;
        }
        // row terms of the second step
        const double coef = c2 * zv_src[q];
        const unsigned int cnt1 = *t1.n;
        for (unsigned int u = (unsigned int)lane; u < cnt1; u += 32) {
            const int slot = t1.U[u];
            const double h = (double)t1.V[slot] * kInvOne;
            long long hi, lo;
            zacc_split(coef * (h * h), hi, lo);
            if (hi != 0) atomicAdd((unsigned long long*)(zhi_next + t1.K[slot]), (unsigned long long)(-hi));
            if (lo != 0) atomicAdd((unsigned long long*)(zlo_next + t1.K[slot]), (unsigned long long)(-lo));
        }
        warp_third_step(t1, t2, rp, col, magic, sc);
        const unsigned long long sq3 = warp_sq_sum(t2);
        if (lane == 0) colsum[i] = sq3;
        twohop_release(t2);
        twohop_release(t1);
    }
}

// Second tier of the last two probe levels: the nodes too large for a warp's tables get
// a whole block (8 warps) and tables in most of its shared memory; warps take the outer
// entries, lanes the inner ones, and the inserts and additions are the same integer
// atomics, so a node gives the same integers on any tier.  Nodes still too large go on
// to the dense probes.
constexpr int kCtaThreads = 256;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kCta2Table = 16384;                      // last level: two-hop multiset <= 8192
constexpr int kCta3Table1 = 4096, kCta3Table2 = 8192;  // level below: <= 2048 and <= 4096
constexpr size_t kCta2Smem = (size_t)kCta2Table * (sizeof(int32_t) + sizeof(unsigned long long)) +
                             (size_t)kCta2Table / 2 * sizeof(uint16_t) + 16;
constexpr size_t kCta3Smem = (size_t)(kCta3Table1 + kCta3Table2) * (sizeof(int32_t) + sizeof(unsigned long long)) +
                             (size_t)(kCta3Table1 + kCta3Table2) / 2 * sizeof(uint16_t) + 16;

// the block's total of v, in every thread
__device__ __forceinline__ unsigned long long block_total(unsigned long long v, unsigned long long* red,
                                                          unsigned long long* out) {
    const unsigned long long r = block_sum(v, red);
    if (threadIdx.x == 0) *out = r;
    __syncthreads();
    const unsigned long long t = *out;
    __syncthreads();
    return t;
}

// frees a block's table for its next node (all threads)
template <int kT>
__device__ void block_release(SlotTable<kT>& tb) {
    __syncthreads();
    tb.reset(threadIdx.x, kCtaThreads);
    __syncthreads();
    if (threadIdx.x == 0) *tb.n = 0u;
    __syncthreads();
}

// H_2 of node q over its two-hop neighbourhood into the block's table (all threads call
// it; the table is free on entry).  Returns false, with the table untouched, when din(q) is
// 0 or the two-hop multiset exceeds half the slots.
template <int kT>
__device__ bool cta_two_hop(int32_t q, const uint32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const unsigned long long* __restrict__ magic, SlotTable<kT>& tb, PushScratch* sc,
                            unsigned long long* red, unsigned long long* bc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t kb = rp[q], ke = rp[q + 1];
    const uint32_t dk = ke - kb;
    unsigned long long e1 = 0;
    for (uint32_t p = kb + threadIdx.x; p < ke; p += kCtaThreads) e1 += rp[col[p] + 1] - rp[col[p]];
    e1 = block_total(e1, red, bc);
    if (dk == 0 || e1 > (unsigned long long)(kT / 2)) return false;
    const unsigned long long x0 = floor_div_magic(kTwoHopOne, dk, magic[q]);
    for (uint32_t base = kb + (uint32_t)wid * 32; base < ke; base += kCtaWarps * 32) {  // warp-uniform
        const uint32_t p = base + (uint32_t)lane;
        push_batch(p < ke ? col[p] : -1, x0, rp, col, magic, tb, sc[wid]);
    }
    __syncthreads();
    return true;
}

// g_2 of the warp kernel's oversized nodes (list in_ids/in_pos, count *nin); the ones
// still too large are appended to out_ids/out_pos.
__global__ void __launch_bounds__(kCtaThreads) probe_g2_cta_kernel(const unsigned int* __restrict__ nin,
                                                                   const int32_t* __restrict__ in_ids,
                                                                   const int32_t* __restrict__ in_pos,
                                                                   const uint32_t* __restrict__ rp,
                                                                   const int32_t* __restrict__ col,
                                                                   const unsigned long long* __restrict__ magic,
                                                                   unsigned long long* __restrict__ colsum,
                                                                   int32_t* __restrict__ out_ids,
                                                                   int32_t* __restrict__ out_pos,
                                                                   unsigned int* __restrict__ nout) {
    extern __shared__ __align__(16) unsigned char cta_smem[];
    SlotTable<kCta2Table> tb;
    tb.V = (unsigned long long*)cta_smem;
    tb.K = (int32_t*)(tb.V + kCta2Table);
    tb.U = (uint16_t*)(tb.K + kCta2Table);
    tb.n = (unsigned int*)(((uintptr_t)(tb.U + kCta2Table / 2) + 7) & ~(uintptr_t)7);
    __shared__ unsigned long long red[kCtaWarps];
    __shared__ unsigned long long bc;
    __shared__ PushScratch sc[kCtaWarps];
    const unsigned int count = *nin;
    if (blockIdx.x >= count) return;
    tb.clear_all(threadIdx.x, kCtaThreads);
    __syncthreads();
    for (unsigned int i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t q = in_ids[i];
        if (!cta_two_hop<kCta2Table>(q, rp, col, magic, tb, sc, red, &bc)) {
            if (threadIdx.x == 0) {
                const unsigned int slot = atomicAdd(nout, 1u);
                out_ids[slot] = q;
                out_pos[slot] = in_pos[i];
            }
            continue;
        }
        unsigned long long sq = tb.sq_part(threadIdx.x, kCtaThreads);
        sq = block_sum(sq, red);
        if (threadIdx.x == 0) colsum[in_pos[i]] = sq;
        block_release(tb);
    }
}

// the row terms and g_3 of the g_3 warp kernel's oversized nodes (as probe_g3_kernel)
__global__ void __launch_bounds__(kCtaThreads) probe_g3_cta_kernel(const unsigned int* __restrict__ nin,
                                                                   const int32_t* __restrict__ in_ids,
                                                                   const int32_t* __restrict__ in_pos,
                                                                   const uint32_t* __restrict__ rp,
                                                                   const int32_t* __restrict__ col,
                                                                   const unsigned long long* __restrict__ magic,
                                                                   const double* __restrict__ zv_src, double c2,
                                                                   long long* __restrict__ zhi_next,
                                                                   long long* __restrict__ zlo_next,
                                                                   unsigned long long* __restrict__ colsum,
                                                                   int32_t* __restrict__ out_ids,
                                                                   int32_t* __restrict__ out_pos,
                                                                   unsigned int* __restrict__ nout) {
    extern __shared__ __align__(16) unsigned char cta_smem[];
    SlotTable<kCta3Table1> t1;
    SlotTable<kCta3Table2> t2;
    carve_tables(cta_smem, t1, t2);
    __shared__ unsigned long long red[kCtaWarps];
    __shared__ unsigned long long bc;
    __shared__ PushScratch sc[kCtaWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned int count = *nin;
    if (blockIdx.x >= count) return;
    t1.clear_all(threadIdx.x, kCtaThreads);
    t2.clear_all(threadIdx.x, kCtaThreads);
    __syncthreads();
    for (unsigned int i = blockIdx.x; i < count; i += gridDim.x) {
        const int32_t q = in_ids[i];
        const bool built = cta_two_hop<kCta3Table1>(q, rp, col, magic, t1, sc, red, &bc);
        bool fits = built;
        if (built) {
            const unsigned int cnt = *t1.n;
            unsigned long long e2 = 0;
            for (unsigned int u = threadIdx.x; u < cnt; u += kCtaThreads) {
                const int32_t a = t1.K[t1.U[u]];
                e2 += rp[a + 1] - rp[a];
            }
            e2 = block_total(e2, red, &bc);
            fits = e2 <= (unsigned long long)(kCta3Table2 / 2);
        }
        if (!fits) {
            if (built) block_release(t1);
            if (threadIdx.x == 0) {
                const unsigned int slot = atomicAdd(nout, 1u);
                out_ids[slot] = q;
                out_pos[slot] = in_pos[i];
            }
            continue;
        }
        const double coef = c2 * zv_src[q];
        const unsigned int cnt1 = *t1.n;
        for (unsigned int u = threadIdx.x; u < cnt1; u += kCtaThreads) {
            const int slot = t1.U[u];
            const double h = (double)t1.V[slot] * kInvOne;
            long long hi, lo;
            zacc_split(coef * (h * h), hi, lo);
            if (hi != 0) atomicAdd((unsigned long long*)(zhi_next + t1.K[slot]), (unsigned long long)(-hi));
            if (lo != 0) atomicAdd((unsigned long long*)(zlo_next + t1.K[slot]), (unsigned long long)(-lo));
        }
        // third step: warps take 32-entry chunks of the two-hop list (warp-uniform bounds)
        for (unsigned int i0 = (unsigned int)wid * 32; i0 < cnt1; i0 += kCtaWarps * 32) {
            const unsigned int u = i0 + (unsigned int)lane;
            const int slot = u < cnt1 ? (int)t1.U[u] : -1;
            push_batch(slot >= 0 ? t1.K[slot] : -1, slot >= 0 ? t1.V[slot] : 0ull, rp, col, magic, t2, sc[wid]);
        }
        __syncthreads();
        unsigned long long sq = t2.sq_part(threadIdx.x, kCtaThreads);
        sq = block_sum(sq, red);
        if (threadIdx.x == 0) colsum[in_pos[i]] = sq;
        block_release(t2);
        block_release(t1);
    }
}

// *zlast += sum_i (cl Zv(ids[i])) (colsum[i] 2^-63), i < count, in a fixed order: thread t
// takes i = t, t + 1024, ... and a fixed tree adds the threads' partials.
__global__ void __launch_bounds__(1024) probe_g2_total_kernel(const uint64_t* __restrict__ count_dev,
                                                              const int32_t* __restrict__ ids,
                                                              const double* __restrict__ zv_src, double cl,
                                                              const unsigned long long* __restrict__ colsum,
                                                              double* __restrict__ zlast) {
    __shared__ double red[1024];
    const int64_t count = (int64_t)*count_dev;
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += 1024) t += (cl * zv_src[ids[i]]) * ((double)colsum[i] * kInvOne);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *zlast += red[0];
}

// D^ of Algorithm 3 for exploited nodes (depth > 0), of Algorithm 2 for the others,
// and the exact values at din <= 1 (Algorithm 3's first cases).
__global__ void dhat_alg3_kernel(int64_t n, const uint64_t* __restrict__ counts, const uint64_t* __restrict__ off,
                                 const uint8_t* __restrict__ depth, const double* __restrict__ zsum,
                                 const uint32_t* __restrict__ in_rp, double c, double* __restrict__ dhat) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t R = off[k + 1] - off[k];
        const double ratio = R ? (double)counts[k] / (double)R : 0.0;
        double d = ratio;
        const unsigned dk = depth[k];
        if (dk) {
            double cd = 1.0;
            for (unsigned i = 0; i < dk; ++i) cd *= c;
            d = 1.0 - zsum[k] - cd * ratio;
        }
        const uint32_t din = in_rp[k + 1] - in_rp[k];
        if (din == 0) d = 1.0;
        else if (din == 1) d = 1.0 - c;
        dhat[k] = d;
    }
}

int eblocks(const Graph& g, int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    if (b > (int64_t)g.sm_count * 8) b = (int64_t)g.sm_count * 8;
    return (int)(b < 1 ? 1 : b);
}

size_t witems_of(int64_t n, int64_t m) { return (size_t)n + (size_t)m / kPushChunk + 64; }

// Bytes of one probe block's slices
size_t probe_block_bytes(int64_t n, int64_t m, int64_t nseg) {
    const size_t nn = (size_t)n;
    return 8 * 3 * kProbeW * nn + 4 * 3 * nn + 2 * 8 * witems_of(n, m) +
           8 * (size_t)kProbeW * (size_t)std::max<int64_t>(nseg, 1) + sizeof(ProbeCtl) + 8 * 2 * kProbeW + 4096;
}

int group_size(int64_t n, int64_t m, int64_t nseg) {
    const size_t per = probe_block_bytes(n, m, nseg);
    const size_t gmax = kProbeBudget / per;
    return (int)std::max<size_t>(1, std::min<size_t>(kGroupMax, gmax));
}

struct A3Ws {
    double* H;        // (D+1) n: h_0 .. h_D from k
    double* Zv;       // (D+1) n: Zv_1 .. Zv_D at rows 1..D (row 0 unused)
    long long* Zfx;   // 2 (D+1) n: fixed-point probe terms per level, hi words then lo words
    double* T;        // n: P~ Zv_{j-1}
    double* x;        // n: sweep input
    double* xa;       // n
    double* xb;       // n
    uint64_t* flag;   // n
    uint64_t* off;    // n + 1
    int32_t* ids;     // n
    uint32_t* Ba;     // reach bit sets (32 nodes per word)
    uint32_t* Bb;
    unsigned long long* rcounts;  // (D + 1) x 32 support sizes
    double* partial;  // kDotBlocks (dot products)
    double* sums;     // 64: [j] = sum_q Zv_j(q); [63] = the last level's probe terms
    unsigned long long* g2;  // n: column sums g_2 of the last probe level, by support position
    int32_t* big_ids;        // n: support nodes too large for the two-hop table
    int32_t* big_pos;        // n: their support positions
    unsigned int* nbig;      // 2: the warp tier's overflow count, then the block tier's
    int32_t* big2_ids;       // n: nodes too large for the block tier too (dense probes)
    int32_t* big2_pos;       // n
    ProbeGroup G;
    int group;        // probe blocks per launch
};

size_t a3_layout(int64_t n_, int64_t m_, int64_t nseg, void* base, A3Ws* out) {
    const size_t n = (size_t)n_;
    const size_t D = (size_t)kAlg3MaxDepth;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? (char*)base + o : nullptr;
        o += (bytes + 255) / 256 * 256;
        return p;
    };
    A3Ws w{};
    w.H = (double*)take(8 * (D + 1) * n);
    w.Zv = (double*)take(8 * (D + 1) * n);
    w.Zfx = (long long*)take(8 * 2 * (D + 1) * n);
    w.T = (double*)take(8 * n);
    w.x = (double*)take(8 * n);
    w.xa = (double*)take(8 * n);
    w.xb = (double*)take(8 * n);
    w.flag = (uint64_t*)take(8 * n);
    w.off = (uint64_t*)take(8 * (n + 1));
    w.ids = (int32_t*)take(4 * n);
    w.Ba = (uint32_t*)take(4 * n);
    w.Bb = (uint32_t*)take(4 * n);
    w.rcounts = (unsigned long long*)take(8 * 32 * (D + 1));
    w.partial = (double*)take(8 * kDotBlocks);
    w.sums = (double*)take(8 * 64);
    w.g2 = (unsigned long long*)take(8 * n);
    w.big_ids = (int32_t*)take(4 * n);
    w.big_pos = (int32_t*)take(4 * n);
    w.nbig = (unsigned int*)take(256);
    w.big2_ids = (int32_t*)take(4 * n);
    w.big2_pos = (int32_t*)take(4 * n);
    const int G = group_size(n_, m_, nseg);
    const size_t gz = (size_t)G;
    w.group = G;
    ProbeGroup& P = w.G;
    P.n = n_;
    P.nx = (size_t)kProbeW * n;
    P.nw = witems_of(n_, m_);
    P.np = (size_t)kProbeW * (size_t)std::max<int64_t>(nseg, 1);
    P.X[0] = (unsigned long long*)take(8 * P.nx * gz);
    P.X[1] = (unsigned long long*)take(8 * P.nx * gz);
    P.Hn = (unsigned long long*)take(8 * P.nx * gz);
    P.mark = (uint32_t*)take(4 * n * gz);
    for (int b = 0; b < 2; ++b) {
        P.F[b] = (int32_t*)take(4 * n * gz);
        P.W[b] = (int2*)take(8 * P.nw * gz);
    }
    P.ppart = (unsigned long long*)take(8 * P.np * gz);
    P.ctl = (ProbeCtl*)take(sizeof(ProbeCtl) * gz);
    P.coef = (double*)take(8 * kProbeW * gz);
    P.colsum = (unsigned long long*)take(8 * kProbeW * gz);
    if (out) *out = w;
    return o;
}

cudaError_t dsum(const Graph& g, const double* a, int kind, const A3Ws& ws, double* out_dev, int* count) {
    wsum_kernel<<<kDotBlocks, kBlock, 0, g.stream>>>(g.n, a, kind, ws.partial);
    sum_partials_kernel<<<1, 1024, 0, g.stream>>>(kDotBlocks, ws.partial, out_dev);
    *count += 2;
    return cudaGetLastError();
}

// One probe step for a group of nb blocks: push, dense pull (whichever the counters
// pick), sparse epilogue.
cudaError_t probe_step(const Graph& g, const A3Ws& ws, const ProbeStepArgs& a, int nb, int* count) {
    const DevCsr& A = g.out;
    const unsigned sparse_blocks = (unsigned)std::max(1, g.sm_count * 4 / nb);
    probe_push_kernel<<<dim3(sparse_blocks, (unsigned)nb), kBlock, 0, g.stream>>>(ws.G, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int wpb = kBlock / 32;
    int64_t sb = (g.n + wpb - 1) / wpb;
    if (sb > (int64_t)g.sm_count * 16) sb = (int64_t)g.sm_count * 16;
    if (sb < 1) sb = 1;
    int64_t segb = A.nseg;  // one block per segment
    if (segb > (int64_t)g.sm_count * 8) segb = (int64_t)g.sm_count * 8;
    probe_rows_kernel<<<dim3((unsigned)(sb + segb), (unsigned)nb), kBlock, 0, g.stream>>>(
        ws.G, a, A.rp, A.col, A.long_min, A.nseg, A.seg, (int)sb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *count += 2;
    if (A.nlong > 0) {
        const int64_t blocks = (A.nlong * 32 + kBlock - 1) / kBlock;
        probe_long_rows_kernel<<<dim3((unsigned)blocks, (unsigned)nb), kBlock, 0, g.stream>>>(ws.G, a, A.nlong,
                                                                                              A.long_rows, A.long_first);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*count;
    }
    probe_sparse_epi_kernel<<<dim3(sparse_blocks, (unsigned)nb), kBlock, 0, g.stream>>>(ws.G, a);
    ++*count;
    return cudaGetLastError();
}

}  // namespace

size_t alg3_workspace_bytes(const Graph& g) { return a3_layout(g.n, g.m, g.out.nseg, nullptr, nullptr); }

cudaError_t alg3_supports(const Graph& g, const int32_t* ks_host, int count, int levels, void* wsp,
                          uint64_t* supp_out, int* launches) {
    A3Ws ws;
    a3_layout(g.n, g.m, g.out.nseg, wsp, &ws);
    const size_t n = (size_t)g.n;
    int nl = 0;
    cudaError_t e = cudaSuccess;
    for (int c0 = 0; c0 < count; c0 += 32) {
        const int cnt = std::min(32, count - c0);
        for (int c = 0; c < cnt; ++c) supp_out[(size_t)(c0 + c) * (kAlg3MaxDepth + 1)] = 1;
        if (levels <= 0) continue;
        if ((e = cudaMemsetAsync(ws.rcounts, 0, 8 * 32 * (size_t)(kAlg3MaxDepth + 1), g.stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(ws.Ba, 0, 4 * n, g.stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ws.ids, ks_host + c0, sizeof(int32_t) * (size_t)cnt, cudaMemcpyHostToDevice,
                                 g.stream)) != cudaSuccess)
            return e;
        reach_init_kernel<<<1, 32, 0, g.stream>>>(ws.ids, cnt, ws.Ba);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++nl;
        uint32_t* B[2] = {ws.Ba, ws.Bb};
        int64_t blocks = (g.n + kBlock / 32 - 1) / (kBlock / 32);
        if (blocks > (int64_t)g.sm_count * 16) blocks = (int64_t)g.sm_count * 16;
        for (int l = 1; l <= levels; ++l) {
            reach_step_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(g.n, g.out.rp, g.out.col, B[(l - 1) & 1],
                                                                         B[l & 1], ws.rcounts + (size_t)l * 32);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++nl;
        }
        std::vector<unsigned long long> host((size_t)32 * (kAlg3MaxDepth + 1));
        if ((e = cudaMemcpyAsync(host.data(), ws.rcounts, 8 * host.size(), cudaMemcpyDeviceToHost, g.stream)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
        for (int c = 0; c < cnt; ++c)
            for (int l = 1; l <= levels; ++l)
                supp_out[(size_t)(c0 + c) * (kAlg3MaxDepth + 1) + l] = host[(size_t)l * 32 + c];
    }
    if (launches) *launches += nl;
    return cudaSuccess;
}

cudaError_t alg3_first_meeting(const Graph& g, int64_t k, int depth, double c, void* wsp, double* z_out, int* launches) {
    A3Ws ws;
    a3_layout(g.n, g.m, g.out.nseg, wsp, &ws);
    const size_t n = (size_t)g.n;
    const int per_sweep = 1 + (g.out.tnlong > 0 ? 1 : 0);  // tile kernel, long rows
    const int eb = eblocks(g, g.n);
    int count = 0;
    cudaError_t e = launch_walk_distributions(g, k, depth, ws.H, ws.xa, ws.xb);
    if (e != cudaSuccess) return e;
    count += 1 + depth * per_sweep;
    long long* const zlo_base = ws.Zfx + (size_t)(kAlg3MaxDepth + 1) * n;
    if ((e = cudaMemsetAsync(ws.Zfx, 0, sizeof(long long) * n * (size_t)(depth + 1), g.stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(zlo_base, 0, sizeof(long long) * n * (size_t)(depth + 1), g.stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(ws.sums, 0, sizeof(double) * 64, g.stream)) != cudaSuccess) return e;
    int cleared = 0;  // probe blocks made zero so far (each group leaves its blocks zero)
    std::vector<double> cpow((size_t)depth + 1, 1.0);
    for (int j = 1; j <= depth; ++j) cpow[(size_t)j] = cpow[(size_t)j - 1] * c;
    const unsigned long long thr = (unsigned long long)(g.m + g.n) / (unsigned long long)std::max(1, g.alg3_push_div);
    for (int j = 1; j <= depth; ++j) {
        double* zv = ws.Zv + (size_t)j * n;
        const double* T = nullptr;
        if (j >= 2) {  // T = P~ Zv_{j-1}
            float2* x2 = reinterpret_cast<float2*>(ws.x);  // n 8-byte entries
            sq_scale_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.Zv + (size_t)(j - 1) * n, g.inv_din, x2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = launch_pull_sum(g, x2, ws.T)) != cudaSuccess) return e;
            count += 1 + per_sweep;
            T = ws.T;
        }
        zv_finalize_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, cpow[(size_t)j], c, ws.H + (size_t)j * n, T,
                                                        ws.Zfx + (size_t)j * n, zlo_base + (size_t)j * n, zv);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++count;
        if ((e = dsum(g, zv, 2, ws, ws.sums + j, &count)) != cudaSuccess) return e;
        // probes from the support of h_j feed the levels j+2 .. depth: the row terms of a
        // level below depth, only the column sums for the last level
        if (j > depth - 2) continue;
        flag_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.H + (size_t)j * n, ws.flag);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_scan_R(g, g.n, ws.flag, ws.off, g.scan_part, nullptr, g.norm_part + allocate_blocks(g.n),
                               false)) != cudaSuccess)
            return e;
        scatter_ids_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.flag, ws.off, ws.ids);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count += 5;
        const int steps = depth - j;
        // the last two probe levels run one warp per node where its neighbourhood fits the
        // tables: g_2 for the last, the row terms and g_3 for the one below it
        const bool hashed = steps == 2 || steps == 3;
        if (hashed) {
            if ((e = cudaMemsetAsync(ws.nbig, 0, 2 * sizeof(unsigned int), g.stream)) != cudaSuccess) return e;
            if (steps == 2) {
                probe_g2_kernel<<<(unsigned)(g.sm_count * 5), kG2Warps * 32, 0, g.stream>>>(
                    ws.off + n, ws.ids, g.in.rp, g.in.col, g.din_magic, ws.g2, ws.big_ids, ws.big_pos, ws.nbig);
            } else {
                if ((e = cudaFuncSetAttribute(probe_g3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kG3Smem)) != cudaSuccess)
                    return e;
                probe_g3_kernel<<<(unsigned)(g.sm_count * 2), kG3Warps * 32, kG3Smem, g.stream>>>(
                    ws.off + n, ws.ids, g.in.rp, g.in.col, g.din_magic, zv, cpow[2], ws.Zfx + (size_t)(j + 2) * n,
                    zlo_base + (size_t)(j + 2) * n, ws.g2, ws.big_ids, ws.big_pos, ws.nbig);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            // the block tier takes the warp tier's overflow
            if (steps == 2) {
                if ((e = cudaFuncSetAttribute(probe_g2_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCta2Smem)) != cudaSuccess)
                    return e;
                probe_g2_cta_kernel<<<(unsigned)g.sm_count, kCtaThreads, kCta2Smem, g.stream>>>(
                    ws.nbig, ws.big_ids, ws.big_pos, g.in.rp, g.in.col, g.din_magic, ws.g2, ws.big2_ids, ws.big2_pos,
                    ws.nbig + 1);
            } else {
                if ((e = cudaFuncSetAttribute(probe_g3_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kCta3Smem)) != cudaSuccess)
                    return e;
                probe_g3_cta_kernel<<<(unsigned)g.sm_count, kCtaThreads, kCta3Smem, g.stream>>>(
                    ws.nbig, ws.big_ids, ws.big_pos, g.in.rp, g.in.col, g.din_magic, zv, cpow[2],
                    ws.Zfx + (size_t)(j + 2) * n, zlo_base + (size_t)(j + 2) * n, ws.g2, ws.big2_ids, ws.big2_pos,
                    ws.nbig + 1);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            count += 2;
        }
        uint64_t nsup = 0;
        unsigned int nbig = 0;
        if ((e = cudaMemcpyAsync(&nsup, ws.off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, g.stream)) != cudaSuccess)
            return e;
        if (hashed && (e = cudaMemcpyAsync(&nbig, ws.nbig + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                           g.stream)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
        // dense probes: every support node of the deeper levels, the large ones of the last two
        const uint64_t nprobe = hashed ? (uint64_t)nbig : nsup;
        const int32_t* probe_ids = hashed ? ws.big2_ids : ws.ids;
        const uint64_t per_group = (uint64_t)kProbeW * (uint64_t)ws.group;
        const int need_blocks = (int)std::min<uint64_t>((uint64_t)ws.group, (nprobe + kProbeW - 1) / kProbeW);
        if (need_blocks > cleared) {  // blocks [cleared, need_blocks) of each buffer
            const size_t b0 = (size_t)cleared, nbk = (size_t)(need_blocks - cleared);
            if ((e = cudaMemsetAsync(ws.G.X[0] + b0 * ws.G.nx, 0, 8 * ws.G.nx * nbk, g.stream)) != cudaSuccess ||
                (e = cudaMemsetAsync(ws.G.X[1] + b0 * ws.G.nx, 0, 8 * ws.G.nx * nbk, g.stream)) != cudaSuccess ||
                (e = cudaMemsetAsync(ws.G.Hn + b0 * ws.G.nx, 0, 8 * ws.G.nx * nbk, g.stream)) != cudaSuccess ||
                (e = cudaMemsetAsync(ws.G.mark + b0 * n, 0, 4 * n * nbk, g.stream)) != cudaSuccess)
                return e;
            cleared = need_blocks;
        }
        for (uint64_t g0 = 0; g0 < nprobe; g0 += per_group) {
            const int cnt = (int)std::min<uint64_t>(per_group, nprobe - g0);
            const int nb = (cnt + kProbeW - 1) / kProbeW;
            const int32_t* ids = probe_ids + g0;
            probe_init_kernel<<<dim3(1, (unsigned)nb), kProbeW, 0, g.stream>>>(ws.G, ids, cnt, g.in.rp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++count;
            for (int lp = 1; lp <= steps; ++lp) {
                ProbeStepArgs a{g.in.rp, g.in.col, g.din_magic, lp - 1, (lp - 1) & 1, 0, lp == steps ? 1 : 0,
                                ws.Zfx + (size_t)(j + lp) * n, zlo_base + (size_t)(j + lp) * n, thr};
                if (lp == steps) {
                    a.mode = 2;
                } else if (lp >= 2) {
                    probe_coef_kernel<<<dim3(1, (unsigned)nb), kProbeW, 0, g.stream>>>(ws.G, ids, cnt, zv,
                                                                                       cpow[(size_t)lp]);
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                    ++count;
                    a.mode = 1;
                }
                if ((e = probe_step(g, ws, a, nb, &count)) != cudaSuccess) return e;
            }
            probe_end_kernel<<<dim3((unsigned)g.sm_count, (unsigned)nb), kBlock, 0, g.stream>>>(
                ws.G, ids, cnt, zv, cpow[(size_t)steps], ws.sums + 63, hashed ? ws.big2_pos + g0 : nullptr,
                hashed ? ws.g2 : nullptr);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++count;
        }
        if (hashed && nsup > 0) {
            probe_g2_total_kernel<<<1, 1024, 0, g.stream>>>(ws.off + n, ws.ids, zv, cpow[(size_t)steps], ws.g2,
                                                            ws.sums + 63);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++count;
        }
    }
    double sums[64] = {};
    if ((e = cudaMemcpyAsync(sums, ws.sums, sizeof(sums), cudaMemcpyDeviceToHost, g.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
    for (int j = 1; j <= depth; ++j) z_out[j - 1] = sums[j];
    z_out[depth - 1] -= sums[63];  // the last level's probe terms, kept as column sums
    if (launches) *launches += count;
    return cudaSuccess;
}

cudaError_t launch_dhat_alg3(const Graph& g, const uint64_t* counts, const uint64_t* off, const uint8_t* depth,
                             const double* zsum, double c, double* dhat) {
    dhat_alg3_kernel<<<eblocks(g, g.n), kBlock, 0, g.stream>>>(g.n, counts, off, depth, zsum, g.in.rp, c, dhat);
    return cudaGetLastError();
}

}  // namespace esim
