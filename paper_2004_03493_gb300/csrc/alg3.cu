// Algorithm 3 ("Improved method for estimating D(k,k)"): exact first-meeting
// probabilities Z_1..Z_d of node k by Lemma 5, for any depth d <= kAlg3MaxDepth,
// and the diagonal estimate that combines them with the tail walk pairs.
//
// Notation: h_l = (P^T)^l(k, .), the distribution of a non-stop walk from k after l
// steps (dense FP64, by pull sweeps over the out-edge CSR with no decay); Zv_l the
// vector Z_l(k, .) of Lemma 5; P~ the transition matrix with squared entries.
// Lemma 5 reads, for each target level j,
//   Zv_j = c^j h_j^2 - c P~ Zv_{j-1} - sum_{l'=2}^{j-1} c^{l'} sum_{q'} Zv_{j-l'}(q') ((P^T)^{l'}(q', .))^2
// (the l' = 1 term is one squared-weight sweep, because (P^T)(q', q)^2 = 1/din(q')^2
// for q in I(q')).  The l' >= 2 terms need the walk distributions of every q' in
// the support of h_{j-l'}: the "probes".  Probes run 32 at a time as an n x 32 FP64
// block through a multi-column pull product whose epilogue subtracts
// sum_col c^{l'} Zv_i(q'_col) h^{q'_col}_{l'}(q)^2 from Zv_{i+l'}(q) (a fixed lane tree;
// blocks of 32 consecutive q' of the ascending support, in order).  Z_j = sum_q Zv_j(q)
// by fixed-order block partials.  Everything is deterministic.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <algorithm>
#include <vector>

namespace esim {

namespace {

constexpr int kDotBlocks = 1024;
constexpr int kProbeW = 32;  // probe columns per block (one warp lane each)

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

// x = v / din^2: the input of the squared-transition sweep P~ v
__global__ void sq_scale_kernel(int64_t n, const double* __restrict__ v, const double* __restrict__ inv_din,
                                double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = inv_din[i];
        x[i] = v[i] * (w * w);
    }
}

// Zv_j = c^j h_j^2 - c T + Zv_j, where Zv_j already holds the (negative) probe terms
// and T = P~ Zv_{j-1} (T = NULL at j = 1)
__global__ void zv_finalize_kernel(int64_t n, double cj, double c, const double* __restrict__ h,
                                   const double* __restrict__ T, double* __restrict__ zv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double hv = h[i];
        double z = cj * (hv * hv);
        if (T) z -= c * T[i];
        zv[i] = z + zv[i];
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

// floor(H^2 / 2^63) for H <= 2^63
__device__ __forceinline__ unsigned long long fx_sq(unsigned long long H) {
    return (__umul64hi(H, H) << 1) | ((H * H) >> 63);
}

// Probe block start: x_0 = e_{q'} / din(q') in column col (row-major n x 32, zeroed before)
__global__ void probe_init_kernel(const int32_t* __restrict__ ids, int count, const uint32_t* __restrict__ in_rp,
                                  unsigned long long* __restrict__ X) {
    const int col = threadIdx.x;
    if (col < count) {
        const int32_t q = ids[col];
        const uint32_t d = in_rp[q + 1] - in_rp[q];
        X[(size_t)q * kProbeW + col] = d ? kOne / d : 0ull;
    }
}

// coef(col) = c^{l'} Zv_i(q'_col); 0 for unused columns
__global__ void probe_coef_kernel(const int32_t* __restrict__ ids, int count, const double* __restrict__ zv_src,
                                  double cl, double* __restrict__ coef) {
    const int col = threadIdx.x;
    if (col < kProbeW) coef[col] = col < count ? cl * zv_src[ids[col]] : 0.0;
}

// zlast += sum_col coef(col) * colsum(col) (columns in order); colsum reset for the next block
__global__ void probe_norm_finish_kernel(const double* __restrict__ coef, unsigned long long* __restrict__ colsum,
                                         double* __restrict__ zlast) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int col = 0; col < kProbeW; ++col) t += coef[col] * ((double)colsum[col] * kInvOne);
        *zlast += t;
    }
    __syncthreads();
    if (threadIdx.x < kProbeW) colsum[threadIdx.x] = 0ull;
}

struct ProbeEpi {
    const uint32_t* in_rp;
    unsigned long long* x_next;  // n x 32: h / din for the next step
    int mode;                    // 0: none; 1: subtract sum_col coef h^2 from zacc(row); 2: column sums of h^2
    const double* coef;          // 32 (mode 1)
    double* zacc;                // n: Zv of the target level (mode 1)
    unsigned long long* colsum;  // 32 (mode 2)
};

// Row `row` of h^{q'}_{l'} is H (fixed point) in lane = column.  All 32 lanes of the
// warp call it.  Returns this lane's h^2 (fixed point) for mode 2, else 0.  The FP64
// row term of mode 1 is a fixed butterfly over the lanes, skipped when the row is zero.
__device__ __forceinline__ unsigned long long probe_epilogue(int64_t row, unsigned long long H, int lane,
                                                             const ProbeEpi& e) {
    const uint32_t d = __ldg(e.in_rp + row + 1) - __ldg(e.in_rp + row);
    e.x_next[(size_t)row * kProbeW + lane] = (d && H) ? H / d : 0ull;
    if (e.mode == 2) return fx_sq(H);
    if (e.mode == 1 && __any_sync(0xffffffffu, H != 0ull)) {
        const double h = (double)H * kInvOne;
        double t = e.coef[lane] * (h * h);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) e.zacc[row] = e.zacc[row] - t;
    }
    return 0ull;
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

// Column sums of mode 2: lane sums of the block's warps, then one integer atomic per
// column (integer addition is order-free, so the result is exact and deterministic).
__device__ __forceinline__ void probe_flush_colsum(unsigned long long v, const ProbeEpi& e) {
    constexpr int kWarps = kBlock / 32;
    __shared__ unsigned long long red[kWarps][kProbeW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    red[wib][lane] = v;
    __syncthreads();
    if (wib == 0) {
        unsigned long long t = 0ull;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += red[w][lane];
        if (t) atomicAdd(e.colsum + lane, t);
    }
}

// ---- direction-optimising probe steps
//
// A probe block starts from 32 single nodes, so its first steps touch few rows.
// While the frontier F_s (the rows of x_s that may be non-zero) has few in-edges,
// a step pushes x_s(j) to the rows i in I(j) with integer atomics into an n x 32
// accumulator (exact, so the order of the atomics does not matter) and processes
// only the touched rows; once the frontier's in-edges exceed (m + n) / 4 the step
// and all later ones of the block run the dense pull above.  Both forms give the
// same integers, so the switch changes no bit of the result.  The frontier, its
// in-edge count and the work list of 64-entry chunks live on the device; the
// kernels of a step read the same counters, so all agree on the form without a
// host round trip.
constexpr int kPushChunk = 64;

struct ProbeStepCnt {
    unsigned int fcount;      // rows in F_s
    unsigned int wcount;      // push work items of F_s (64-entry chunks of in-rows)
    unsigned long long push;  // in-edges of F_s
};

struct ProbeCtl {
    ProbeStepCnt st[kAlg3MaxDepth + 2];
    int dense_plus1;  // 0: sparse so far; s + 1: dense from step s on
};

__device__ __forceinline__ bool probe_dense_at(const ProbeCtl* ctl, int s, unsigned long long thr) {
    const int d = *(volatile const int*)&ctl->dense_plus1;
    return (d != 0 && d - 1 <= s) || ctl->st[s].push > thr;
}

struct ProbePush {
    const uint32_t* in_rp;
    const int32_t* in_col;
    const unsigned long long* X;  // x_s (rows of F_s)
    unsigned long long* Hn;       // accumulator of h_{s+1}, zero outside the step
    uint32_t* mark;               // rows already in F_{s+1}
    const int2* W;                // work items of F_s
    int32_t* Fnext;               // F_{s+1}
    ProbeCtl* ctl;
    int s;
    unsigned long long thr;
};

// One warp per work item (row j, chunk): every entry i of the chunk receives x_s(j)
// in all 32 columns; each lane marks one entry's row and the new rows are appended
// to F_{s+1} with one atomic per warp.
__global__ void __launch_bounds__(kBlock) probe_push_kernel(ProbePush a) {
    if (probe_dense_at(a.ctl, a.s, a.thr)) return;
    const int lane = threadIdx.x & 31;
    const unsigned int items = a.ctl->st[a.s].wcount;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (int64_t)items; w += nwarps) {
        const int2 it = a.W[w];
        const int32_t j = it.x;
        const unsigned long long xv = a.X[(size_t)j * kProbeW + lane];
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
                fresh = atomicExch(a.mark + mine, 1u) == 0u;
                if (fresh) din_new = __ldg(a.in_rp + mine + 1) - __ldg(a.in_rp + mine);
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            unsigned int base = 0;
            if (fm) {
                unsigned long long dsum = din_new;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                if (lane == 0) {
                    base = atomicAdd(&a.ctl->st[a.s + 1].fcount, (unsigned int)__popc(fm));
                    atomicAdd(&a.ctl->st[a.s + 1].push, dsum);
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                if (fresh) a.Fnext[base + __popc(fm & ((1u << lane) - 1u))] = mine;
            }
            const int cnt = (int)(end - p0 < 32 ? end - p0 : 32);  // warp-uniform
            for (int t = 0; t < cnt; ++t) {
                const int32_t i = __shfl_sync(0xffffffffu, mine, t);
                if (xv) atomicAdd(a.Hn + (size_t)i * kProbeW + lane, xv);
            }
        }
    }
}

struct ProbeSparseEpi {
    const uint32_t* in_rp;
    unsigned long long* Hn;
    uint32_t* mark;
    const int32_t* Fnext;        // F_{s+1}
    const int32_t* Fcur;         // F_s: its x_s rows are cleared
    unsigned long long* Xcur;    // x_s
    int2* Wnext;                 // work items of F_{s+1}
    ProbeCtl* ctl;
    int s;
    int last;                    // no further step: x_{s+1} and its work items are not needed
    unsigned long long thr;
};

// The rows of F_{s+1}: h_{s+1} from the accumulator (which is cleared), x_{s+1},
// the epilogue terms, and the next step's work items; then x_s is cleared on F_s.
__global__ void __launch_bounds__(kBlock) probe_sparse_epi_kernel(ProbeSparseEpi a, ProbeEpi epi) {
    if (probe_dense_at(a.ctl, a.s, a.thr)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned int nf = a.ctl->st[a.s + 1].fcount;
    unsigned long long nacc = 0ull;
    for (int64_t r = w0; r < (int64_t)nf; r += nwarps) {
        const int32_t i = a.Fnext[r];
        const size_t at = (size_t)i * kProbeW + lane;
        const unsigned long long H = a.Hn[at];
        a.Hn[at] = 0ull;
        const uint32_t d = __ldg(a.in_rp + i + 1) - __ldg(a.in_rp + i);
        if (lane == 0) {
            a.mark[i] = 0u;
            if (!a.last && d) {
                const unsigned int nch = (d + kPushChunk - 1) / kPushChunk;
                const unsigned int base = atomicAdd(&a.ctl->st[a.s + 1].wcount, nch);
                for (unsigned int ch = 0; ch < nch; ++ch) a.Wnext[base + ch] = make_int2(i, (int)ch);
            }
        }
        if (a.last) {
            if (epi.mode == 2) nacc += fx_sq(H);
        } else {
            nacc += probe_epilogue(i, H, lane, epi);
        }
    }
    const unsigned int nc = a.ctl->st[a.s].fcount;
    for (int64_t r = w0; r < (int64_t)nc; r += nwarps) a.Xcur[(size_t)a.Fcur[r] * kProbeW + lane] = 0ull;
    if (epi.mode == 2) probe_flush_colsum(nacc, epi);
}

// Block start: x_0 = e_{q'} / din(q') per column, F_0 = the sources, their work items.
__global__ void probe_sparse_init_kernel(const int32_t* __restrict__ ids, int count, const uint32_t* __restrict__ in_rp,
                                         unsigned long long* __restrict__ X, int32_t* __restrict__ F, int2* __restrict__ W,
                                         ProbeCtl* __restrict__ ctl) {
    const int lane = threadIdx.x;
    int32_t q = -1;
    uint32_t d = 0;
    if (lane < count) {
        q = ids[lane];
        d = in_rp[q + 1] - in_rp[q];
        X[(size_t)q * kProbeW + lane] = d ? kOne / d : 0ull;
        F[lane] = q;
    }
    const unsigned int nch = (d + kPushChunk - 1) / kPushChunk;
    unsigned int incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned int base = incl - nch;
    for (unsigned int ch = 0; ch < nch; ++ch) W[base + ch] = make_int2(q, (int)ch);
    unsigned long long dsum = d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {
        ctl->st[0].fcount = (unsigned int)(count < 32 ? count : 32);
        ctl->st[0].wcount = total;
        ctl->st[0].push = dsum;
    }
}

// After a block that went dense: both x buffers are cleared for the next block.
__global__ void probe_cleanup_kernel(const ProbeCtl* __restrict__ ctl, unsigned long long* __restrict__ Xa,
                                     unsigned long long* __restrict__ Xb, size_t words) {
    if (ctl->dense_plus1 == 0) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        Xa[i] = 0ull;
        Xb[i] = 0ull;
    }
}

// One probe step: h(i, col) = sum_{j in Out(i)} X(j, col), a pull over the out-edge
// CSR for 32 columns at once.  Short rows: one warp per row, lane = column.  Long
// rows: one block per 4096-entry segment, each warp adding a contiguous eighth of it
// into the segment's partial; probe_long_rows_kernel adds a row's partials.
__global__ void __launch_bounds__(kBlock) probe_rows_kernel(int64_t n, const uint32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const unsigned long long* __restrict__ X,
                                                            uint32_t long_min, int64_t nseg,
                                                            const Segment* __restrict__ seg,
                                                            unsigned long long* __restrict__ partial, int short_blocks,
                                                            ProbeEpi epi, ProbeCtl* ctl, int step,
                                                            unsigned long long thr) {
    constexpr int kWarps = kBlock / 32;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if (ctl) {
        if (!probe_dense_at(ctl, step, thr)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&ctl->dense_plus1, 0, step + 1);
    }
    if ((int)blockIdx.x >= short_blocks) {
        __shared__ unsigned long long red[kWarps][kProbeW];
        const int64_t nsb = (int64_t)gridDim.x - short_blocks;
        for (int64_t s = (int64_t)blockIdx.x - short_blocks; s < nseg; s += nsb) {  // uniform per block
            const Segment sg = seg[s];
            const uint32_t per = (sg.end - sg.beg + kWarps - 1) / kWarps;
            uint32_t b = sg.beg + (uint32_t)wib * per;
            if (b > sg.end) b = sg.end;
            const uint32_t e = b + per < sg.end ? b + per : sg.end;
            red[wib][lane] = probe_range(col, X, b, e, lane);
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
    unsigned long long nacc = 0ull;
    const int64_t nw = (int64_t)short_blocks * kWarps;
    for (int64_t row = (int64_t)blockIdx.x * kWarps + wib; row < n; row += nw) {
        const uint32_t b = __ldg(rp + row), e = __ldg(rp + row + 1);
        if (e - b >= long_min) continue;  // warp-uniform: a long row
        nacc += probe_epilogue(row, probe_range(col, X, b, e, lane), lane, epi);
    }
    if (epi.mode == 2) probe_flush_colsum(nacc, epi);
}

__global__ void __launch_bounds__(kBlock) probe_long_rows_kernel(int64_t nlong, const int32_t* __restrict__ long_rows,
                                                                 const int32_t* __restrict__ long_first,
                                                                 const unsigned long long* __restrict__ partial,
                                                                 ProbeEpi epi, const ProbeCtl* ctl, int step,
                                                                 unsigned long long thr) {
    if (ctl && !probe_dense_at(ctl, step, thr)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned long long nacc = 0ull;
    if (w < nlong) {  // warp-uniform
        unsigned long long acc = 0ull;
        for (int32_t s = long_first[w]; s < long_first[w + 1]; ++s) acc += partial[(size_t)s * kProbeW + lane];
        nacc = probe_epilogue(long_rows[w], acc, lane, epi);
    }
    if (epi.mode == 2) probe_flush_colsum(nacc, epi);
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

struct A3Ws {
    double* H;        // (D+1) n: h_0 .. h_D from k
    double* Zv;       // (D+1) n: Zv_1 .. Zv_D at rows 1..D (row 0 unused)
    double* T;        // n: P~ Zv_{j-1}
    double* x;        // n: sweep input
    double* xa;       // n
    double* xb;       // n
    uint64_t* flag;   // n
    uint64_t* off;    // n + 1
    int32_t* ids;     // n
    unsigned long long* Xa;      // 32 n probe block (fixed point)
    unsigned long long* Xb;      // 32 n
    unsigned long long* Hn;      // 32 n push accumulator (zero between steps)
    uint32_t* mark;              // n (zero between steps)
    int32_t* F[2];               // frontiers, n each
    int2* W[2];                  // push work items, n + m/64 + 64 each
    ProbeCtl* ctl;
    uint32_t* Ba;                // reach bit sets (32 nodes per word)
    uint32_t* Bb;
    unsigned long long* rcounts; // (D + 1) x 32 support sizes
    double* partial;             // kDotBlocks (dot products)
    unsigned long long* ppart;   // 32 nseg (probe segment partials)
    double* coef;                // 32
    unsigned long long* colsum;  // 32
    double* sums;                // 64: [j] = sum_q Zv_j(q); [63] = the last level's probe terms
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
    w.T = (double*)take(8 * n);
    w.x = (double*)take(8 * n);
    w.xa = (double*)take(8 * n);
    w.xb = (double*)take(8 * n);
    w.flag = (uint64_t*)take(8 * n);
    w.off = (uint64_t*)take(8 * (n + 1));
    w.ids = (int32_t*)take(4 * n);
    w.Xa = (unsigned long long*)take(8 * kProbeW * n);
    w.Xb = (unsigned long long*)take(8 * kProbeW * n);
    w.Hn = (unsigned long long*)take(8 * kProbeW * n);
    w.mark = (uint32_t*)take(4 * n);
    const size_t witems = n + (size_t)m_ / kPushChunk + 64;
    for (int b = 0; b < 2; ++b) {
        w.F[b] = (int32_t*)take(4 * n);
        w.W[b] = (int2*)take(8 * witems);
    }
    w.ctl = (ProbeCtl*)take(sizeof(ProbeCtl));
    w.Ba = (uint32_t*)take(4 * n);
    w.Bb = (uint32_t*)take(4 * n);
    w.rcounts = (unsigned long long*)take(8 * 32 * (size_t)(kAlg3MaxDepth + 1));
    w.partial = (double*)take(8 * kDotBlocks);
    w.ppart = (unsigned long long*)take(8 * (size_t)kProbeW * (size_t)std::max<int64_t>(nseg, 1));
    w.coef = (double*)take(8 * kProbeW);
    w.colsum = (unsigned long long*)take(8 * kProbeW);
    w.sums = (double*)take(8 * 64);
    if (out) *out = w;
    return o;
}

cudaError_t dsum(const Graph& g, const double* a, int kind, const A3Ws& ws, double* out_dev, int* count) {
    wsum_kernel<<<kDotBlocks, kBlock, 0, g.stream>>>(g.n, a, kind, ws.partial);
    sum_partials_kernel<<<1, 1024, 0, g.stream>>>(kDotBlocks, ws.partial, out_dev);
    *count += 2;
    return cudaGetLastError();
}

// One probe step for the block: X_prev -> h (epilogue: X_next, accumulation).
cudaError_t probe_step(const Graph& g, const unsigned long long* X_prev, const ProbeEpi& epi,
                       unsigned long long* partial, int* count, ProbeCtl* ctl, int step, unsigned long long thr) {
    const DevCsr& A = g.out;
    const int wpb = kBlock / 32;
    int64_t sb = (g.n + wpb - 1) / wpb;
    if (sb > (int64_t)g.sm_count * 16) sb = (int64_t)g.sm_count * 16;
    if (sb < 1) sb = 1;
    int64_t segb = A.nseg;  // one block per segment
    if (segb > (int64_t)g.sm_count * 8) segb = (int64_t)g.sm_count * 8;
    probe_rows_kernel<<<(unsigned)(sb + segb), kBlock, 0, g.stream>>>(g.n, A.rp, A.col, X_prev, A.long_min, A.nseg,
                                                                       A.seg, partial, (int)sb, epi, ctl, step, thr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*count;
    if (A.nlong > 0) {
        const int64_t blocks = (A.nlong * 32 + kBlock - 1) / kBlock;
        probe_long_rows_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(A.nlong, A.long_rows, A.long_first, partial,
                                                                          epi, ctl, step, thr);
        e = cudaGetLastError();
        ++*count;
    }
    return e;
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
    const int per_sweep = 1 + (g.out.nlong > 0 ? 1 : 0);
    const int eb = eblocks(g, g.n);
    int count = 0;
    cudaError_t e = launch_walk_distributions(g, k, depth, ws.H, ws.xa, ws.xb);
    if (e != cudaSuccess) return e;
    count += 1 + depth * per_sweep;
    if ((e = cudaMemsetAsync(ws.Zv, 0, sizeof(double) * n * (size_t)(depth + 1), g.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.sums, 0, sizeof(double) * 64, g.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.colsum, 0, sizeof(unsigned long long) * kProbeW, g.stream)) != cudaSuccess) return e;
    if (depth >= 3) {  // the probe blocks, accumulator and marks start (and each block ends) all zero
        if ((e = cudaMemsetAsync(ws.Xa, 0, sizeof(unsigned long long) * kProbeW * n, g.stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(ws.Xb, 0, sizeof(unsigned long long) * kProbeW * n, g.stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(ws.Hn, 0, sizeof(unsigned long long) * kProbeW * n, g.stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(ws.mark, 0, sizeof(uint32_t) * n, g.stream)) != cudaSuccess)
            return e;
    }
    std::vector<double> cpow((size_t)depth + 1, 1.0);
    for (int j = 1; j <= depth; ++j) cpow[(size_t)j] = cpow[(size_t)j - 1] * c;
    for (int j = 1; j <= depth; ++j) {
        double* zv = ws.Zv + (size_t)j * n;
        const double* T = nullptr;
        if (j >= 2) {  // T = P~ Zv_{j-1}
            sq_scale_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.Zv + (size_t)(j - 1) * n, g.inv_din, ws.x);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = launch_pull_sum(g, ws.x, ws.T)) != cudaSuccess) return e;
            count += 1 + per_sweep;
            T = ws.T;
        }
        zv_finalize_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, cpow[(size_t)j], c, ws.H + (size_t)j * n, T, zv);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++count;
        if ((e = dsum(g, zv, 2, ws, ws.sums + j, &count)) != cudaSuccess) return e;
        // probes from the support of h_j feed the levels j+2 .. depth: the vector Zv of
        // a level below depth, only the sum for the last level
        if (j <= depth - 2) {
            flag_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.H + (size_t)j * n, ws.flag);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = launch_scan_R(g, g.n, ws.flag, ws.off, g.scan_part, nullptr, g.norm_part + allocate_blocks(g.n))) !=
                cudaSuccess)
                return e;
            scatter_ids_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, ws.flag, ws.off, ws.ids);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            count += 5;
            uint64_t nsup = 0;
            if ((e = cudaMemcpyAsync(&nsup, ws.off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, g.stream)) !=
                cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
            const int steps = depth - j;
            const unsigned long long thr = (unsigned long long)(g.m + g.n) / 4;
            const unsigned sparse_blocks = (unsigned)g.sm_count * 4;
            for (uint64_t b0 = 0; b0 < nsup; b0 += kProbeW) {
                const int cnt = (int)std::min<uint64_t>(kProbeW, nsup - b0);
                const int32_t* ids = ws.ids + b0;
                if ((e = cudaMemsetAsync(ws.ctl, 0, sizeof(ProbeCtl), g.stream)) != cudaSuccess) return e;
                probe_sparse_init_kernel<<<1, kProbeW, 0, g.stream>>>(ids, cnt, g.in.rp, ws.Xa, ws.F[0], ws.W[0], ws.ctl);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                ++count;
                unsigned long long* X[2] = {ws.Xa, ws.Xb};
                for (int lp = 1; lp <= steps; ++lp) {
                    const int st = lp - 1;
                    ProbeEpi epi{g.in.rp, X[lp & 1], 0, nullptr, ws.Zv + (size_t)(j + lp) * n, ws.colsum};
                    if (lp == steps) {
                        epi.mode = 2;
                    } else if (lp >= 2) {
                        probe_coef_kernel<<<1, kProbeW, 0, g.stream>>>(ids, cnt, zv, cpow[(size_t)lp], ws.coef);
                        if ((e = cudaGetLastError()) != cudaSuccess) return e;
                        ++count;
                        epi.mode = 1;
                        epi.coef = ws.coef;
                    }
                    const ProbePush push{g.in.rp, g.in.col, X[st & 1], ws.Hn, ws.mark, ws.W[st & 1],
                                         ws.F[(st + 1) & 1], ws.ctl, st, thr};
                    probe_push_kernel<<<sparse_blocks, kBlock, 0, g.stream>>>(push);
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                    ++count;
                    if ((e = probe_step(g, X[st & 1], epi, ws.ppart, &count, ws.ctl, st, thr)) != cudaSuccess) return e;
                    const ProbeSparseEpi se{g.in.rp, ws.Hn, ws.mark, ws.F[(st + 1) & 1], ws.F[st & 1], X[st & 1],
                                            ws.W[(st + 1) & 1], ws.ctl, st, lp == steps ? 1 : 0, thr};
                    probe_sparse_epi_kernel<<<sparse_blocks, kBlock, 0, g.stream>>>(se, epi);
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                    ++count;
                }
                probe_cleanup_kernel<<<sparse_blocks, kBlock, 0, g.stream>>>(ws.ctl, ws.Xa, ws.Xb, (size_t)kProbeW * n);
                probe_coef_kernel<<<1, kProbeW, 0, g.stream>>>(ids, cnt, zv, cpow[(size_t)steps], ws.coef);
                probe_norm_finish_kernel<<<1, kProbeW, 0, g.stream>>>(ws.coef, ws.colsum, ws.sums + 63);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                count += 3;
            }
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
