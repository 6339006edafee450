// Forward and reverse sweeps of Algorithm 1: pull-style sparse matrix-vector
// products over the device CSRs.
//
//   forward (Algorithm 1, forward loop):  pi^l(i) = sqrt(c) * sum_{j in Out(i)} x^{l-1}(j),
//           x^{l}(i) = pi^l(i) / din(i)            -- rows of the out-edge CSR
//   reverse (Algorithm 1, reverse loop; Eq. sL):
//           s^l(j) = sqrt(c) / din(j) * sum_{i in I(j)} s^{l-1}(i) + D^(j) pi^{L-l}(j) / a
//                                                   -- rows of the in-edge CSR
//
// (P pi)(i) = sum_j P(i,j) pi(j) with P(i,j) = 1/din(j) for i in I(j), so the
// forward product pulls along out-edges with the 1/din factor folded into the
// gathered vector x; (P^T s)(j) = (1/din(j)) sum_{i in I(j)} s(i) pulls along
// in-edges.  Both are atomic-free and deterministic: each row's sum is formed in
// a fixed order by one thread group (short rows) or by fixed segments plus an
// in-order combine (long rows).
//
// Two arithmetic forms share the kernels through a value/accumulator policy:
//   FP64  -- the plain method: the history pi^l and the result s in FP64.  GB300's
//            scalar FP64 unit issues about 0.4 additions per SM per clock, so the
//            per-level arithmetic runs in two-float on the FP32 pipe: the gathered
//            vectors x^l and s^l are two-floats (float2, 8 bytes like a double), each
//            row sum is two-float, and the FP64 values are read and written through
//            integer conversions (f2conv.cuh).  Every stored value is within about
//            2^-46 relative of an FP64 computation of the same sums (the step and query
//            parity tests hold it to 1e-12 of the oracle).  The Lemma 5 sweeps of
//            Algorithm 3 and the sparse history keep FP64 sums (Pol64);
//   FP32c -- the precision form: pi^l and x^l stored in FP32 with two-float
//            (compensated) row sums; s^l stored and summed as two-floats; FP64
//            only for the final s^L and the D^ ratio.  On GB300, whose FP64 issue
//            rate is a small fraction of FP32, this keeps the sweeps bound by
//            memory rather than by FP64 arithmetic.
#include "common.cuh"
#include "f2conv.cuh"
#include "internal.h"
#include "twofloat.cuh"

#include <type_traits>

namespace esim {

// ---------------------------------------------------------------- policies

struct Pol64 {  // FP64 values, FP64 sums
    using V = double;
    using A = double;
    static __device__ __forceinline__ A zero() { return 0.0; }
    static __device__ __forceinline__ A add(A a, V v) { return a + v; }
    static __device__ __forceinline__ A combine(A a, A b) { return a + b; }
    static __device__ __forceinline__ A shfl(A a, int o, int w) { return __shfl_down_sync(0xffffffffu, a, o, w); }
};

struct Pol32c {  // FP32 values, two-float sums
    using V = float;
    using A = f2;
    static __device__ __forceinline__ A zero() { return f2{0.f, 0.f}; }
    static __device__ __forceinline__ A add(A a, V v) { return f2_add_f(a, v); }
    static __device__ __forceinline__ A combine(A a, A b) { return f2_add(a, b); }
    static __device__ __forceinline__ A shfl(A a, int o, int w) { return f2_shfl_down(a, o, w); }
};

struct Pol2f {  // two-float values (float2: hi, lo), two-float sums
    using V = float2;
    using A = f2;
    static __device__ __forceinline__ A zero() { return f2{0.f, 0.f}; }
    static __device__ __forceinline__ A add(A a, V v) { return f2_add(a, f2{v.x, v.y}); }
    static __device__ __forceinline__ A combine(A a, A b) { return f2_add(a, b); }
    static __device__ __forceinline__ A shfl(A a, int o, int w) { return f2_shfl_down(a, o, w); }
};

template <class Pol>
__device__ __forceinline__ typename Pol::A block_combine(typename Pol::A v, typename Pol::A* smem) {
    using A = typename Pol::A;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Pol::combine(v, Pol::shfl(v, o, 32));
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    A r = Pol::zero();
    if (wid == 0) {
        r = lane < nw ? smem[lane] : Pol::zero();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = Pol::combine(r, Pol::shfl(r, o, 32));
    }
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- row epilogues

struct ForwardOp {  // FP64
    double sc;
    const double* __restrict__ inv_din;
    double* __restrict__ pi_out;
    double* __restrict__ x_out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const {
        const double p = sc * acc;
        pi_out[row] = p;
        x_out[row] = p * inv_din[row];
    }
};

struct ReverseOp {  // FP64; 1/a is a host constant (an FP64 division per row is costly on GB300)
    double sc;
    double inv_a;
    const double* __restrict__ inv_din;
    const double* __restrict__ dhat;
    const double* __restrict__ h;  // pi^{L-l}
    double* __restrict__ s_out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const {
        s_out[row] = (sc * acc) * inv_din[row] + dhat[row] * h[row] * inv_a;
    }
};

struct ReverseSparseOp {  // FP64; the D^ pi^{L-l} / a term is scattered from the sparse history
    double sc;
    const double* __restrict__ inv_din;
    double* __restrict__ s_out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const { s_out[row] = (sc * acc) * inv_din[row]; }
};

struct ForwardOp32c {  // FP32 storage, two-float sum
    f2 sc;
    const uint32_t* __restrict__ in_rp;
    float* __restrict__ pi_out;
    float* __restrict__ x_out;
    __device__ __forceinline__ void operator()(int64_t row, f2 acc) const {
        const f2 p = f2_mul(acc, sc);
        const float pf = __fadd_rn(p.hi, p.lo);
        pi_out[row] = pf;
        const uint32_t d = in_rp[row + 1] - in_rp[row];
        x_out[row] = d ? __fdiv_rn(pf, (float)d) : 0.f;
    }
};

// Reverse level in two-float: s^l = sqrt(c) (P^T s^{l-1}) + w pi^{L-l}, w = D^/a
// as a two-float; intermediate levels store float2, the last level FP64.
template <bool kFinal>
struct ReverseOp2f {
    f2 sc;
    const uint32_t* __restrict__ rp;
    const float2* __restrict__ w;
    const float* __restrict__ h;
    float2* __restrict__ s_out;
    double* __restrict__ s_final;
    __device__ __forceinline__ void operator()(int64_t row, f2 acc) const {
        const uint32_t d = rp[row + 1] - rp[row];
        f2 prop = f2{0.f, 0.f};
        if (d) prop = f2_div_f(f2_mul(acc, sc), (float)d);
        const float2 wv = w[row];
        const f2 s = f2_add(prop, f2_mul_f(f2{wv.x, wv.y}, h[row]));
        if (kFinal) s_final[row] = f2_to_double(s);
        else s_out[row] = make_float2(s.hi, s.lo);
    }
};

// FP64 form, forward level: pi^l = sqrt(c) * row sum in two-float, stored as FP64;
// x^l = pi^l / din stored as a two-float for the next level's gathers.
struct ForwardOpD {
    f2 sc;
    const uint32_t* __restrict__ in_rp;
    double* __restrict__ pi_out;
    float2* __restrict__ x_out;
    __device__ __forceinline__ void operator()(int64_t row, f2 acc) const {
        const f2 p = f2_mul(acc, sc);
        pi_out[row] = f2_to_double_bits(p);
        const uint32_t d = in_rp[row + 1] - in_rp[row];
        const f2 x = d ? f2_div_f(p, (float)d) : f2{0.f, 0.f};
        x_out[row] = make_float2(x.hi, x.lo);
    }
};

// FP64 form: D^(k) pi^{L-l}(k) / a in two-float from the FP64 values (exact quotient
// correction, so pi = a and D^ = 1 give 1 exactly)
__device__ __forceinline__ f2 diag_term(double dhat, double h, f2 a) {
    return f2_div(f2_mul(double_to_f2_bits(dhat), double_to_f2_bits(h)), a);
}

// FP64 form, reverse level: s^l = sqrt(c) (P^T s^{l-1}) + D^ pi^{L-l} / a in two-float,
// pi^{L-l} and D^ read in FP64; s^l stored as a two-float, the last level as FP64.
template <bool kFinal>
struct ReverseOpD {
    f2 sc;
    f2 a;
    const uint32_t* __restrict__ rp;
    const double* __restrict__ dhat;
    const double* __restrict__ h;
    float2* __restrict__ s_out;
    double* __restrict__ s_final;
    __device__ __forceinline__ void operator()(int64_t row, f2 acc) const {
        const uint32_t d = rp[row + 1] - rp[row];
        const f2 prop = d ? f2_div_f(f2_mul(acc, sc), (float)d) : f2{0.f, 0.f};
        const f2 s = f2_add(prop, diag_term(dhat[row], h[row], a));
        if (kFinal) s_final[row] = f2_to_double_bits(s);
        else s_out[row] = make_float2(s.hi, s.lo);
    }
};

// ---------------------------------------------------------------- row kernels
//
// A sweep level is gather-bound: each entry reads one value x[col[p]] from a vector
// that sits in L2, and a random 4- or 8-byte gather costs a 32-byte sector whatever its
// width.  The tile kernel keeps every lane gathering and no warp waiting on another:
// each warp takes a tile of consecutive rows holding at most tile_cap (<= kSweepTile)
// entries, gathers all of its entries (coalesced column loads, eight gathers in
// flight per lane) into its own slice of shared memory, and then sums the rows from
// there -- rows of up to 32 entries one lane each (two chains, even and odd entries),
// longer rows by the whole warp (lanes stride the row, a fixed shuffle tree joins
// them).  Rows longer than a tile are cut into segments: the blocks past tile_blocks
// sum one segment each into partial[], and long_rows_kernel adds a row's partials in
// order.  Every row's sum has a fixed order, so the sweeps are deterministic.

template <class Pol, class Op>
__global__ void __launch_bounds__(kBlock) tile_rows_kernel(const uint32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const typename Pol::V* __restrict__ x,
                                                           const uint32_t* __restrict__ tiles, int64_t ntiles,
                                                           uint32_t tile_cap, Op op, int64_t nseg,
                                                           const Segment* __restrict__ seg,
                                                           typename Pol::A* __restrict__ partial, int tile_blocks) {
    using A = typename Pol::A;
    using V = typename Pol::V;
    constexpr int kWarps = kBlock / 32;
    constexpr int kU = 8;  // gathers in flight per lane
    __shared__ V vals[kWarps][kSweepTile];
    __shared__ A red[kWarps];
    if ((int)blockIdx.x >= tile_blocks) {
        const int64_t nsb = (int64_t)gridDim.x - tile_blocks;
        for (int64_t s = (int64_t)blockIdx.x - tile_blocks; s < nseg; s += nsb) {
            const Segment sg = seg[s];
            A acc = Pol::zero();
            for (uint32_t p = sg.beg + threadIdx.x; p < sg.end; p += blockDim.x) acc = Pol::add(acc, x[__ldg(col + p)]);
            acc = block_combine<Pol>(acc, red);
            if (threadIdx.x == 0) partial[s] = acc;
        }
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    V* my = vals[wid];
    const int64_t nwarps = (int64_t)tile_blocks * kWarps;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + wid; t < ntiles; t += nwarps) {
        const uint32_t r0 = __ldg(tiles + t), r1 = __ldg(tiles + t + 1);
        const uint32_t b = __ldg(rp + r0), e = __ldg(rp + r1);
        if (e - b > kSweepTile) continue;  // one long row: the segment blocks sum it (warp-uniform)
        for (uint32_t p = b + lane; p < e; p += 32 * kU) {
            V g[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t q = p + (uint32_t)(32 * u);
                if (q < e) g[u] = x[__ldg(col + q)];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint32_t q = p + (uint32_t)(32 * u);
                if (q < e) my[q - b] = g[u];
            }
        }
        __syncwarp();
        for (uint32_t base = r0; base < r1; base += 32) {
            const uint32_t r = base + (uint32_t)lane;
            uint32_t rb = 0, re = 0;
            if (r < r1) {
                rb = __ldg(rp + r);
                re = __ldg(rp + r + 1);
            }
            const bool big = re - rb > 32u;
            if (r < r1 && !big) {
                A acc0 = Pol::zero(), acc1 = Pol::zero();
                uint32_t q = rb;
                for (; q + 1 < re; q += 2) {
                    acc0 = Pol::add(acc0, my[q - b]);
                    acc1 = Pol::add(acc1, my[q + 1 - b]);
                }
                if (q < re) acc0 = Pol::add(acc0, my[q - b]);
                op((int64_t)r, Pol::combine(acc0, acc1));
            }
            unsigned mask = __ballot_sync(0xffffffffu, big);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1u;
                const uint32_t wb = __shfl_sync(0xffffffffu, rb, src), we = __shfl_sync(0xffffffffu, re, src);
                A acc = Pol::zero();
                for (uint32_t q = wb + (uint32_t)lane; q < we; q += 32) acc = Pol::add(acc, my[q - b]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc = Pol::combine(acc, Pol::shfl(acc, o, 32));
                if (lane == 0) op((int64_t)(base + (uint32_t)src), acc);
            }
        }
        __syncwarp();
    }
}

// FP64 sums (Pol64: Algorithm 3's Lemma 5 sweeps and the sparse history) use a row
// kernel with G lanes per row instead: its short dependency chains suit the slow FP64
// unit on the small graphs those sweeps run on.
// Blocks [0, short_blocks) sweep the short rows, G lanes per row; the remaining
// blocks each combine one segment of a long row into partial[].
template <class Pol, int G, class Op>
__global__ void __launch_bounds__(kBlock) rows_kernel(int64_t n, const uint32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const typename Pol::V* __restrict__ x, uint32_t long_min, Op op,
                                                      int64_t nseg, const Segment* __restrict__ seg,
                                                      typename Pol::A* __restrict__ partial, int short_blocks) {
    using A = typename Pol::A;
    __shared__ A red[kBlock / 32];
    if ((int)blockIdx.x >= short_blocks) {
        const int64_t nsb = (int64_t)gridDim.x - short_blocks;
        for (int64_t s = (int64_t)blockIdx.x - short_blocks; s < nseg; s += nsb) {
            const Segment sg = seg[s];
            A acc = Pol::zero();
            for (uint32_t p = sg.beg + threadIdx.x; p < sg.end; p += blockDim.x) acc = Pol::add(acc, x[__ldg(col + p)]);
            acc = block_combine<Pol>(acc, red);
            if (threadIdx.x == 0) partial[s] = acc;
        }
        return;
    }
    constexpr int RPW = 32 / G;  // rows per warp per iteration
    const int lane = threadIdx.x & 31;
    const int sub = lane / G, gl = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)short_blocks * blockDim.x) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t row = base + sub;
        uint32_t b = 0, e = 0;
        bool mine = false;
        if (row < n) {
            b = __ldg(rp + row);
            e = __ldg(rp + row + 1);
            mine = (e - b) < long_min;
            if (!mine) e = b;
        }
        A acc0 = Pol::zero(), acc1 = Pol::zero();
        uint32_t p = b + gl;
        for (; p + G < e; p += 2 * G) {
            const int32_t c0 = __ldg(col + p), c1 = __ldg(col + p + G);
            acc0 = Pol::add(acc0, x[c0]);
            acc1 = Pol::add(acc1, x[c1]);
        }
        if (p < e) acc0 = Pol::add(acc0, x[__ldg(col + p)]);
        A acc = Pol::combine(acc0, acc1);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc = Pol::combine(acc, Pol::shfl(acc, o, G));
        if (gl == 0 && mine) op(row, acc);
    }
}

// One warp per long row: combine the row's segment partials in order.
template <class Pol, class Op>
__global__ void __launch_bounds__(kBlock) long_rows_kernel(int64_t nlong, const int32_t* __restrict__ long_rows,
                                                           const int32_t* __restrict__ long_first,
                                                           const typename Pol::A* __restrict__ partial, Op op) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nlong || lane != 0) return;
    typename Pol::A acc = Pol::zero();
    for (int32_t s = long_first[w]; s < long_first[w + 1]; ++s) acc = Pol::combine(acc, partial[s]);
    op(long_rows[w], acc);
}

// ---------------------------------------------------------------- level 0

__global__ void forward_init_kernel(int64_t n, int64_t u, double a, const double* __restrict__ inv_din,
                                    double* __restrict__ pi0, double* __restrict__ x0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        pi0[i] = i == u ? a : 0.0;
        x0[i] = i == u ? a * inv_din[i] : 0.0;
    }
}

// FP64 form, level 0: pi^0 = a e_u (FP64), x^0 = a / din(u) e_u as a two-float.
__global__ void forward_init_d_kernel(int64_t n, int64_t u, double a, float xhi, float xlo,
                                      double* __restrict__ pi0, float2* __restrict__ x0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        pi0[i] = i == u ? a : 0.0;
        x0[i] = i == u ? make_float2(xhi, xlo) : make_float2(0.f, 0.f);
    }
}

// FP64 form: s^0 = D^ pi^L / a as a two-float (in FP64 when L = 0).
__global__ void reverse_init_d_kernel(int64_t n, float a_hi, float a_lo, const double* __restrict__ dhat,
                                      const double* __restrict__ h, float2* __restrict__ s0,
                                      double* __restrict__ s_final) {
    const f2 a{a_hi, a_lo};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const f2 s = diag_term(dhat[i], h[i], a);
        if (s_final) s_final[i] = f2_to_double_bits(s);
        else s0[i] = make_float2(s.hi, s.lo);
    }
}

__global__ void forward_init32_kernel(int64_t n, int64_t u, float a, const uint32_t* __restrict__ in_rp,
                                      float* __restrict__ pi0, float* __restrict__ x0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p = 0.f, xv = 0.f;
        if (i == u) {
            p = a;
            const uint32_t d = in_rp[i + 1] - in_rp[i];
            xv = d ? __fdiv_rn(a, (float)d) : 0.f;
        }
        pi0[i] = p;
        x0[i] = xv;
    }
}

__global__ void reverse_init_kernel(int64_t n, double inv_a, const double* __restrict__ dhat,
                                    const double* __restrict__ h, double* __restrict__ s0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s0[i] = dhat[i] * h[i] * inv_a;
}

// w = D^ / a as two-floats, and s^0 = w pi^L (float2, or FP64 when L = 0)
__global__ void reverse_init2f_kernel(int64_t n, double inv_a, const double* __restrict__ dhat,
                                      const float* __restrict__ h, float2* __restrict__ w, float2* __restrict__ s0,
                                      double* __restrict__ s_final) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const f2 wv = f2_from_double(dhat[i] * inv_a);
        w[i] = make_float2(wv.hi, wv.lo);
        const f2 s = f2_mul_f(wv, h[i]);
        if (s_final) s_final[i] = f2_to_double(s);
        else s0[i] = make_float2(s.hi, s.lo);
    }
}

// ---------------------------------------------------------------- launchers

namespace {

// Sparse linearization (Section 3.2): after forward level l, pi_run += pi^l (level
// order, as the dense sum) and the entries pi^l(k) > theta are appended to the
// sparse history as (k, pi^l(k)).  Warps take their slots with one atomic each; the
// order of entries within a level therefore varies, but each node appears at most
// once per level, so the reverse scatter gives the same values whatever the order.
// The last block to finish records the level's end (a ticket, no waiting).
__global__ void __launch_bounds__(kBlock) compact_level_kernel(int64_t n, const double* __restrict__ lev,
                                                               double* __restrict__ pi_run, int first, double theta,
                                                               SparseHist h, int level, Status* __restrict__ st) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {  // uniform per block
        const int64_t i = base + threadIdx.x;
        double v = 0.0;
        bool keep = false;
        if (i < n) {
            v = lev[i];
            pi_run[i] = first ? v : pi_run[i] + v;
            keep = v > theta;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (mask) {
            unsigned long long pos0 = 0ull;
            if (lane == 0) pos0 = atomicAdd(&st->hist_count, (unsigned long long)__popc(mask));
            pos0 = __shfl_sync(0xffffffffu, pos0, 0);
            if (keep) {
                const unsigned long long pos = pos0 + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
                if (pos < h.cap) {
                    h.idx[pos] = (int32_t)i;
                    h.val[pos] = v;
                } else if (h.cap) {
                    atomicOr(&st->err, kErrCapacity);
                }  // cap = 0: counting pass
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&st->ticket, 1u);
        if (t == gridDim.x - 1) {
            const unsigned long long end = atomicAdd(&st->hist_count, 0ull);
            if (h.lvl) h.lvl[level + 1] = end < h.cap ? end : h.cap;
            st->ticket = 0u;
        }
    }
}

// s(k) += D^(k) pi^level(k) / a (times the host's 1/a) over the sparse entries of one
// level (unique nodes).
__global__ void __launch_bounds__(kBlock) scatter_level_kernel(const uint64_t* __restrict__ lvl, int level,
                                                               const int32_t* __restrict__ idx,
                                                               const double* __restrict__ val,
                                                               const double* __restrict__ dhat, double inv_a,
                                                               double* __restrict__ s) {
    const uint64_t beg = lvl[level], end = lvl[level + 1];
    for (uint64_t p = beg + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t k = idx[p];
        s[k] = s[k] + dhat[k] * val[p] * inv_a;
    }
}

int elementwise_blocks(const Graph& g, int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)g.sm_count * 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <class Pol, int G, class Op>
cudaError_t sweep_level_g(const Graph& g, const DevCsr& A, const typename Pol::V* x, const Op& op) {
    using Acc = typename Pol::A;
    Acc* partial = reinterpret_cast<Acc*>(g.partial);
    int64_t rows_per_block = kBlock / G;
    int64_t sb = (g.n + rows_per_block - 1) / rows_per_block;
    int64_t cap = (int64_t)g.sm_count * 16;
    if (sb > cap) sb = cap;
    if (sb < 1) sb = 1;
    int64_t segb = A.nseg;
    if (segb > (int64_t)g.sm_count * 16) segb = (int64_t)g.sm_count * 16;
    rows_kernel<Pol, G, Op><<<(unsigned)(sb + segb), kBlock, 0, g.stream>>>(g.n, A.rp, A.col, x, A.long_min, op, A.nseg,
                                                                            A.seg, partial, (int)sb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (A.nlong > 0) {
        int64_t blocks = (A.nlong * 32 + kBlock - 1) / kBlock;
        long_rows_kernel<Pol, Op><<<(unsigned)blocks, kBlock, 0, g.stream>>>(A.nlong, A.long_rows, A.long_first,
                                                                             partial, op);
        e = cudaGetLastError();
    }
    return e;
}

template <class Pol, class Op>
cudaError_t sweep_level_rows(const Graph& g, const DevCsr& A, const typename Pol::V* x, const Op& op) {
    switch (A.group) {
        case 2: return sweep_level_g<Pol, 2>(g, A, x, op);
        case 4: return sweep_level_g<Pol, 4>(g, A, x, op);
        case 8: return sweep_level_g<Pol, 8>(g, A, x, op);
        case 16: return sweep_level_g<Pol, 16>(g, A, x, op);
        default: return sweep_level_g<Pol, 32>(g, A, x, op);
    }
}

template <class Pol, class Op>
cudaError_t sweep_level(const Graph& g, const DevCsr& A, const typename Pol::V* x, const Op& op) {
    if constexpr (std::is_same<Pol, Pol64>::value) return sweep_level_rows<Pol>(g, A, x, op);
    using Acc = typename Pol::A;
    Acc* partial = reinterpret_cast<Acc*>(g.partial);
    // one block per eight tiles (the hardware balances the blocks over the SMs), then the
    // segment blocks
    const int64_t warps = kBlock / 32;
    int64_t tb = (A.ntiles + warps - 1) / warps;
    if (tb < 1) tb = 1;
    const int64_t cap = (int64_t)g.sm_count * 8;
    int64_t segb = A.tnseg;
    if (segb > cap) segb = cap;
    tile_rows_kernel<Pol, Op><<<(unsigned)(tb + segb), kBlock, 0, g.stream>>>(
        A.rp, A.col, x, A.tiles, A.ntiles, A.tile_cap, op, A.tnseg, A.tseg, partial, (int)tb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (A.tnlong > 0) {
        int64_t blocks = (A.tnlong * 32 + kBlock - 1) / kBlock;
        long_rows_kernel<Pol, Op><<<(unsigned)blocks, kBlock, 0, g.stream>>>(A.tnlong, A.tlong_rows, A.tlong_first,
                                                                             partial, op);
        e = cudaGetLastError();
    }
    return e;
}

f2 host_f2(double v) {
    const float h = (float)v;
    return f2{h, (float)(v - (double)h)};
}

}  // namespace

cudaError_t launch_forward(const Graph& g, int64_t u, double c, int32_t L, double* hist, double* xa, double* xb) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    const uint32_t din_u = (*g.din_host)[(size_t)u];
    const f2 x0 = din_u ? host_f2(a / (double)din_u) : f2{0.f, 0.f};
    float2* x[2] = {reinterpret_cast<float2*>(xa), reinterpret_cast<float2*>(xb)};
    forward_init_d_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, a, x0.hi, x0.lo, hist, x[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const f2 sc2 = host_f2(sc);
    for (int32_t l = 1; l <= L; ++l) {
        ForwardOpD op{sc2, g.in.rp, hist + (size_t)l * (size_t)g.n, x[l & 1]};
        e = sweep_level<Pol2f>(g, g.out, x[(l - 1) & 1], op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Two-float vectors: s^l in sa and (as scratch) in s_out, alternating so that level L-1
// lands in sa and the last level reads sa and writes s_out in FP64.
cudaError_t launch_reverse(const Graph& g, const double* hist, int32_t L, double c, const double* dhat, double* s_out,
                           double* sa, double* /*sb*/) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    float2* A = reinterpret_cast<float2*>(sa);
    float2* S = reinterpret_cast<float2*>(s_out);
    auto buf = [&](int32_t l) { return ((L - 1 - l) & 1) == 0 ? A : S; };
    const f2 a2 = host_f2(a);
    reverse_init_d_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(
        g.n, a2.hi, a2.lo, dhat, hist + (size_t)L * g.n, L > 0 ? buf(0) : nullptr, L == 0 ? s_out : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const f2 sc2 = host_f2(sc);
    for (int32_t l = 1; l <= L; ++l) {
        const float2* sp = buf(l - 1);
        const double* h = hist + (size_t)(L - l) * g.n;
        if (l < L) {
            ReverseOpD<false> op{sc2, a2, g.in.rp, dhat, h, buf(l), nullptr};
            e = sweep_level<Pol2f>(g, g.in, sp, op);
        } else {
            ReverseOpD<true> op{sc2, a2, g.in.rp, dhat, h, nullptr, s_out};
            e = sweep_level<Pol2f>(g, g.in, sp, op);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Forward sweeps with the sparse history: dense rolling vectors (lev = pi^l, x^l),
// pi = sum_l pi^l accumulated in level order, and only pi^l(k) > theta kept.  With
// h.cap = 0 and h.lvl = NULL the entries are only counted (into Status::hist_count).
cudaError_t launch_forward_sparse(const Graph& g, int64_t u, double c, int32_t L, double theta, const SparseHist& h,
                                  double* lev, double* pi_run, double* xa, double* xb) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    cudaError_t e = cudaSuccess;
    if (h.lvl && (e = cudaMemsetAsync(h.lvl, 0, sizeof(uint64_t) * (size_t)(L + 2), g.stream)) != cudaSuccess)
        return e;
    const int eb = elementwise_blocks(g, g.n);
    forward_init_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, u, a, g.inv_din, lev, xa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    compact_level_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, lev, pi_run, 1, theta, h, 0, g.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double* x[2] = {xa, xb};
    for (int32_t l = 1; l <= L; ++l) {
        ForwardOp op{sc, g.inv_din, lev, x[l & 1]};
        if ((e = sweep_level<Pol64>(g, g.out, x[(l - 1) & 1], op)) != cudaSuccess) return e;
        compact_level_kernel<<<eb, kBlock, 0, g.stream>>>(g.n, lev, pi_run, 0, theta, h, l, g.status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Reverse sweeps with the sparse history: s^l = sqrt(c) P^T s^{l-1}, then the kept
// entries of pi^{L-l} add D^ pi^{L-l} / a.
cudaError_t launch_reverse_sparse(const Graph& g, const SparseHist& h, int32_t L, double c, const double* dhat,
                                  double* s_out, double* sa) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    double* buf[2] = {s_out, sa};
    const unsigned sb = (unsigned)g.sm_count * 4;
    cudaError_t e = launch_fill(g, g.n, 0.0, buf[L & 1]);
    if (e != cudaSuccess) return e;
    scatter_level_kernel<<<sb, kBlock, 0, g.stream>>>(h.lvl, L, h.idx, h.val, dhat, 1.0 / a, buf[L & 1]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int32_t l = 1; l <= L; ++l) {
        double* sn = buf[(L - l) & 1];
        ReverseSparseOp op{sc, g.inv_din, sn};
        if ((e = sweep_level<Pol64>(g, g.in, buf[(L - l + 1) & 1], op)) != cudaSuccess) return e;
        scatter_level_kernel<<<sb, kBlock, 0, g.stream>>>(h.lvl, L - l, h.idx, h.val, dhat, 1.0 / a, sn);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Algorithm 3 helpers: h_l = (P^T)^l(u, .), the distribution of a non-stop walk from
// u (no decay, no stop), for l = 0..steps, into H[(steps+1) * n] (FP64 storage), on the
// warp-tile kernel in the FP64 form's two-float arithmetic (x_l = h_l / din as two-floats
// in xa/xb, n 8-byte entries each).
cudaError_t launch_walk_distributions(const Graph& g, int64_t u, int steps, double* H, double* xa, double* xb) {
    const uint32_t din_u = (*g.din_host)[(size_t)u];
    const f2 x0 = din_u ? host_f2(1.0 / (double)din_u) : f2{0.f, 0.f};
    float2* x[2] = {reinterpret_cast<float2*>(xa), reinterpret_cast<float2*>(xb)};
    forward_init_d_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, 1.0, x0.hi, x0.lo, H, x[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const f2 one{1.f, 0.f};
    for (int l = 1; l <= steps; ++l) {
        ForwardOpD op{one, g.in.rp, H + (size_t)l * (size_t)g.n, x[l & 1]};
        e = sweep_level<Pol2f>(g, g.out, x[(l - 1) & 1], op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct PlainOpD {
    double* __restrict__ out;
    __device__ __forceinline__ void operator()(int64_t row, f2 acc) const { out[row] = f2_to_double_bits(acc); }
};

// out(i) = sum_{j in Out(i)} x(j): the pull product over out-edges without weights, x as
// two-floats, the sums in two-float, out in FP64.
cudaError_t launch_pull_sum(const Graph& g, const float2* x, double* out) {
    return sweep_level<Pol2f>(g, g.out, x, PlainOpD{out});
}

cudaError_t launch_forward32(const Graph& g, int64_t u, double c, int32_t L, float* hist, float* xa, float* xb) {
    const double sc = sqrt(c);
    const float a = (float)(1.0 - sc);
    forward_init32_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, a, g.in.rp, hist, xa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float* x[2] = {xa, xb};
    const f2 sc2 = host_f2(sc);
    for (int32_t l = 1; l <= L; ++l) {
        ForwardOp32c op{sc2, g.in.rp, hist + (size_t)l * (size_t)g.n, x[l & 1]};
        e = sweep_level<Pol32c>(g, g.out, x[(l - 1) & 1], op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reverse32(const Graph& g, const float* hist, int32_t L, double c, const double* dhat,
                             double* s_out, float2* w, float2* sa, float2* sb) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    float2* buf[2] = {sa, sb};
    reverse_init2f_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(
        g.n, 1.0 / a, dhat, hist + (size_t)L * g.n, w, buf[0], L == 0 ? s_out : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const f2 sc2 = host_f2(sc);
    for (int32_t l = 1; l <= L; ++l) {
        const float2* sp = buf[(l - 1) & 1];
        const float* h = hist + (size_t)(L - l) * g.n;
        if (l < L) {
            ReverseOp2f<false> op{sc2, g.in.rp, w, h, buf[l & 1], nullptr};
            e = sweep_level<Pol2f>(g, g.in, sp, op);
        } else {
            ReverseOp2f<true> op{sc2, g.in.rp, w, h, nullptr, s_out};
            e = sweep_level<Pol2f>(g, g.in, sp, op);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace esim
