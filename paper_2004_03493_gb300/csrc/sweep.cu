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
//   FP64  -- values and sums in FP64 (the plain method);
//   FP32c -- the precision form: pi^l and x^l stored in FP32 with two-float
//            (compensated) row sums; s^l stored and summed as two-floats; FP64
//            only for the final s^L and the D^ ratio.  On GB300, whose FP64 issue
//            rate is a small fraction of FP32, this keeps the sweeps bound by
//            memory rather than by FP64 arithmetic.
#include "common.cuh"
#include "internal.h"
#include "twofloat.cuh"

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

// ---------------------------------------------------------------- row kernels

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
cudaError_t sweep_level(const Graph& g, const DevCsr& A, const typename Pol::V* x, const Op& op) {
    switch (A.group) {
        case 2: return sweep_level_g<Pol, 2>(g, A, x, op);
        case 4: return sweep_level_g<Pol, 4>(g, A, x, op);
        case 8: return sweep_level_g<Pol, 8>(g, A, x, op);
        case 16: return sweep_level_g<Pol, 16>(g, A, x, op);
        default: return sweep_level_g<Pol, 32>(g, A, x, op);
    }
}

f2 host_f2(double v) {
    const float h = (float)v;
    return f2{h, (float)(v - (double)h)};
}

}  // namespace

cudaError_t launch_forward(const Graph& g, int64_t u, double c, int32_t L, double* hist, double* xa, double* xb) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    forward_init_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, a, g.inv_din, hist, xa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* x[2] = {xa, xb};
    for (int32_t l = 1; l <= L; ++l) {
        const double* xp = x[(l - 1) & 1];
        double* xn = x[l & 1];
        ForwardOp op{sc, g.inv_din, hist + (size_t)l * (size_t)g.n, xn};
        e = sweep_level<Pol64>(g, g.out, xp, op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reverse(const Graph& g, const double* hist, int32_t L, double c, const double* dhat, double* s_out,
                           double* sa, double* /*sb*/) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    // level l writes buf[(L - l) & 1]; buf[0] = s_out, so level L lands in s_out
    double* buf[2] = {s_out, sa};
    const double inv_a = 1.0 / a;
    reverse_init_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, inv_a, dhat,
                                                                             hist + (size_t)L * g.n, buf[L & 1]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int32_t l = 1; l <= L; ++l) {
        const double* sp = buf[(L - l + 1) & 1];
        double* sn = buf[(L - l) & 1];
        ReverseOp op{sc, inv_a, g.inv_din, dhat, hist + (size_t)(L - l) * g.n, sn};
        e = sweep_level<Pol64>(g, g.in, sp, op);
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
// u (no decay, no stop), for l = 0..steps, into H[(steps+1) * n] (FP64).
cudaError_t launch_walk_distributions(const Graph& g, int64_t u, int steps, double* H, double* xa, double* xb) {
    forward_init_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, 1.0, g.inv_din, H, xa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* x[2] = {xa, xb};
    for (int l = 1; l <= steps; ++l) {
        ForwardOp op{1.0, g.inv_din, H + (size_t)l * (size_t)g.n, x[l & 1]};
        e = sweep_level<Pol64>(g, g.out, x[(l - 1) & 1], op);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct PlainOp {
    double* __restrict__ out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const { out[row] = acc; }
};

// out(i) = sum_{j in Out(i)} x(j): the pull product over out-edges without weights.
cudaError_t launch_pull_sum(const Graph& g, const double* x, double* out) {
    return sweep_level<Pol64>(g, g.out, x, PlainOp{out});
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
