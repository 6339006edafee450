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
// in-edges.  Both are atomic-free and deterministic: each row's sum is formed
// in a fixed order by one thread group (short rows) or by fixed segments plus an
// in-order combine (long rows).
#include "common.cuh"
#include "internal.h"

namespace esim {

struct ForwardOp {
    double sc;
    const uint32_t* __restrict__ in_rp;
    double* __restrict__ pi_out;
    double* __restrict__ x_out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const {
        const double p = sc * acc;
        pi_out[row] = p;
        const uint32_t d = in_rp[row + 1] - in_rp[row];
        x_out[row] = d ? p / (double)d : 0.0;
    }
};

struct ReverseOp {
    double sc;
    double a;
    const uint32_t* __restrict__ rp;  // the in-edge CSR being swept
    const double* __restrict__ dhat;
    const double* __restrict__ h;     // pi^{L-l}
    double* __restrict__ s_out;
    __device__ __forceinline__ void operator()(int64_t row, double acc) const {
        const uint32_t d = rp[row + 1] - rp[row];
        const double prop = d ? (sc * acc) / (double)d : 0.0;
        s_out[row] = prop + dhat[row] * h[row] / a;
    }
};

// Blocks [0, short_blocks) sweep the short rows, G lanes per row; the remaining
// blocks each sum one segment of a long row into partial[].
template <int G, class Op>
__global__ void __launch_bounds__(kBlock) rows_kernel(int64_t n, const uint32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ x, uint32_t long_min, Op op,
                                                      int64_t nseg, const Segment* __restrict__ seg,
                                                      double* __restrict__ partial, int short_blocks) {
    __shared__ double red[kBlock / 32];
    if ((int)blockIdx.x >= short_blocks) {
        const int64_t nsb = (int64_t)gridDim.x - short_blocks;
        for (int64_t s = (int64_t)blockIdx.x - short_blocks; s < nseg; s += nsb) {
            const Segment sg = seg[s];
            double acc = 0.0;
            for (uint32_t p = sg.beg + threadIdx.x; p < sg.end; p += blockDim.x) acc += __ldg(x + __ldg(col + p));
            acc = block_sum(acc, red);
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
        double acc0 = 0.0, acc1 = 0.0;
        uint32_t p = b + gl;
        for (; p + G < e; p += 2 * G) {
            const int32_t c0 = __ldg(col + p), c1 = __ldg(col + p + G);
            acc0 += __ldg(x + c0);
            acc1 += __ldg(x + c1);
        }
        if (p < e) acc0 += __ldg(x + __ldg(col + p));
        double acc = acc0 + acc1;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
        if (gl == 0 && mine) op(row, acc);
    }
}

// One warp per long row: combine the row's segment partials in order.
template <class Op>
__global__ void __launch_bounds__(kBlock) long_rows_kernel(int64_t nlong, const int32_t* __restrict__ long_rows,
                                                           const int32_t* __restrict__ long_first,
                                                           const double* __restrict__ partial, Op op) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nlong || lane != 0) return;
    double acc = 0.0;
    for (int32_t s = long_first[w]; s < long_first[w + 1]; ++s) acc += partial[s];
    op(long_rows[w], acc);
}

__global__ void forward_init_kernel(int64_t n, int64_t u, double a, const uint32_t* __restrict__ in_rp,
                                    double* __restrict__ pi0, double* __restrict__ x0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double p = 0.0, xv = 0.0;
        if (i == u) {
            p = a;
            const uint32_t d = in_rp[i + 1] - in_rp[i];
            xv = d ? a / (double)d : 0.0;
        }
        pi0[i] = p;
        x0[i] = xv;
    }
}

__global__ void reverse_init_kernel(int64_t n, double a, const double* __restrict__ dhat,
                                    const double* __restrict__ h, double* __restrict__ s0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s0[i] = dhat[i] * h[i] / a;
}

namespace {

int elementwise_blocks(const Graph& g, int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)g.sm_count * 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <int G, class Op>
cudaError_t sweep_level_g(const Graph& g, const DevCsr& A, const double* x, const Op& op, double* partial) {
    int64_t rows_per_block = kBlock / G;
    int64_t sb = (g.n + rows_per_block - 1) / rows_per_block;
    int64_t cap = (int64_t)g.sm_count * 16;
    if (sb > cap) sb = cap;
    if (sb < 1) sb = 1;
    int64_t segb = A.nseg;
    if (segb > (int64_t)g.sm_count * 16) segb = (int64_t)g.sm_count * 16;
    rows_kernel<G, Op><<<(unsigned)(sb + segb), kBlock, 0, g.stream>>>(g.n, A.rp, A.col, x, A.long_min, op, A.nseg,
                                                                       A.seg, partial, (int)sb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (A.nlong > 0) {
        int64_t blocks = (A.nlong * 32 + kBlock - 1) / kBlock;
        long_rows_kernel<Op><<<(unsigned)blocks, kBlock, 0, g.stream>>>(A.nlong, A.long_rows, A.long_first, partial, op);
        e = cudaGetLastError();
    }
    return e;
}

template <class Op>
cudaError_t sweep_level(const Graph& g, const DevCsr& A, const double* x, const Op& op, double* partial) {
    switch (A.group) {
        case 2: return sweep_level_g<2>(g, A, x, op, partial);
        case 4: return sweep_level_g<4>(g, A, x, op, partial);
        case 8: return sweep_level_g<8>(g, A, x, op, partial);
        case 16: return sweep_level_g<16>(g, A, x, op, partial);
        default: return sweep_level_g<32>(g, A, x, op, partial);
    }
}

}  // namespace

cudaError_t launch_forward(const Graph& g, int64_t u, double c, int32_t L, double* hist, double* xa, double* xb) {
    const double sc = sqrt(c);
    const double a = 1.0 - sc;
    forward_init_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, u, a, g.in.rp, hist, xa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* x[2] = {xa, xb};
    for (int32_t l = 1; l <= L; ++l) {
        const double* xp = x[(l - 1) & 1];
        double* xn = x[l & 1];
        ForwardOp op{sc, g.in.rp, hist + (size_t)l * (size_t)g.n, xn};
        e = sweep_level(g, g.out, xp, op, g.partial);
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
    reverse_init_kernel<<<elementwise_blocks(g, g.n), kBlock, 0, g.stream>>>(g.n, a, dhat, hist + (size_t)L * g.n,
                                                                             buf[L & 1]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int32_t l = 1; l <= L; ++l) {
        const double* sp = buf[(L - l + 1) & 1];
        double* sn = buf[(L - l) & 1];
        ReverseOp op{sc, a, g.in.rp, dhat, hist + (size_t)(L - l) * g.n, sn};
        e = sweep_level(g, g.in, sp, op, g.partial);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace esim
