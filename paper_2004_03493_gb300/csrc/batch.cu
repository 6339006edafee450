// Batched queries: B sources (B <= 64) with their own eps share every sweep, so the
// sparse matrix-vector products of Algorithm 1 become sparse matrix times dense
// n x W products (W = 32 or 64 columns, row-major, padding columns are zero).
//
// Precision form throughout: pi^l stored in FP32 with two-float row sums; s^l
// stored and summed as two-floats; FP64 only for the final s and for D^.
//
// Column q uses its own depth L_q = ceil(log_{1/c}(2/eps_q)); history levels
// above L_q are stored as zero, so the shared reverse loop over L_max levels
// (Algorithm 1, Eq. sL) gives each column exactly its own sum over l <= L_q.
//
// Every column accumulates a row's entries one after another in index order
// (long rows: fixed 4096-entry segments, combined in segment order), whatever the
// tile shape: a column's result does not depend on which other columns share the
// batch nor on the tile chosen by the autotuner.
#include "common.cuh"
#include "internal.h"
#include "twofloat.cuh"

#include <math.h>

namespace esim {

namespace {

template <int CPL>
__device__ __forceinline__ void load_f(const float* __restrict__ p, float (&v)[CPL]) {
    if constexpr (CPL == 1) {
        v[0] = __ldg(p);
    } else if constexpr (CPL == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < CPL; i += 4) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p + i));
            v[i] = a.x; v[i + 1] = a.y; v[i + 2] = a.z; v[i + 3] = a.w;
        }
    }
}

template <int CPL>
__device__ __forceinline__ void load_f2(const float2* __restrict__ p, f2 (&v)[CPL]) {
    if constexpr (CPL == 1) {
        const float2 a = __ldg(p);
        v[0] = f2{a.x, a.y};
    } else {
#pragma unroll
        for (int i = 0; i < CPL; i += 2) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(p + i));
            v[i] = f2{a.x, a.y};
            v[i + 1] = f2{a.z, a.w};
        }
    }
}

// Row epilogue of the batched forward level l: pi^l = sqrt(c) * sum (zero above
// the column's L_q), x^l = pi^l / din.
struct BFwdOp {
    f2 sc;
    int level;
    const int32_t* __restrict__ Lq;  // W
    const uint32_t* __restrict__ in_rp;
    float* __restrict__ hist_l;  // n x W
    float* __restrict__ x_out;   // n x W
    int W;
    template <int CPL>
    __device__ __forceinline__ void operator()(int64_t row, int c0, const f2 (&acc)[CPL]) const {
        const uint32_t d = in_rp[row + 1] - in_rp[row];
        const float fd = (float)d;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const f2 p = f2_mul(acc[i], sc);
            float pf = __fadd_rn(p.hi, p.lo);
            if (level > Lq[c0 + i]) pf = 0.f;
            hist_l[row * W + c0 + i] = pf;
            x_out[row * W + c0 + i] = d ? __fdiv_rn(pf, fd) : 0.f;
        }
    }
};

// Row epilogue of the batched reverse level: s = sqrt(c) (P^T s_prev) + w pi^{L-l}.
// The last level writes FP64 into the query-major output s_out[q * n + row].
template <bool kFinal>
struct BRevOp {
    f2 sc;
    const uint32_t* __restrict__ rp;
    const float2* __restrict__ w;  // n x W
    const float* __restrict__ h;   // n x W (history level L_max - l)
    float2* __restrict__ s_next;   // n x W
    double* __restrict__ s_out;    // B x n
    int W;
    int B;
    int64_t n;
    template <int CPL>
    __device__ __forceinline__ void operator()(int64_t row, int c0, const f2 (&acc)[CPL]) const {
        const uint32_t d = rp[row + 1] - rp[row];
        const float fd = (float)d;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int q = c0 + i;
            f2 prop = f2{0.f, 0.f};
            if (d) prop = f2_div_f(f2_mul(acc[i], sc), fd);
            const float2 wv = w[row * W + q];
            const f2 s = f2_add(prop, f2_mul_f(f2{wv.x, wv.y}, h[row * W + q]));
            if (kFinal) {
                if (q < B) s_out[(int64_t)q * n + row] = f2_to_double(s);
            } else {
                s_next[row * W + q] = make_float2(s.hi, s.lo);
            }
        }
    }
};

// Short rows: LPR lanes per row, CPL columns per lane (W = LPR * CPL), entries of
// the row in order.  Blocks past short_blocks sum one segment of a long row per
// warp-group into partial[seg * W + column].
template <typename V, int LPR, int CPL, class Op>
__global__ void __launch_bounds__(kBlock) batch_rows_kernel(int64_t n, const uint32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col, const V* __restrict__ X,
                                                            uint32_t long_min, Op op, int64_t nseg,
                                                            const Segment* __restrict__ seg, f2* __restrict__ partial,
                                                            int short_blocks) {
    constexpr int W = LPR * CPL;
    constexpr int RPW = 32 / LPR;  // rows (or segments) per warp per iteration
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPR, cl = lane % LPR;
    const int c0 = cl * CPL;
    const bool segs = (int)blockIdx.x >= short_blocks;
    const int64_t nblk = segs ? (int64_t)gridDim.x - short_blocks : short_blocks;
    const int64_t blk = segs ? (int64_t)blockIdx.x - short_blocks : blockIdx.x;
    const int64_t warp = (blk * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (nblk * blockDim.x) >> 5;
    const int64_t items = segs ? nseg : n;
    for (int64_t base = warp * RPW; base < items; base += nwarps * RPW) {
        const int64_t it = base + sub;
        uint32_t b = 0, e = 0;
        bool mine = false;
        int64_t row = it;
        if (it < items) {
            if (segs) {
                const Segment sg = seg[it];
                b = sg.beg;
                e = sg.end;
                mine = true;
            } else {
                b = __ldg(rp + it);
                e = __ldg(rp + it + 1);
                mine = (e - b) < long_min;
                if (!mine) e = b;
            }
        }
        f2 acc[CPL];
#pragma unroll
        for (int i = 0; i < CPL; ++i) acc[i] = f2{0.f, 0.f};
        for (uint32_t p = b; p < e; ++p) {
            const int64_t j = __ldg(col + p);
            if constexpr (sizeof(V) == 4) {
                float v[CPL];
                load_f<CPL>(reinterpret_cast<const float*>(X) + j * W + c0, v);
#pragma unroll
                for (int i = 0; i < CPL; ++i) acc[i] = f2_add_f(acc[i], v[i]);
            } else {
                f2 v[CPL];
                load_f2<CPL>(reinterpret_cast<const float2*>(X) + j * W + c0, v);
#pragma unroll
                for (int i = 0; i < CPL; ++i) acc[i] = f2_add(acc[i], v[i]);
            }
        }
        if (!mine) continue;
        if (segs) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) partial[it * W + c0 + i] = acc[i];
        } else {
            op.template operator()<CPL>(row, c0, acc);
        }
    }
}

// Long rows: one lane per column combines the row's segment partials in order.
template <int W, class Op>
__global__ void __launch_bounds__(kBlock) batch_long_rows_kernel(int64_t nlong, const int32_t* __restrict__ long_rows,
                                                                 const int32_t* __restrict__ long_first,
                                                                 const f2* __restrict__ partial, Op op) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = t / W;
    const int q = (int)(t % W);
    if (r >= nlong) return;
    f2 acc[1] = {f2{0.f, 0.f}};
    for (int32_t s = long_first[r]; s < long_first[r + 1]; ++s) acc[0] = f2_add(acc[0], partial[(int64_t)s * W + q]);
    op.template operator()<1>(long_rows[r], q, acc);
}

// Level 0: pi^0 column q = (1 - sqrt c) e_{u_q}; x^0 = pi^0 / din.
__global__ void batch_forward_init_kernel(int64_t n, int W, int B, const int64_t* __restrict__ u, float a,
                                          const uint32_t* __restrict__ in_rp, float* __restrict__ hist0,
                                          float* __restrict__ x0) {
    const int64_t total = n * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / W;
        const int q = (int)(i % W);
        float p = 0.f, xv = 0.f;
        if (q < B && u[q] == row) {
            p = a;
            const uint32_t d = in_rp[row + 1] - in_rp[row];
            xv = d ? __fdiv_rn(a, (float)d) : 0.f;
        }
        hist0[i] = p;
        x0[i] = xv;
    }
}

// pi_q(k) = sum over levels (two-float), R_q(k) = ceil(R_b,q pi^2) (>= 1 where pi > 0)
// into the column-major R[q * n + k].  A block takes 32 nodes x W columns; a shared
// tile turns the node-major reads into column-major writes.
__global__ void __launch_bounds__(kBlock) batch_alloc_kernel(int64_t n, int W, int B, const float* __restrict__ hist,
                                                             int32_t Lmax, const double* __restrict__ Rb, int mode,
                                                             uint64_t* __restrict__ R, Status* __restrict__ st) {
    __shared__ unsigned long long tile[64][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const size_t level_stride = (size_t)n * W;
    bool overflow = false;
    for (int idx = threadIdx.x; idx < 32 * W; idx += blockDim.x) {
        const int kk = idx / W, q = idx % W;
        const int64_t k = k0 + kk;
        unsigned long long r = 0;
        if (k < n && q < B) {
            f2 p = f2{0.f, 0.f};
            for (int32_t l = 0; l <= Lmax; ++l) p = f2_add_f(p, hist[(size_t)l * level_stride + (size_t)k * W + q]);
            const double pd = f2_to_double(p);
            const double v = mode == 0 ? Rb[q] * (pd * pd) : Rb[q] * pd;
            if (v >= 9.2e18 || v != v) {
                overflow = true;
            } else {
                r = (unsigned long long)ceil(v);
                if (r == 0ull && pd > 0.0) r = 1ull;
            }
        }
        tile[q][kk] = r;
    }
    if (overflow) atomicOr(&st->err, kErrBudget);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * B; idx += blockDim.x) {
        const int q = idx / 32, kk = idx % 32;
        const int64_t k = k0 + kk;
        if (k < n) R[(int64_t)q * n + k] = tile[q][kk];
    }
}

// w = D^ / (1 - sqrt c) as two-floats, node-major (n x W), from the column-major D^;
// s^0 = w pi^{L_max} (two-float), or the FP64 output when L_max = 0.
__global__ void __launch_bounds__(kBlock) batch_reverse_init_kernel(int64_t n, int W, int B,
                                                                    const double* __restrict__ dhat, double inv_a,
                                                                    const float* __restrict__ hL, float2* __restrict__ w,
                                                                    float2* __restrict__ s0, double* __restrict__ s_out) {
    __shared__ double tile[64][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < 32 * B; idx += blockDim.x) {
        const int q = idx / 32, kk = idx % 32;
        const int64_t k = k0 + kk;
        tile[q][kk] = k < n ? dhat[(int64_t)q * n + k] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * W; idx += blockDim.x) {
        const int kk = idx / W, q = idx % W;
        const int64_t k = k0 + kk;
        if (k >= n) continue;
        const f2 wv = q < B ? f2_from_double(tile[q][kk] * inv_a) : f2{0.f, 0.f};
        w[k * W + q] = make_float2(wv.hi, wv.lo);
        const f2 s = f2_mul_f(wv, hL[k * W + q]);
        if (s_out) {
            if (q < B) s_out[(int64_t)q * n + k] = f2_to_double(s);
        } else {
            s0[k * W + q] = make_float2(s.hi, s.lo);
        }
    }
}

int grid_cap(const Graph& g, int64_t work, int64_t per_block) {
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)g.sm_count * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename V, int LPR, int CPL, class Op>
cudaError_t batch_level(const Graph& g, const DevCsr& A, const V* X, const Op& op, f2* partial) {
    constexpr int W = LPR * CPL;
    const int rows_per_block = (kBlock / 32) * (32 / LPR);
    const int sb = grid_cap(g, g.n, rows_per_block);
    const int segb = A.nseg ? grid_cap(g, A.nseg, rows_per_block) : 0;
    batch_rows_kernel<V, LPR, CPL, Op><<<(unsigned)(sb + segb), kBlock, 0, g.stream>>>(
        g.n, A.rp, A.col, X, A.long_min, op, A.nseg, A.seg, partial, sb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || A.nlong == 0) return e;
    const int64_t threads = A.nlong * W;
    batch_long_rows_kernel<W, Op><<<(unsigned)((threads + kBlock - 1) / kBlock), kBlock, 0, g.stream>>>(
        A.nlong, A.long_rows, A.long_first, partial, op);
    return cudaGetLastError();
}

}  // namespace

// Tile shapes: lanes per row (the rest of the columns go to each lane): for W >= 32
// the tiles are 32, 16 and 8 lanes per row; for W = 16 they are 16, 8 and 4.
int batch_tile_count() { return 3; }
int batch_tile_lpr(int tile) { return tile == 0 ? 32 : (tile == 1 ? 16 : 8); }

template <int W>
cudaError_t batch_level_dispatch_fwd(const Graph& g, int tile, const float* X, const BFwdOp& op, f2* partial) {
    constexpr int L0 = W >= 32 ? 32 : 16;
    switch (tile) {
        case 0: return batch_level<float, L0, W / L0>(g, g.out, X, op, partial);
        case 1: return batch_level<float, L0 / 2, W / (L0 / 2)>(g, g.out, X, op, partial);
        default: return batch_level<float, L0 / 4, W / (L0 / 4)>(g, g.out, X, op, partial);
    }
}

template <int W, bool kFinal>
cudaError_t batch_level_dispatch_rev(const Graph& g, int tile, const float2* S, const BRevOp<kFinal>& op, f2* partial) {
    constexpr int L0 = W >= 32 ? 32 : 16;
    switch (tile) {
        case 0: return batch_level<float2, L0, W / L0>(g, g.in, S, op, partial);
        case 1: return batch_level<float2, L0 / 2, W / (L0 / 2)>(g, g.in, S, op, partial);
        default: return batch_level<float2, L0 / 4, W / (L0 / 4)>(g, g.in, S, op, partial);
    }
}

cudaError_t launch_batch_forward_level(const Graph& g, int W, int tile, int level, double c, const int32_t* Lq,
                                       const float* x_prev, float* hist_l, float* x_next, void* partial) {
    const double sc = sqrt(c);
    const f2 sc2 = f2{(float)sc, (float)(sc - (double)(float)sc)};
    BFwdOp op{sc2, level, Lq, g.in.rp, hist_l, x_next, W};
    if (W == 16) return batch_level_dispatch_fwd<16>(g, tile, x_prev, op, (f2*)partial);
    if (W == 32) return batch_level_dispatch_fwd<32>(g, tile, x_prev, op, (f2*)partial);
    return batch_level_dispatch_fwd<64>(g, tile, x_prev, op, (f2*)partial);
}

cudaError_t launch_batch_reverse_level(const Graph& g, int W, int B, int tile, bool final_level, double c,
                                       const float2* w, const float* h, const float2* s_prev, float2* s_next,
                                       double* s_out, void* partial) {
    const double sc = sqrt(c);
    const f2 sc2 = f2{(float)sc, (float)(sc - (double)(float)sc)};
    if (final_level) {
        BRevOp<true> op{sc2, g.in.rp, w, h, nullptr, s_out, W, B, g.n};
        if (W == 16) return batch_level_dispatch_rev<16, true>(g, tile, s_prev, op, (f2*)partial);
        if (W == 32) return batch_level_dispatch_rev<32, true>(g, tile, s_prev, op, (f2*)partial);
        return batch_level_dispatch_rev<64, true>(g, tile, s_prev, op, (f2*)partial);
    }
    BRevOp<false> op{sc2, g.in.rp, w, h, s_next, nullptr, W, B, g.n};
    if (W == 16) return batch_level_dispatch_rev<16, false>(g, tile, s_prev, op, (f2*)partial);
    if (W == 32) return batch_level_dispatch_rev<32, false>(g, tile, s_prev, op, (f2*)partial);
    return batch_level_dispatch_rev<64, false>(g, tile, s_prev, op, (f2*)partial);
}

// ---------------------------------------------------------------- shared walks
//
// The walk spec keys pair r of node k by (seed, k, r) alone, so column q of a batch,
// which needs pairs 0 .. R_q(k)-1 of node k, sees the same pairs as every other
// column.  The batch therefore samples max_q R_q(k) pairs of each node once, cut at
// the distinct values of R_q(k) into intervals, and column q's count for node k is
// the sum of the intervals below R_q(k) -- the same integer as sampling alone.
// Segments are node-major: segment k*B + i is interval i of node k (zero length
// past the node's distinct counts).
__global__ void shared_plan_kernel(int64_t n, int B, const uint64_t* __restrict__ R, uint64_t* __restrict__ len,
                                   uint64_t* __restrict__ rbase) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t t[kBatchMax];
        int m = 0;
        for (int q = 0; q < B; ++q) {  // distinct non-zero R_q(k), ascending (insertion)
            const uint64_t v = R[(size_t)q * (size_t)n + (size_t)k];
            if (v == 0) continue;
            int i = m;
            while (i > 0 && t[i - 1] > v) --i;
            if (i > 0 && t[i - 1] == v) continue;
            for (int j = m; j > i; --j) t[j] = t[j - 1];
            t[i] = v;
            ++m;
        }
        uint64_t prev = 0;
        for (int i = 0; i < B; ++i) {
            const size_t sidx = (size_t)k * (size_t)B + (size_t)i;
            rbase[sidx] = prev;
            if (i < m) {
                len[sidx] = t[i] - prev;
                prev = t[i];
            } else {
                len[sidx] = 0;
            }
        }
    }
}

// nonmeet(q, k) = the counts of node k's intervals that end at or below R_q(k)
__global__ void shared_columns_kernel(int64_t n, int B, const uint64_t* __restrict__ R,
                                      const uint64_t* __restrict__ rbase, const uint64_t* __restrict__ soff,
                                      const uint64_t* __restrict__ scount, uint64_t* __restrict__ nonmeet) {
    const int64_t N = n * (int64_t)B;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = idx / n, k = idx % n;
        const uint64_t Rq = R[idx];
        uint64_t sum = 0;
        for (int i = 0; i < B; ++i) {
            const size_t sidx = (size_t)k * (size_t)B + (size_t)i;
            const uint64_t len = soff[sidx + 1] - soff[sidx];
            if (len == 0 || rbase[sidx] + len > Rq) break;
            sum += scount[sidx];
        }
        (void)q;
        nonmeet[idx] = sum;
    }
}

__global__ void dhat_from_R_kernel(int64_t N, const uint64_t* __restrict__ nonmeet, const uint64_t* __restrict__ R,
                                   double* __restrict__ dhat) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dhat[i] = R[i] ? (double)nonmeet[i] / (double)R[i] : 0.0;
}

cudaError_t launch_shared_plan(const Graph& g, int B, const uint64_t* R, uint64_t* len, uint64_t* rbase) {
    shared_plan_kernel<<<grid_cap(g, g.n, kBlock), kBlock, 0, g.stream>>>(g.n, B, R, len, rbase);
    return cudaGetLastError();
}

cudaError_t launch_shared_columns(const Graph& g, int B, const uint64_t* R, const uint64_t* rbase, const uint64_t* soff,
                                  const uint64_t* scount, uint64_t* nonmeet) {
    shared_columns_kernel<<<grid_cap(g, g.n * B, kBlock), kBlock, 0, g.stream>>>(g.n, B, R, rbase, soff, scount,
                                                                                  nonmeet);
    return cudaGetLastError();
}

cudaError_t launch_dhat_from_R(const Graph& g, int64_t N, const uint64_t* nonmeet, const uint64_t* R, double* dhat) {
    dhat_from_R_kernel<<<grid_cap(g, N, kBlock), kBlock, 0, g.stream>>>(N, nonmeet, R, dhat);
    return cudaGetLastError();
}

cudaError_t launch_batch_forward_init(const Graph& g, int W, int B, const int64_t* u, double c, float* hist0,
                                      float* x0) {
    const int blocks = grid_cap(g, g.n * W, kBlock);
    batch_forward_init_kernel<<<blocks, kBlock, 0, g.stream>>>(g.n, W, B, u, (float)(1.0 - sqrt(c)), g.in.rp, hist0, x0);
    return cudaGetLastError();
}

cudaError_t launch_batch_alloc(const Graph& g, int W, int B, const float* hist, int32_t Lmax, const double* Rb,
                               int mode, uint64_t* R) {
    const int64_t blocks = (g.n + 31) / 32;
    batch_alloc_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(g.n, W, B, hist, Lmax, Rb, mode, R, g.status);
    return cudaGetLastError();
}

cudaError_t launch_batch_reverse_init(const Graph& g, int W, int B, const double* dhat, double c, const float* hL,
                                      float2* w, float2* s0, double* s_out_if_final) {
    const int64_t blocks = (g.n + 31) / 32;
    batch_reverse_init_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(g.n, W, B, dhat, 1.0 / (1.0 - sqrt(c)), hL,
                                                                          w, s0, s_out_if_final);
    return cudaGetLastError();
}

}  // namespace esim
