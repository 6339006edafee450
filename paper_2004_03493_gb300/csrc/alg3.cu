// Algorithm 3 ("Improved method for estimating D(k,k)"), depth-limited: exact
// first-meeting probabilities Z_1..Z_d of node k (d <= 3) from Lemma 5, and the
// diagonal estimate that combines them with the tail walk pairs.
//
// With h_l = (P^T)^l(k, .) the distribution of a non-stop walk from k after l steps
// (dense FP64, by the pull sweep with no decay), C_j(q) = sum_x (P^T)^j(q, x)^2 the
// chance that two non-stop walks from q coincide at step j, and P~ the transition
// matrix with squared entries, Lemma 5 summed over q gives
//   Z_1 = c   * |h_1|^2
//   Z_2 = c^2 * (|h_2|^2 - <h_1^2, C_1>)
//   Z_3 = c^3 * (|h_3|^2 - <h_2^2 - P~ h_1^2, C_1> - sum_{q in I(k)} h_1(q)^2 C_2(q))
// On a graph without repeated in-edges C_1(q) = 1/din(q), h_1(q) = 1/din(k) on I(k),
// and (P~ v)(i) = sum_{j : i in I(j)} v(j) / din(j)^2.  C_2(q) of each in-neighbour q
// of k comes from two more sweeps from q.  Every sum uses fixed-order block
// partials, so the values are deterministic.
#include "common.cuh"
#include "internal.h"

#include <math.h>

#include <vector>

namespace esim {

namespace {

constexpr int kDotBlocks = 1024;

// partial[block] of sum_i a(i)^2 * w(i) (w = NULL: sum a(i)^2); kind 1: sum_i a(i) * w(i)
__global__ void __launch_bounds__(kBlock) wsum_kernel(int64_t n, const double* __restrict__ a,
                                                      const double* __restrict__ w, int kind,
                                                      double* __restrict__ partial) {
    __shared__ double red[kBlock / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        if (kind == 1) acc += v * w[i];
        else acc += w ? v * v * w[i] : v * v;
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

// x(j) = (v(j) / din(j))^2: the input of the squared-transition sweep
__global__ void sq_scale_kernel(int64_t n, const double* __restrict__ v, const double* __restrict__ inv_din,
                                double* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = v[i] * inv_din[i];
        x[i] = t * t;
    }
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
    double* H;        // 4 n: h_0 .. h_3 from k
    double* Hq;       // 3 n: h_0 .. h_2 from an in-neighbour of k
    double* xa;       // n
    double* xb;       // n
    double* t;        // n: P~ h_1^2
    double* x;        // n: sweep input
    double* partial;  // kDotBlocks
    double* sums;     // 16
};

A3Ws a3_layout(int64_t n_, void* base) {
    const size_t n = (size_t)n_;
    double* p = (double*)base;
    A3Ws w;
    w.H = p; p += 4 * n;
    w.Hq = p; p += 3 * n;
    w.xa = p; p += n;
    w.xb = p; p += n;
    w.t = p; p += n;
    w.x = p; p += n;
    w.partial = p; p += kDotBlocks;
    w.sums = p;
    return w;
}

cudaError_t wsum(const Graph& g, const double* a, const double* w, int kind, const A3Ws& ws, double* out_dev) {
    wsum_kernel<<<kDotBlocks, kBlock, 0, g.stream>>>(g.n, a, w, kind, ws.partial);
    sum_partials_kernel<<<1, 1024, 0, g.stream>>>(kDotBlocks, ws.partial, out_dev);
    return cudaGetLastError();
}

}  // namespace

size_t alg3_workspace_bytes(int64_t n) { return sizeof(double) * ((size_t)n * 11 + kDotBlocks + 16); }

cudaError_t alg3_first_meeting(const Graph& g, int64_t k, int depth, double c, void* wsp, double* z_out, int* launches) {
    const A3Ws ws = a3_layout(g.n, wsp);
    const int per_sweep = 1 + (g.out.nlong > 0 ? 1 : 0);
    int count = 1 + depth * per_sweep + 2;
    const size_t n = (size_t)g.n;
    cudaError_t e = launch_walk_distributions(g, k, depth, ws.H, ws.xa, ws.xb);
    if (e != cudaSuccess) return e;
    // sums: [0] |h_1|^2  [1] |h_2|^2  [2] <h_1^2, C_1>  [3] |h_3|^2  [4] <h_2^2, C_1>  [5] <P~ h_1^2, C_1>
    if ((e = wsum(g, ws.H + n, nullptr, 0, ws, ws.sums + 0)) != cudaSuccess) return e;
    if (depth >= 2) {
        if ((e = wsum(g, ws.H + 2 * n, nullptr, 0, ws, ws.sums + 1)) != cudaSuccess) return e;
        if ((e = wsum(g, ws.H + n, g.inv_din, 0, ws, ws.sums + 2)) != cudaSuccess) return e;
        count += 4;
    }
    if (depth >= 3) {
        if ((e = wsum(g, ws.H + 3 * n, nullptr, 0, ws, ws.sums + 3)) != cudaSuccess) return e;
        if ((e = wsum(g, ws.H + 2 * n, g.inv_din, 0, ws, ws.sums + 4)) != cudaSuccess) return e;
        sq_scale_kernel<<<eblocks(g, g.n), kBlock, 0, g.stream>>>(g.n, ws.H + n, g.inv_din, ws.x);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_pull_sum(g, ws.x, ws.t)) != cudaSuccess) return e;
        if ((e = wsum(g, ws.t, g.inv_din, 1, ws, ws.sums + 5)) != cudaSuccess) return e;
        count += 7 + per_sweep;
    }
    double sums[8] = {};
    if ((e = cudaMemcpyAsync(sums, ws.sums, sizeof(double) * 6, cudaMemcpyDeviceToHost, g.stream)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
    z_out[0] = c * sums[0];
    if (depth >= 2) z_out[1] = c * c * (sums[1] - sums[2]);
    if (depth >= 3) {
        uint32_t rp2[2];
        if ((e = cudaMemcpy(rp2, g.in.rp + k, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost)) != cudaSuccess) return e;
        const uint32_t beg = rp2[0], end = rp2[1];
        std::vector<int32_t> nbrs(end - beg);
        if (end > beg &&
            (e = cudaMemcpy(nbrs.data(), g.in.col + beg, sizeof(int32_t) * (end - beg), cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
            return e;
        const double dk = (double)(end - beg);
        double e3 = 0.0;
        for (int32_t q : nbrs) {
            if ((e = launch_walk_distributions(g, q, 2, ws.Hq, ws.xa, ws.xb)) != cudaSuccess) return e;
            if ((e = wsum(g, ws.Hq + 2 * n, nullptr, 0, ws, ws.sums + 8)) != cudaSuccess) return e;
            double c2 = 0.0;
            if ((e = cudaMemcpyAsync(&c2, ws.sums + 8, sizeof(double), cudaMemcpyDeviceToHost, g.stream)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(g.stream)) != cudaSuccess) return e;
            e3 += c2 / (dk * dk);
            count += 1 + 2 * per_sweep + 2;
        }
        z_out[2] = c * c * c * (sums[3] - (sums[4] - sums[5]) - e3);
    }
    if (launches) *launches += count;
    return cudaSuccess;
}

cudaError_t launch_dhat_alg3(const Graph& g, const uint64_t* counts, const uint64_t* off, const uint8_t* depth,
                             const double* zsum, double c, double* dhat) {
    dhat_alg3_kernel<<<eblocks(g, g.n), kBlock, 0, g.stream>>>(g.n, counts, off, depth, zsum, g.in.rp, c, dhat);
    return cudaGetLastError();
}

}  // namespace esim
