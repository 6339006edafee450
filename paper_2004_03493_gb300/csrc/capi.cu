// C ABI of the library (include/exactsim.h): graph loading, options, the whole
// query pipeline (Algorithm 1 with Algorithm 2 and the Lemma 4 allocation) and
// the step entry points.
#include "exactsim.h"
#include "internal.h"

#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

using namespace esim;

struct esim_graph {
    Graph g;
};

namespace {

thread_local std::string t_err;

esim_status fail(esim_status st, const std::string& msg) {
    t_err = msg;
    return st;
}

esim_status cuda_fail(cudaError_t e, const char* where) {
    return fail(ESIM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ESIM_CUDA_TRY(expr, where)                        \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

void free_csr(DevCsr& c) {
    cudaFree(c.rp);
    cudaFree(c.col);
    cudaFree(c.info);
    cudaFree(c.seg);
    cudaFree(c.long_rows);
    cudaFree(c.long_first);
    cudaFree(c.tiles);
    cudaFree(c.tseg);
    cudaFree(c.tlong_rows);
    cudaFree(c.tlong_first);
    c = DevCsr{};
}

int group_for(double avg_degree) {
    if (avg_degree <= 3.0) return 2;
    if (avg_degree <= 6.0) return 4;
    if (avg_degree <= 12.0) return 8;
    if (avg_degree <= 24.0) return 16;
    return 32;
}

constexpr uint32_t kSegLen = 4096;

// Upload a host CSR and build its row-split table.
esim_status upload_csr(int64_t n, const std::vector<uint32_t>& rp, const std::vector<int32_t>& col, DevCsr& d,
                       bool with_info, int sm_count) {
    const int64_t m = (int64_t)rp[n];
    d.group = group_for(n ? (double)m / (double)n : 1.0);
    d.long_min = std::max<uint32_t>(256u, 32u * (uint32_t)d.group);
    std::vector<Segment> seg;
    std::vector<int32_t> long_rows, long_first;
    for (int64_t r = 0; r < n; ++r) {
        const uint32_t b = rp[r], e = rp[r + 1];
        if (e - b < d.long_min) continue;
        long_rows.push_back((int32_t)r);
        long_first.push_back((int32_t)seg.size());
        const uint32_t first = (uint32_t)seg.size();
        for (uint32_t s = b; s < e; s += kSegLen) seg.push_back(Segment{(int32_t)r, s, std::min(e, s + kSegLen), first});
    }
    long_first.push_back((int32_t)seg.size());
    d.nseg = (int64_t)seg.size();
    d.nlong = (int64_t)long_rows.size();
    // tiles of the single-vector sweeps (one warp each): consecutive rows up to tile_cap
    // entries (and kSweepTileRows rows); a longer row forms a tile alone, and a row longer
    // than kSweepTile is cut into segments.  tile_cap is kSweepTile, or less on a small
    // graph so that its tiles still number about 256 per SM (a power of two, at least 64)
    d.tile_cap = kSweepTile;
    while (d.tile_cap > 64u && (int64_t)d.tile_cap * 256 * (int64_t)std::max(sm_count, 1) > m) d.tile_cap >>= 1;
    const uint32_t cap = d.tile_cap;
    std::vector<uint32_t> tiles{0};
    std::vector<Segment> tseg;
    std::vector<int32_t> tlong_rows, tlong_first;
    for (int64_t r = 0; r < n;) {
        const uint32_t len = rp[r + 1] - rp[r];
        if (len > cap && len <= kSweepTile) {  // a tile of its own (one warp still holds it)
            ++r;
        } else if (len > cap) {
            tlong_rows.push_back((int32_t)r);
            tlong_first.push_back((int32_t)tseg.size());
            const uint32_t first = (uint32_t)tseg.size();
            for (uint32_t s = rp[r]; s < rp[r + 1]; s += kSegLen)
                tseg.push_back(Segment{(int32_t)r, s, std::min(rp[r + 1], s + kSegLen), first});
            ++r;
        } else {
            const int64_t start = r;
            uint32_t cnt = 0;
            while (r < n && r - start < (int64_t)kSweepTileRows) {
                const uint32_t l = rp[r + 1] - rp[r];
                if (l > cap || cnt + l > cap) break;
                cnt += l;
                ++r;
            }
        }
        tiles.push_back((uint32_t)r);
    }
    tlong_first.push_back((int32_t)tseg.size());
    d.ntiles = (int64_t)tiles.size() - 1;
    d.tnseg = (int64_t)tseg.size();
    d.tnlong = (int64_t)tlong_rows.size();
    cudaError_t e;
    if ((e = dev_alloc(&d.rp, (size_t)n + 1)) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(rowptr)");
    if ((e = dev_alloc(&d.col, (size_t)m)) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(col)");
    if ((e = dev_alloc(&d.seg, seg.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(segments)");
    if ((e = dev_alloc(&d.long_rows, long_rows.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(long rows)");
    if ((e = dev_alloc(&d.long_first, long_first.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(long first)");
    ESIM_CUDA_TRY(cudaMemcpy(d.rp, rp.data(), sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice), "upload rowptr");
    if (m) ESIM_CUDA_TRY(cudaMemcpy(d.col, col.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice), "upload col");
    if (!seg.empty())
        ESIM_CUDA_TRY(cudaMemcpy(d.seg, seg.data(), sizeof(Segment) * seg.size(), cudaMemcpyHostToDevice), "upload segments");
    if ((e = dev_alloc(&d.tiles, tiles.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(tiles)");
    if ((e = dev_alloc(&d.tseg, tseg.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(tile segments)");
    if ((e = dev_alloc(&d.tlong_rows, tlong_rows.size())) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(tile long rows)");
    if ((e = dev_alloc(&d.tlong_first, tlong_first.size())) != cudaSuccess)
        return fail(ESIM_ENOMEM, "cudaMalloc(tile long first)");
    ESIM_CUDA_TRY(cudaMemcpy(d.tiles, tiles.data(), sizeof(uint32_t) * tiles.size(), cudaMemcpyHostToDevice), "upload tiles");
    if (!tseg.empty())
        ESIM_CUDA_TRY(cudaMemcpy(d.tseg, tseg.data(), sizeof(Segment) * tseg.size(), cudaMemcpyHostToDevice),
                      "upload tile segments");
    if (!tlong_rows.empty())
        ESIM_CUDA_TRY(cudaMemcpy(d.tlong_rows, tlong_rows.data(), sizeof(int32_t) * tlong_rows.size(),
                                 cudaMemcpyHostToDevice), "upload tile long rows");
    ESIM_CUDA_TRY(cudaMemcpy(d.tlong_first, tlong_first.data(), sizeof(int32_t) * tlong_first.size(),
                             cudaMemcpyHostToDevice), "upload tile long first");
    if (!long_rows.empty())
        ESIM_CUDA_TRY(cudaMemcpy(d.long_rows, long_rows.data(), sizeof(int32_t) * long_rows.size(), cudaMemcpyHostToDevice),
                      "upload long rows");
    ESIM_CUDA_TRY(cudaMemcpy(d.long_first, long_first.data(), sizeof(int32_t) * long_first.size(), cudaMemcpyHostToDevice),
                  "upload long first");
    if (with_info) {
        std::vector<uint2> info((size_t)n);
        for (int64_t r = 0; r < n; ++r) info[r] = make_uint2(rp[r], rp[r + 1] - rp[r]);
        if (dev_alloc(&d.info, (size_t)n) != cudaSuccess) return fail(ESIM_ENOMEM, "cudaMalloc(row info)");
        ESIM_CUDA_TRY(cudaMemcpy(d.info, info.data(), sizeof(uint2) * (size_t)n, cudaMemcpyHostToDevice), "upload row info");
    }
    return ESIM_OK;
}

size_t partial_count(const Graph& g) {
    return (size_t)std::max<int64_t>(1, std::max(std::max(g.in.nseg, g.out.nseg), std::max(g.in.tnseg, g.out.tnseg)));
}

void free_a3workers(Graph& g) {
    for (auto& wk : g.a3workers) {
        if (wk.stream) {
            cudaStreamSynchronize(wk.stream);
            cudaStreamDestroy(wk.stream);
        }
        cudaFree(wk.ws);
        cudaFree(wk.partial);
        cudaFree(wk.scan_part);
        cudaFree(wk.norm_part);
    }
    g.a3workers.clear();
    g.a3worker_ws_bytes = 0;
}

// Up to `extra` workers beside the query's stream; returns how many exist (fewer when
// the device cannot hold more: the computation then uses fewer, never fails for it).
int ensure_a3workers(Graph& g, int extra) {
    const size_t need = alg3_workspace_bytes(g);
    if (g.a3worker_ws_bytes < need) free_a3workers(g);
    const int64_t nb = allocate_blocks(g.n);
    while ((int)g.a3workers.size() < extra) {
        Graph::A3Worker wk;
        const bool ok = cudaStreamCreateWithFlags(&wk.stream, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaMalloc(&wk.ws, need) == cudaSuccess && dev_alloc(&wk.partial, partial_count(g)) == cudaSuccess &&
                        dev_alloc(&wk.scan_part, (size_t)nb) == cudaSuccess &&
                        dev_alloc(&wk.norm_part, 2 * (size_t)nb) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (wk.stream) cudaStreamDestroy(wk.stream);
            cudaFree(wk.ws);
            cudaFree(wk.partial);
            cudaFree(wk.scan_part);
            cudaFree(wk.norm_part);
            break;
        }
        g.a3workers.push_back(wk);
        g.a3worker_ws_bytes = need;
    }
    return std::min<int>(extra, (int)g.a3workers.size());
}

void release(Graph& g) {
    cudaSetDevice(g.device);
    // no work of this handle may still use its buffers: its own streams drain first (a
    // caller's stream set by esim_set_stream is the caller's to drain)
    if (g.own_stream) cudaStreamSynchronize(g.own_stream);
    if (g.side_stream) cudaStreamSynchronize(g.side_stream);
    free_a3workers(g);
    free_csr(g.in);
    free_csr(g.out);
    cudaFree(g.inv_din);
    cudaFree(g.din_magic);
    cudaFree(g.status);
    if (g.status_host) cudaFreeHost(g.status_host);
    cudaFree(g.ws);
    cudaFree(g.bws);
    cudaFree(g.a3ws);
    cudaFree(g.a3pws);
    cudaFree(g.zstage);
    cudaFree(g.partial);
    cudaFree(g.scan_part);
    cudaFree(g.norm_part);
    cudaFree(g.topk_ws);
    for (auto& ev : g.ev)
        if (ev) cudaEventDestroy(ev);
    if (g.own_stream) cudaStreamDestroy(g.own_stream);
    if (g.side_stream) cudaStreamDestroy(g.side_stream);
    for (auto& ev : g.side_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& ev : g.side_tev)
        if (ev) cudaEventDestroy(ev);
    g = Graph{};
}

size_t topk_stage_offset(int64_t n) { return (topk_workspace_bytes(n) + 255) / 256 * 256; }

bool valid_c_eps(double c, double eps) { return c > 0.0 && c < 1.0 && eps > 0.0 && eps < 1.0; }

double kappa_of(const Graph& g, double c) {
    if (g.kappa > 0.0) return g.kappa;
    const double a = 1.0 - sqrt(c);
    return 6.0 / (a * a * a * a);
}

// Query workspace (one device arena per graph handle, grown on demand).  The
// FP64 form uses hist/xa/xb; the FP32c form uses hist32/xa32/xb32 and the
// two-float buffers w/sa2/sb2.  Every buffer starts on a 256-byte boundary.
struct Ws {
    double* hist;      // (L+1) n  FP64 history
    double* xa;        // n        forward x, then reverse ping-pong (FP64)
    double* xb;        // n
    float* hist32;     // (L+1) n  FP32 history
    float* xa32;       // n
    float* xb32;       // n
    float2* w2;        // n        D^/a as two-floats
    float2* sa2;       // n        reverse ping-pong (two-float)
    float2* sb2;       // n
    double* pi;        // n
    uint64_t* R;       // n
    uint64_t* off;     // n+1
    uint64_t* nonmeet; // n
    double* dhat;      // n
    double* s;         // n
    uint8_t* depth;    // n  Algorithm 3 depth per node (0: Algorithm 2)
    double* zsum;      // n  Algorithm 3: sum of the exact Z_l(k)
    uint8_t* cand;     // n  Algorithm 3: 0 other node, 1 candidate walked after the plan, 2 early candidate
    uint64_t* R2;      // n  R of the side sampler's nodes, then of the other candidates
    uint64_t* off2;    // n+1  offsets of the side sampler's walks (read by the side stream)
    uint64_t* offc;    // n+1  offsets of the candidates' walks
    uint64_t* nm2;     // n  counts of the other nodes
    int32_t* cand_ids; // 4096
    PlanEntry* plan;   // 4096  the cost model's plan, staged for the scatter
    // sparse linearization (FP64): rolling pi^l, the running pi, the kept entries
    double* lev;       // n
    double* pirun;     // n
    SparseHist sh;     // cap entries, L+2 level ends
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Lay out the arena at `base` (or only measure it when base is null); returns bytes.
// Capacity of the sparse history: fewer than 1/theta entries exceed theta, because
// the pi^l(k) over all levels and nodes sum to at most 1 (pigeonhole, Section 3.2);
// never more than the dense (L+1) n.
uint64_t sparse_capacity(int64_t n, int32_t L, double theta) {
    const double bound = floor(1.000001 / theta) + 1.0;
    const double dense = (double)(L + 1) * (double)n;
    return (uint64_t)(bound < dense ? bound : dense);
}

size_t ws_layout(int64_t n_, int32_t L, int precision, char* base, Ws* w, uint64_t sparse_cap = 0) {
    const size_t n = (size_t)n_;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += round256(bytes);
        return p;
    };
    Ws t{};
    if (precision == 0 && sparse_cap > 0) {  // the entries themselves go last (see below)
        t.lev = (double*)take(8 * n);
        t.pirun = (double*)take(8 * n);
        t.xa = (double*)take(8 * n);
        t.xb = (double*)take(8 * n);
    } else if (precision == 0) {
        t.hist = (double*)take(8 * n * (size_t)(L + 1));
        t.xa = (double*)take(8 * n);
        t.xb = (double*)take(8 * n);
    } else {
        t.hist32 = (float*)take(4 * n * (size_t)(L + 1));
        t.xa32 = (float*)take(4 * n);
        t.xb32 = (float*)take(4 * n);
        t.w2 = (float2*)take(8 * n);
        t.sa2 = (float2*)take(8 * n);
        t.sb2 = (float2*)take(8 * n);
        t.xa = (double*)t.sa2;  // FP64 scratch for step calls that need one (aliases sa2)
        t.xb = (double*)t.sb2;
    }
    t.pi = (double*)take(8 * n);
    t.R = (uint64_t*)take(8 * n);
    t.off = (uint64_t*)take(8 * (n + 1));
    t.nonmeet = (uint64_t*)take(8 * n);
    t.dhat = (double*)take(8 * n);
    t.s = (double*)take(8 * n);
    t.depth = (uint8_t*)take(n);
    t.zsum = (double*)take(8 * n);
    t.cand = (uint8_t*)take(n);
    t.R2 = (uint64_t*)take(8 * n);
    t.off2 = (uint64_t*)take(8 * (n + 1));
    t.offc = (uint64_t*)take(8 * (n + 1));
    t.nm2 = (uint64_t*)take(8 * n);
    t.cand_ids = (int32_t*)take(4 * 4096);
    t.plan = (PlanEntry*)take(sizeof(PlanEntry) * 4096);
    if (precision == 0 && sparse_cap > 0) {
        // last, so that the layout for a smaller capacity is a prefix of this one
        t.sh.lvl = (uint64_t*)take(8 * (size_t)(L + 2));
        t.sh.idx = (int32_t*)take(4 * (size_t)sparse_cap);
        t.sh.val = (double*)take(8 * (size_t)sparse_cap);
        t.sh.cap = sparse_cap;
    }
    if (w) *w = t;
    return o;
}

esim_status ensure_ws(Graph& g, int32_t L, int precision, Ws& w, uint64_t sparse_cap = 0) {
    const size_t need = ws_layout(g.n, L, precision, nullptr, nullptr, sparse_cap);
    g.last_ws_bytes = need;
    if (need > g.ws_bytes) {
        cudaStreamSynchronize(g.stream);
        cudaFree(g.ws);
        g.ws = nullptr;
        g.ws_bytes = 0;
        if (cudaMalloc(&g.ws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ESIM_ENOMEM, "cudaMalloc(query workspace of " + std::to_string(need) + " bytes)");
        }
        g.ws_bytes = need;
    }
    ws_layout(g.n, L, precision, (char*)g.ws, &w, sparse_cap);
    return ESIM_OK;
}

esim_status check_graph(const esim_graph* h) {
    if (!h) return fail(ESIM_EINVAL, "graph handle is NULL");
    return ESIM_OK;
}

esim_status ensure_a3ws(Graph& g) {
    const size_t need = alg3_workspace_bytes(g);
    if (g.a3ws && g.a3ws_bytes >= need) return ESIM_OK;
    cudaStreamSynchronize(g.stream);
    cudaFree(g.a3ws);
    g.a3ws = nullptr;
    g.a3ws_bytes = 0;
    if (cudaMalloc(&g.a3ws, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(ESIM_ENOMEM, "cudaMalloc(Algorithm 3 workspace of " + std::to_string(need) + " bytes)");
    }
    g.a3ws_bytes = need;
    return ESIM_OK;
}

// Algorithm 3's depth choice under option alg3_rule = 1.  The paper grows l(k) until the
// explored edges reach 2 R(k) / sqrt(c), the walk work they replace.  Here the
// exploitation is done with dense sweeps, so the depth d of node k minimises an
// estimate of the GPU work, in walk pair-steps of the sampler:
//   walks      R_d (d + 1/(1-c)),  R_d = max(1, ceil(v c^(2d)))  (v = R_b pi(k)^2)
//   Lemma 5    2d-1 single-vector sweeps of m+n entries (h_1..h_d and the P~ sweeps);
//              sum_{i=1}^{d-4} |supp h_i| (d-i) probe column-sweeps for the deeper probe
//              levels; the last two probe levels (i = d-2 and d-3, two and three steps)
//              run one warp per node over its two- and three-hop neighbourhood and dense
//              probes only for the nodes too large for that, charged as
//              w_last (d-i) |supp h_i| column-sweeps; and the launches;
// d = 0 is Algorithm 2 alone.  The weights (options alg3_w_sweep, alg3_w_probe,
// alg3_w_launch, alg3_w_last: pair-steps per entry of a single sweep, per entry and
// column of a probe sweep, per launch, and the last level's share of a dense probe) are
// calibrated by timing whole queries on GB300.
double alg3_cost(int d, double v, double c, const uint64_t* supp, int64_t n, int64_t m, double w_sweep,
                 double w_probe, double w_launch, double w_last) {
    double r = d == 0 ? ceil(v) : ceil(v * pow(c, (double)(2 * d)));
    if (r < 1.0) r = 1.0;
    double cost = r * ((double)d + 1.0 / (1.0 - c));
    if (d > 0) {
        const double edges = (double)(m + n);
        uint64_t probe = 0, launches = 3 * (uint64_t)(2 * d - 1);
        for (int i = 1; i <= d - 4; ++i) {
            probe += supp[i] * (uint64_t)(d - i);
            launches += (supp[i] + 31) / 32 * (uint64_t)(3 * (d - i) + 2);
        }
        double last = 0.0;
        for (int i = std::max(1, d - 3); i <= d - 2; ++i) {
            last += w_last * ((double)(d - i) * (double)supp[i]);
            launches += 2;
        }
        cost += w_sweep * edges * (double)(2 * d - 1);
        cost += w_probe * edges * ((double)probe + last);
        cost += w_launch * (double)launches;
    }
    return cost;
}

// The depth of least estimated work, 0..max_depth (the first on ties).
int alg3_depth(double v, double c, const uint64_t* supp, int max_depth, int64_t n, int64_t m, double w_sweep,
               double w_probe, double w_launch, double w_last) {
    int d = 0;
    double best = alg3_cost(0, v, c, supp, n, m, w_sweep, w_probe, w_launch, w_last);
    for (int dd = 1; dd <= max_depth; ++dd) {
        const double cost = alg3_cost(dd, v, c, supp, n, m, w_sweep, w_probe, w_launch, w_last);
        if (cost < best) {
            best = cost;
            d = dd;
        }
    }
    return d;
}

// Algorithm 3 for the heaviest nodes (by pi, at most alg3_max_nodes, with din >= 2
// and an Algorithm 2 count of at least alg3_min_pairs): the depth by alg3_cost (at
// most alg3_max_depth), exact Z_1..Z_d (Lemma 5) on the GPU, and the pair count
// max(1, ceil(R_b pi(k)^2 c^(2d))) (pi(k) for the basic allocation): the tail
// estimator's variance and range are c^(2d) and c^d of Algorithm 2's.  Nodes with
// din <= 1 already got no pairs from the allocation.  Then the offsets are rescanned.
// The sampler on the side stream after the work queued so far on g.stream: offsets off,
// counts nm2, pair-steps to the status block's side counter; at most alg3_overlap
// blocks per SM, leaving room for the planning's kernels.  Records side_ev[1] at its end.
esim_status launch_side_walks(Graph& g, const Ws& w, const uint64_t* off, double c, uint64_t seed,
                              const uint8_t* depth) {
    ESIM_CUDA_TRY(cudaEventRecord(g.side_ev[0], g.stream), "record");
    ESIM_CUDA_TRY(cudaStreamWaitEvent(g.side_stream, g.side_ev[0], 0), "side wait");
    Graph view = g;
    view.stream = g.side_stream;
    view.sample_block_cap = g.alg3_overlap;
    if (g.timing) {
        for (auto& ev : g.side_tev)
            if (!ev) ESIM_CUDA_TRY(cudaEventCreate(&ev), "cudaEventCreate");
        cudaEventRecord(g.side_tev[0], g.side_stream);
    }
    ESIM_CUDA_TRY(launch_sample(view, off, c, seed, w.nm2, (uint64_t*)&g.status->pair_steps_side, depth),
                  "side walk pairs");
    if (g.timing) cudaEventRecord(g.side_tev[1], g.side_stream);
    ESIM_CUDA_TRY(cudaEventRecord(g.side_ev[1], g.side_stream), "record");
    return ESIM_OK;
}

// Starts, on the side stream, the walks of every node that is not an Algorithm 3
// candidate and of the early candidates (cand = 2), in one launch: their R(k) and depths
// are final, and the walk spec keys a pair by (seed, k, r), so splitting the nodes
// between sampler launches changes no count.  One launch, not one per group, so that
// the planning's kernels keep their share of every SM.
esim_status start_side_walks(Graph& g, const Ws& w, double c, uint64_t seed, int* launches) {
    ESIM_CUDA_TRY(launch_mask_R(g, w.R, w.cand, (1u << 0) | (1u << 2), w.R2), "side nodes' R");
    const int64_t nb = allocate_blocks(g.n);
    ESIM_CUDA_TRY(launch_scan_R(g, g.n, w.R2, w.off2, g.scan_part, nullptr, g.norm_part + nb, false), "side nodes' scan");
    esim_status st = launch_side_walks(g, w, w.off2, c, seed, w.depth);
    if (st != ESIM_OK) return st;
    *launches += 5;
    return ESIM_OK;
}

esim_status ensure_a3pws(Graph& g) {
    if (!alg3_paper_fits(g.n))
        return fail(ESIM_ENOTSUP, "the paper's Algorithm 3 depth rule keeps n x n support bit sets; n = " +
                                      std::to_string(g.n) + " is above its 4 GiB budget (option alg3_rule = 1 "
                                      "chooses depths by the cost model)");
    const size_t need = alg3_paper_bytes(g.n, kAlg3MaxDepth);
    if (g.a3pws && g.a3pws_bytes >= need) return ESIM_OK;
    cudaStreamSynchronize(g.stream);
    cudaFree(g.a3pws);
    g.a3pws = nullptr;
    g.a3pws_bytes = 0;
    if (cudaMalloc(&g.a3pws, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(ESIM_ENOMEM, "cudaMalloc(Algorithm 3 depth-rule workspace of " + std::to_string(need) + " bytes)");
    }
    g.a3pws_bytes = need;
    return ESIM_OK;
}

// zsum(k) = sum_{l <= depth(k)} Z_l(k) for the nodes of the given depths (every other
// entry 0): Z_1 = c/din(k) for every node of depth 1 in depth_dev, the closed form of
// depth 2 (alg3_paper.cu) for the nodes in d2, and Z_1..Z_d from alg3_first_meeting, one
// node at a time, for the nodes in deep and for the depth-2 nodes whose two-hop
// neighbourhood is too large for the closed form's table.  Synchronises g.stream.
esim_status alg3_zsums_of(Graph& g, const uint8_t* depth_dev, const std::vector<int32_t>& d2,
                          std::vector<std::pair<int32_t, int>> deep, double c, double* zsum, int* launches) {
    ESIM_CUDA_TRY(cudaMemsetAsync(zsum, 0, sizeof(double) * (size_t)g.n, g.stream), "reset zsum");
    ESIM_CUDA_TRY(alg3_paper_z1(g, depth_dev, c, zsum), "Algorithm 3 Z_1");
    *launches += 1;
    if (!d2.empty()) {
        const int cnt = (int)d2.size();
        const size_t need = round256(4 * d2.size()) + 8 * d2.size();  // ids, then the gathered values
        if (g.zstage_bytes < need) {
            cudaStreamSynchronize(g.stream);
            cudaFree(g.zstage);
            g.zstage = nullptr;
            g.zstage_bytes = 0;
            const size_t want = round256(4 * (size_t)g.n) + 8 * (size_t)g.n;
            if (cudaMalloc(&g.zstage, want) != cudaSuccess) {
                cudaGetLastError();
                return fail(ESIM_ENOMEM, "cudaMalloc(Algorithm 3 staging of " + std::to_string(want) + " bytes)");
            }
            g.zstage_bytes = want;
        }
        int32_t* stage_ids = (int32_t*)g.zstage;
        double* stage_vals = (double*)((char*)g.zstage + round256(4 * d2.size()));
        std::vector<double> v2((size_t)cnt);
        ESIM_CUDA_TRY(cudaMemcpyAsync(stage_ids, d2.data(), sizeof(int32_t) * d2.size(), cudaMemcpyHostToDevice,
                                      g.stream),
                      "upload depth-2 nodes");
        ESIM_CUDA_TRY(alg3_paper_z2(g, stage_ids, cnt, c, zsum), "Algorithm 3 Z_1 + Z_2");
        ESIM_CUDA_TRY(alg3_gather_f64(g, stage_ids, cnt, zsum, stage_vals), "gather depth-2 terms");
        ESIM_CUDA_TRY(cudaMemcpyAsync(v2.data(), stage_vals, sizeof(double) * d2.size(), cudaMemcpyDeviceToHost,
                                      g.stream),
                      "copy depth-2 terms");
        ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "Algorithm 3 depth-2 terms");  // d2 and v2 are locals
        *launches += 2;
        for (int i = 0; i < cnt; ++i)
            if (v2[(size_t)i] != v2[(size_t)i]) deep.emplace_back(d2[(size_t)i], 2);  // NaN: too large
    }
    if (!deep.empty()) {
        esim_status a3 = ensure_a3ws(g);
        if (a3 != ESIM_OK) return a3;
        // Each node's Lemma 5 computation waits on the host between its levels (the next
        // level's probe count); workers on their own streams take nodes from a shared
        // counter, so one node's waits leave the GPU to the others.  A node's result does
        // not depend on the worker that computes it.
        const int want = std::max(1, std::min<int>(g.alg3_workers, (int)deep.size()));
        const int nw = 1 + (want > 1 ? ensure_a3workers(g, want - 1) : 0);
        std::vector<double> zs(deep.size());
        std::atomic<size_t> next{0};
        std::vector<cudaError_t> errs((size_t)nw, cudaSuccess);
        std::vector<int> counts((size_t)nw, 0);
        auto run = [&](int wi) {
            Graph view = g;
            void* ws = g.a3ws;
            if (wi > 0) {
                const Graph::A3Worker& wk = g.a3workers[(size_t)wi - 1];
                if ((errs[(size_t)wi] = cudaSetDevice(g.device)) != cudaSuccess) return;
                view.stream = wk.stream;
                view.partial = wk.partial;
                view.scan_part = wk.scan_part;
                view.norm_part = wk.norm_part;
                ws = wk.ws;
            }
            for (;;) {
                const size_t i = next.fetch_add(1);
                if (i >= deep.size()) return;
                const int d = deep[i].second;
                double z[kAlg3MaxDepth] = {};
                const cudaError_t e = alg3_first_meeting(view, deep[i].first, d, c, ws, z, &counts[(size_t)wi]);
                if (e != cudaSuccess) {
                    errs[(size_t)wi] = e;
                    next.store(deep.size());  // the others stop after their current node
                    return;
                }
                double sum = 0.0;
                for (int j = 0; j < d; ++j) sum += z[j];
                zs[i] = sum;
            }
        };
        std::vector<std::thread> threads;
        for (int wi = 1; wi < nw; ++wi) threads.emplace_back(run, wi);
        run(0);
        for (auto& t : threads) t.join();
        for (int wi = 0; wi < nw; ++wi) {
            ESIM_CUDA_TRY(errs[(size_t)wi], "Algorithm 3 first meetings");
            *launches += counts[(size_t)wi];
        }
        for (size_t i = 0; i < deep.size(); ++i)
            ESIM_CUDA_TRY(cudaMemcpyAsync(zsum + deep[i].first, &zs[i], sizeof(double), cudaMemcpyHostToDevice,
                                          g.stream),
                          "set zsum");
        ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "Algorithm 3 plan");  // zs is a local
    }
    return ESIM_OK;
}

// The same from a device depth array alone (every node): the host reads it back and
// lists the nodes.  Returns the number of nodes with depth >= 1 in *used.
esim_status alg3_zsums(Graph& g, const uint8_t* depth_dev, double c, double* zsum, int* launches, int* used_out) {
    std::vector<uint8_t> depth((size_t)g.n);
    ESIM_CUDA_TRY(cudaMemcpyAsync(depth.data(), depth_dev, (size_t)g.n, cudaMemcpyDeviceToHost, g.stream), "copy depth");
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "Algorithm 3 depths");
    std::vector<int32_t> d2;
    std::vector<std::pair<int32_t, int>> deep;
    int used = 0;
    for (int64_t k = 0; k < g.n; ++k) {
        const int d = depth[(size_t)k];
        if (d == 0) continue;
        ++used;
        if (d == 2) d2.push_back((int32_t)k);
        else if (d > 2) deep.emplace_back((int32_t)k, d);
    }
    *used_out = used;
    return alg3_zsums_of(g, depth_dev, d2, std::move(deep), c, zsum, launches);
}

// Algorithm 3 with the paper's adaptive depth: every node with R(k) > 0 (din >= 2; the
// allocation gave the others none) explores until its explored edges reach
// 2 R(k)/sqrt(c), at most alg3_max_depth levels (alg3_paper.cu); it keeps its R(k)
// pairs, which move without the continuation draw for depth(k) steps; then the sums of
// its exact Z (alg3_zsums).
esim_status plan_alg3_paper(Graph& g, const Ws& w, double c, int* launches, uint64_t seed, bool* side) {
    esim_status a3 = ensure_a3pws(g);
    if (a3 != ESIM_OK) return a3;
    ESIM_CUDA_TRY(alg3_paper_depths(g, w.R, c, g.alg3_max_depth, g.a3pws, w.depth, launches),
                  "Algorithm 3 depths (explored edges)");
    // Every node's walks are final now (the allocation's R(k) and offsets, the depths):
    // with a side stream they all run there while the first-meeting sums are computed,
    // and the main stream's candidate launch is empty (cand = 0 everywhere).
    if (g.side_stream && g.alg3_overlap > 0) {
        ESIM_CUDA_TRY(cudaMemsetAsync(w.cand, 0, (size_t)g.n, g.stream), "reset candidates");
        esim_status st = launch_side_walks(g, w, w.off, c, seed, w.depth);
        if (st != ESIM_OK) return st;
        g.side_candidates = 0;
        *side = true;
        *launches += 1;
    }
    int used = 0;
    a3 = alg3_zsums(g, w.depth, c, w.zsum, launches, &used);
    if (a3 != ESIM_OK) return a3;
    g.last_alg3_nodes = used;
    return ESIM_OK;
}

esim_status plan_alg3(Graph& g, const Ws& w, double c, double R_b, int* launches, uint64_t seed, bool* side) {
    if (g.has_duplicates) return fail(ESIM_ENOTSUP, "Algorithm 3 needs a graph without repeated in-edges");
    *side = false;
    if (g.alg3_rule == 0) return plan_alg3_paper(g, w, c, launches, seed, side);
    esim_status a3 = ensure_a3ws(g);
    if (a3 != ESIM_OK) return a3;
    ESIM_CUDA_TRY(cudaMemsetAsync(w.depth, 0, (size_t)g.n, g.stream), "reset depth");
    const int K = (int)std::min<int64_t>(g.alg3_max_nodes, g.n);
    char* stage = (char*)g.topk_ws + topk_stage_offset(g.n);
    double* vals_d = (double*)stage;
    int32_t* ids_d = (int32_t*)(stage + sizeof(double) * kTopkMax);
    ESIM_CUDA_TRY(launch_topk(g, w.pi, -1, K, ids_d, vals_d, g.topk_ws), "Algorithm 3 node selection");
    *launches += 27;
    std::vector<int32_t> ids((size_t)K);
    std::vector<double> pis((size_t)K);
    ESIM_CUDA_TRY(cudaMemcpyAsync(ids.data(), ids_d, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, g.stream), "copy ids");
    ESIM_CUDA_TRY(cudaMemcpyAsync(pis.data(), vals_d, sizeof(double) * K, cudaMemcpyDeviceToHost, g.stream), "copy pi");
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "Algorithm 3 node selection");
    const std::vector<uint32_t>& din = *g.din_host;
    // candidates: the heaviest nodes with din >= 2 and enough Algorithm 2 pairs
    std::vector<int32_t> cand;
    std::vector<double> cand_v;
    for (int i = 0; i < K; ++i) {
        const int32_t kk = ids[i];
        const double p = pis[i];
        if (kk < 0 || !(p > 0.0)) break;
        if (din[kk] < 2) continue;
        const double v = g.alloc_mode == 0 ? R_b * (p * p) : R_b * p;
        double r0 = ceil(v);
        if (r0 < 1.0) r0 = 1.0;
        if (r0 < g.alg3_min_pairs) continue;
        cand.push_back(kk);
        cand_v.push_back(v);
    }
    // The budget applies to the pairs actually drawn: drop the verdict on the
    // Algorithm 2 counts (no other error can be raised before the walks); the side
    // sampler judges the other nodes' pairs and the rescan below all of them.
    ESIM_CUDA_TRY(cudaMemsetAsync((char*)g.status + offsetof(Status, err), 0, sizeof(int), g.stream), "reset budget");
    g.side_candidates = 0;
    *side = !cand.empty() && g.side_stream && g.alg3_overlap > 0;
    if (*side) {  // cand = 1 for the candidates (2 for the early ones below)
        ESIM_CUDA_TRY(cudaMemsetAsync(w.cand, 0, (size_t)g.n, g.stream), "reset candidates");
        ESIM_CUDA_TRY(cudaMemcpyAsync(w.cand_ids, cand.data(), sizeof(int32_t) * cand.size(), cudaMemcpyHostToDevice,
                                      g.stream),
                      "upload candidates");
        ESIM_CUDA_TRY(launch_mark(g, w.cand_ids, (int)cand.size(), w.cand), "mark candidates");
        *launches += 1;
    }
    const int levels = std::max(0, g.alg3_max_depth - 2);
    std::vector<uint64_t> supps(cand.size() * (kAlg3MaxDepth + 1), 0);
    if (!cand.empty())
        ESIM_CUDA_TRY(alg3_supports(g, cand.data(), (int)cand.size(), levels, g.a3ws, supps.data(), launches),
                      "Algorithm 3 supports");
    // The cost model picks each depth from the supports alone, so every plan is final
    // before any first-meeting term is computed: R(k) and depth(k) go to the device at
    // once, and the walks of the other nodes and of the candidates with at least
    // alg3_early_pairs pairs start on the side stream while the terms are computed.
    std::vector<PlanEntry> plan;
    std::vector<int32_t> d2;
    std::vector<std::pair<int32_t, int>> deep;
    int used = 0, n_early = 0;
    for (size_t ci = 0; ci < cand.size(); ++ci) {
        const int32_t kk = cand[ci];
        const double v = cand_v[ci];
        const uint64_t* supp = supps.data() + ci * (kAlg3MaxDepth + 1);
        const int d = alg3_depth(v, c, supp, g.alg3_max_depth, g.n, g.m, g.alg3_w_sweep, g.alg3_w_probe,
                                 g.alg3_w_launch, g.alg3_w_last);
        double r = d >= 1 ? ceil(v * pow(c, (double)(2 * d))) : ceil(v);
        if (r < 1.0) r = 1.0;
        if (r >= 1.8e19) r = 1.8e19;  // the rescan's budget check reports it
        PlanEntry e{};
        e.k = kk;
        e.depth = (uint8_t)std::max(0, d);
        e.early = (uint8_t)(*side && r >= g.alg3_early_pairs ? 1 : 0);
        e.R = (uint64_t)r;
        if (!e.depth && !e.early) continue;
        plan.push_back(e);
        n_early += e.early;
        if (d >= 1) ++used;
        if (d == 2) d2.push_back(kk);
        else if (d > 2) deep.emplace_back(kk, d);
    }
    if (!plan.empty()) {
        ESIM_CUDA_TRY(cudaMemcpyAsync(w.plan, plan.data(), sizeof(PlanEntry) * plan.size(), cudaMemcpyHostToDevice,
                                      g.stream),
                      "upload the plan");
        ESIM_CUDA_TRY(launch_plan_scatter(g, w.plan, (int)plan.size(), w.R, w.depth, w.cand), "scatter the plan");
        *launches += 1;
    }
    g.side_candidates = n_early;
    if (*side) {
        esim_status ss = start_side_walks(g, w, c, seed, launches);
        if (ss != ESIM_OK) return ss;
    }
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "Algorithm 3 plan");  // plan is a local
    esim_status zs = alg3_zsums_of(g, w.depth, d2, std::move(deep), c, w.zsum, launches);
    if (zs != ESIM_OK) return zs;
    g.last_alg3_nodes = used;
    const int64_t nb = allocate_blocks(g.n);
    ESIM_CUDA_TRY(launch_scan_R(g, g.n, w.R, w.off, g.scan_part, nullptr, g.norm_part + nb), "Algorithm 3 rescan");
    *launches += 3;
    return ESIM_OK;
}

// Runs the whole query; s_dev may be NULL (the workspace holds s); k > 0 adds top-k.
esim_status run_query(Graph& g, int64_t u, double c, double eps, uint64_t seed, double* s_dev, int32_t k,
                      int32_t* ids_dev, double* vals_dev, double* s_host, int32_t* ids_host, double* vals_host) {
    if (u < 0 || u >= g.n) return fail(ESIM_EINVAL, "source node out of range");
    if (!valid_c_eps(c, eps)) return fail(ESIM_EINVAL, "need 0 < c < 1 and 0 < eps < 1");
    if (k > kTopkMax) return fail(ESIM_ENOTSUP, "k above 4096");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    // sparse linearization (Section 3.2): the query runs at eps/2 and drops the
    // history entries pi^l(k) <= (1 - sqrt c)^2 eps/2, which adds at most eps/2
    const bool sparse = g.sparse_hist && g.precision == 0;
    const double eps_q = sparse ? 0.5 * eps : eps;
    const int32_t L = esim_levels(c, eps_q);
    const double kappa = kappa_of(g, c);
    const double R_b = kappa * log((double)g.n) / (eps_q * eps_q);
    const double a_c = 1.0 - sqrt(c);
    const double theta = a_c * a_c * eps_q;
    Ws w;
    uint64_t cap = 0;
    int count_launches = 0;
    if (sparse) {
        // counting pass: the forward sweeps once without storing, then a workspace
        // sized to the kept entries (never above the pigeonhole bound)
        esim_status st0 = ensure_ws(g, L, 0, w, 1);
        if (st0 != ESIM_OK) return st0;
        ESIM_CUDA_TRY(cudaMemsetAsync(g.status, 0, sizeof(Status), g.stream), "reset status");
        const SparseHist none{nullptr, nullptr, nullptr, 0};
        ESIM_CUDA_TRY(launch_forward_sparse(g, u, c, L, theta, none, w.lev, w.pirun, w.xa, w.xb),
                      "forward sweeps (counting pass)");
        ESIM_CUDA_TRY(cudaMemcpyAsync(g.status_host, g.status, sizeof(Status), cudaMemcpyDeviceToHost, g.stream),
                      "copy status");
        ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "forward sweeps (counting pass)");
        const uint64_t kept = g.status_host->hist_count;
        cap = std::max<uint64_t>(1, std::min<uint64_t>(kept, sparse_capacity(g.n, L, theta)));
        count_launches = 2 + L * (2 + (g.out.nlong > 0 ? 1 : 0));
    }
    esim_status st = ensure_ws(g, L, g.precision, w, cap);
    if (st != ESIM_OK) return st;
    double* s = s_dev ? s_dev : w.s;
    if (g.timing)
        for (auto& ev : g.ev)
            if (!ev) ESIM_CUDA_TRY(cudaEventCreate(&ev), "cudaEventCreate");
    ESIM_CUDA_TRY(cudaMemsetAsync(g.status, 0, sizeof(Status), g.stream), "reset status");
    if (g.timing) cudaEventRecord(g.ev[0], g.stream);
    if (sparse)
        ESIM_CUDA_TRY(launch_forward_sparse(g, u, c, L, theta, w.sh, w.lev, w.pirun, w.xa, w.xb),
                      "forward sweeps (sparse history)");
    else if (g.precision == 0) ESIM_CUDA_TRY(launch_forward(g, u, c, L, w.hist, w.xa, w.xb), "forward sweeps");
    else ESIM_CUDA_TRY(launch_forward32(g, u, c, L, w.hist32, w.xa32, w.xb32), "forward sweeps (FP32c)");
    if (g.timing) cudaEventRecord(g.ev[1], g.stream);
    // kernels of the allocation, sampling and D^ phases (the default counts 3 + 1 + 1)
    int extra_launches = 0;
    bool side_used = false;
    g.last_alg3_nodes = 0;
    if (g.diag_mode == 1) {
        // ParSim's approximation D = (1-c) I: no allocation and no walk pairs
        if (g.timing) {
            cudaEventRecord(g.ev[2], g.stream);
            cudaEventRecord(g.ev[6], g.stream);
            cudaEventRecord(g.ev[7], g.stream);
            cudaEventRecord(g.ev[3], g.stream);
        }
        ESIM_CUDA_TRY(launch_fill(g, g.n, 1.0 - c, w.dhat), "dhat (ParSim)");
        extra_launches -= 4;
    } else {
        if (sparse)  // pi was summed level by level during the forward sweeps
            ESIM_CUDA_TRY(launch_allocate(g, w.pirun, 0, R_b, g.alloc_mode, w.pi, w.R, w.off), "allocation");
        else if (g.precision == 0)
            ESIM_CUDA_TRY(launch_allocate(g, w.hist, L, R_b, g.alloc_mode, w.pi, w.R, w.off), "allocation");
        else
            ESIM_CUDA_TRY(launch_allocate32(g, w.hist32, L, R_b, g.alloc_mode, w.pi, w.R, w.off),
                          "allocation (FP32c)");
        bool side = false;
        if (g.alg3) {
            esim_status a3 = plan_alg3(g, w, c, R_b, &extra_launches, seed, &side);
            if (a3 != ESIM_OK) {
                if (side) cudaStreamSynchronize(g.side_stream);  // no walks left running into the next query
                return a3;
            }
        }
        if (g.timing) cudaEventRecord(g.ev[2], g.stream);
        if (side) {
            // the remaining candidates' walks here; the side stream's counts for the rest
            ESIM_CUDA_TRY(launch_mask_R(g, w.R, w.cand, 1u << 1, w.R2), "candidates' R");
            ESIM_CUDA_TRY(launch_scan_R(g, g.n, w.R2, w.offc, g.scan_part, nullptr, g.norm_part + allocate_blocks(g.n),
                                        false),
                          "candidates' scan");
            if (g.timing) cudaEventRecord(g.ev[6], g.stream);
            ESIM_CUDA_TRY(launch_sample(g, w.offc, c, seed, w.nonmeet, nullptr, w.depth), "candidates' walk pairs");
            if (g.timing) cudaEventRecord(g.ev[7], g.stream);
            ESIM_CUDA_TRY(cudaStreamWaitEvent(g.stream, g.side_ev[1], 0), "wait for the side walks");
            ESIM_CUDA_TRY(launch_merge_counts(g, w.cand, w.nm2, w.nonmeet), "merge counts");
            extra_launches += 5;
        } else {
            if (g.timing) cudaEventRecord(g.ev[6], g.stream);
            ESIM_CUDA_TRY(launch_sample(g, w.off, c, seed, w.nonmeet, nullptr, g.alg3 ? w.depth : nullptr),
                          "walk pairs");
            if (g.timing) cudaEventRecord(g.ev[7], g.stream);
        }
        side_used = side;
        if (g.timing) cudaEventRecord(g.ev[3], g.stream);
        if (g.alg3)
            ESIM_CUDA_TRY(launch_dhat_alg3(g, w.nonmeet, w.off, w.depth, w.zsum, c, w.dhat), "dhat (Algorithm 3)");
        else ESIM_CUDA_TRY(launch_dhat(g, w.nonmeet, w.off, w.dhat), "dhat");
    }
    if (sparse)
        ESIM_CUDA_TRY(launch_reverse_sparse(g, w.sh, L, c, w.dhat, s, w.xa), "reverse sweeps (sparse history)");
    else if (g.precision == 0)
        ESIM_CUDA_TRY(launch_reverse(g, w.hist, L, c, w.dhat, s, w.xa, w.xb), "reverse sweeps");
    else
        ESIM_CUDA_TRY(launch_reverse32(g, w.hist32, L, c, w.dhat, s, w.w2, w.sa2, w.sb2), "reverse sweeps (FP32c)");
    if (g.timing) cudaEventRecord(g.ev[4], g.stream);
    if (k > 0) {
        int32_t* ids = ids_dev;
        double* vals = vals_dev;
        if (!ids) {  // host outputs: stage behind the top-k workspace
            char* stage = (char*)g.topk_ws + topk_stage_offset(g.n);
            vals = (double*)stage;
            ids = (int32_t*)(stage + sizeof(double) * kTopkMax);
        }
        ESIM_CUDA_TRY(launch_topk(g, s, g.exclude_source ? u : -1, k, ids, vals, g.topk_ws), "top-k");
        if (ids_host) {
            ESIM_CUDA_TRY(cudaMemcpyAsync(ids_host, ids, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, g.stream),
                          "copy ids");
            ESIM_CUDA_TRY(cudaMemcpyAsync(vals_host, vals, sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, g.stream),
                          "copy scores");
        }
    }
    if (g.timing) cudaEventRecord(g.ev[5], g.stream);
    if (s_host)
        ESIM_CUDA_TRY(cudaMemcpyAsync(s_host, s, sizeof(double) * (size_t)g.n, cudaMemcpyDeviceToHost, g.stream),
                      "copy scores");
    ESIM_CUDA_TRY(cudaMemcpyAsync(g.status_host, g.status, sizeof(Status), cudaMemcpyDeviceToHost, g.stream),
                  "copy status");
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "query");
    const Status hs = *g.status_host;
    g.last_L = L;
    // kernels launched: forward init + per level (rows [+ long rows]), 3 allocation
    // kernels, the sampler, D^, reverse init + per level, and 27 for top-k
    // the sparse history's sweeps sum in FP64 on the row kernel (long-row table nlong), the
    // others on the tile kernel (tnlong)
    const int fwd_per = 1 + (sparse ? (g.out.nlong > 0) : (g.out.tnlong > 0));
    const int rev_per = 1 + (sparse ? (g.in.nlong > 0) : (g.in.tnlong > 0));
    g.last_launches = (1 + L * fwd_per) + 3 + 1 + 1 + (1 + L * rev_per) + (k > 0 ? 27 : 0) + extra_launches;
    if (sparse) g.last_launches += 2 * (L + 1) + count_launches;  // compactions, scatters, counting pass
    g.last_hist_entries = sparse ? std::min<uint64_t>(hs.hist_count, cap) : (uint64_t)(L + 1) * (uint64_t)g.n;
    g.last_R_b = R_b;
    g.last_kappa = kappa;
    g.last_norm2 = hs.pi_norm2;
    g.last_sum_R = hs.sum_R;
    g.last_steps = hs.pair_steps + (side_used ? hs.pair_steps_side : 0ull);
    g.last_steps_side = side_used ? hs.pair_steps_side : 0ull;
    for (float& x : g.last_ms) x = 0.f;
    g.last_ms_kernel = g.last_ms_side = 0.f;
    g.last_side_candidates = side_used ? g.side_candidates : 0;
    if (g.timing) {
        for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&g.last_ms[i], g.ev[i], g.ev[i + 1]);
        cudaEventElapsedTime(&g.last_ms[5], g.ev[0], g.ev[5]);
        cudaEventElapsedTime(&g.last_ms_kernel, g.ev[6], g.ev[7]);
        if (side_used) cudaEventElapsedTime(&g.last_ms_side, g.side_tev[0], g.side_tev[1]);
    }
    if (hs.err & kErrBudget)
        return fail(ESIM_EBUDGET, "sum of R(k) = " + std::to_string((double)hs.sum_R) + " exceeds the pair budget");
    if (hs.err & kErrTimeout) return fail(ESIM_ETIMEOUT, "device wait timed out");
    if (hs.err & kErrCapacity) return fail(ESIM_ENOMEM, "sparse history above its capacity");
    return ESIM_OK;
}


// ---------------------------------------------------------------- batches

// Batch workspace (its own arena).
struct BWs {
    float* hist;      // (Lmax+1) n W
    float* xa;        // n W
    float* xb;        // n W
    float2* w;        // n W
    float2* sa;       // n W
    float2* sb;       // n W
    void* partial;    // nseg_max W two-floats
    uint64_t* R;      // B n
    uint64_t* off;    // B n + 1
    uint64_t* nonmeet;// B n
    uint64_t* rbase;  // B n  shared walks: first pair of each (node, interval) segment
    uint64_t* scount; // B n  shared walks: interval lengths, then interval counts
    double* dhat;     // B n
    double* s;        // B n
    int64_t* u;       // W
    int32_t* L;       // W
    double* Rb;       // W
    unsigned long long* part_R;  // tiles of B n
    double* part_norm;
    double* part_Rd;
    void* topk;       // batched top-k state
    int32_t* ids;     // B k (staging)
    double* vals;     // B k
};

size_t bws_layout(int64_t n_, int W, int B, int32_t Lmax, int64_t nseg_max, int k, char* base, BWs* out) {
    const size_t n = (size_t)n_, nw = n * (size_t)W, bn = n * (size_t)B;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + o : nullptr;
        o += round256(bytes);
        return p;
    };
    BWs t{};
    t.hist = (float*)take(4 * nw * (size_t)(Lmax + 1));
    t.xa = (float*)take(4 * nw);
    t.xb = (float*)take(4 * nw);
    t.w = (float2*)take(8 * nw);
    t.sa = (float2*)take(8 * nw);
    t.sb = (float2*)take(8 * nw);
    t.partial = take(8 * (size_t)std::max<int64_t>(1, nseg_max) * (size_t)W);
    t.R = (uint64_t*)take(8 * bn);
    t.off = (uint64_t*)take(8 * (bn + 1));
    t.nonmeet = (uint64_t*)take(8 * bn);
    t.rbase = (uint64_t*)take(8 * bn);
    t.scount = (uint64_t*)take(8 * bn);
    t.dhat = (double*)take(8 * bn);
    t.s = (double*)take(8 * bn);
    t.u = (int64_t*)take(8 * W);
    t.L = (int32_t*)take(4 * W);
    t.Rb = (double*)take(8 * W);
    const size_t nb = (size_t)allocate_blocks((int64_t)bn);
    t.part_R = (unsigned long long*)take(8 * nb);
    t.part_norm = (double*)take(8 * nb);
    t.part_Rd = (double*)take(8 * nb);
    t.topk = take(topk_batch_workspace_bytes(B));
    t.ids = (int32_t*)take(4 * (size_t)B * (size_t)std::max(k, 1));
    t.vals = (double*)take(8 * (size_t)B * (size_t)std::max(k, 1));
    if (out) *out = t;
    return o;
}

// Autotune: time each tile shape on one forward and one reverse level of the live
// batch (the results are identical for every tile, so the timing runs are harmless).
esim_status tune_batch_tiles(Graph& g, const Graph& view, int W, int B, double c, const BWs& w) {
    const int wi = batch_wi(W);
    if (g.batch_tile_force >= 0) {
        g.batch_tile_fwd[wi] = g.batch_tile_rev[wi] = g.batch_tile_force;
        return ESIM_OK;
    }
    if (g.batch_tile_fwd[wi] >= 0) return ESIM_OK;
    cudaEvent_t e0, e1;
    ESIM_CUDA_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    ESIM_CUDA_TRY(cudaEventCreate(&e1), "cudaEventCreate");
    const size_t nw = (size_t)g.n * W;
    float best_f = 1e30f, best_r = 1e30f;
    for (int t = 0; t < batch_tile_count(); ++t) {
        for (int rep = 0; rep < 2; ++rep) {  // first run warms up
            cudaEventRecord(e0, view.stream);
            ESIM_CUDA_TRY(launch_batch_forward_level(view, W, t, 1, c, w.L, w.xa, w.hist + nw, w.xb, w.partial),
                          "batch tune forward");
            cudaEventRecord(e1, view.stream);
            ESIM_CUDA_TRY(cudaEventSynchronize(e1), "batch tune");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1) {
                g.batch_tune_ms[wi][0][t] = ms;
                if (ms < best_f) { best_f = ms; g.batch_tile_fwd[wi] = t; }
            }
            cudaEventRecord(e0, view.stream);
            ESIM_CUDA_TRY(launch_batch_reverse_level(view, W, B, t, false, c, w.w, w.hist, w.sa, w.sb, nullptr,
                                                     w.partial),
                          "batch tune reverse");
            cudaEventRecord(e1, view.stream);
            ESIM_CUDA_TRY(cudaEventSynchronize(e1), "batch tune");
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1) {
                g.batch_tune_ms[wi][1][t] = ms;
                if (ms < best_r) { best_r = ms; g.batch_tile_rev[wi] = t; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ESIM_OK;
}

esim_status run_batch(Graph& g, int32_t B, const int64_t* u, const double* eps, uint64_t seed, double c,
                      double* s_dev, double* s_host, int32_t k, int32_t* ids_dev, double* vals_dev, int32_t* ids_host,
                      double* vals_host) {
    BatchPlan plan;
    esim_status st = (esim_status)batch_plan(g, B, u, eps, c, k, &plan);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    const size_t need = batch_ws_bytes(g, plan);
    if (need > g.bws_bytes) {
        cudaStreamSynchronize(g.stream);
        cudaFree(g.bws);
        g.bws = nullptr;
        g.bws_bytes = 0;
        if (cudaMalloc(&g.bws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ESIM_ENOMEM, "cudaMalloc(batch workspace of " + std::to_string(need) + " bytes)");
        }
        g.bws_bytes = need;
    }
    if (g.timing)
        for (auto& ev : g.ev)
            if (!ev) ESIM_CUDA_TRY(cudaEventCreate(&ev), "cudaEventCreate");
    st = (esim_status)batch_enqueue(g, g, plan, g.bws, seed, c, s_dev, s_host, ids_dev, vals_dev, ids_host, vals_host,
                                   true);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "batch query");
    const Status hs = *g.status_host;
    g.last_L = plan.Lmax;
    g.last_launches = 1 + plan.Lmax * (1 + (g.out.nlong > 0 ? 1 : 0)) + 1 + 3 + 1 + 1 + 1 +
                      plan.Lmax * (1 + (g.in.nlong > 0 ? 1 : 0)) + (k > 0 ? 27 : 0) + (g.shared_walks ? 2 : 0);
    g.last_R_b = plan.Rb[0];
    g.last_kappa = kappa_of(g, c);
    g.last_norm2 = 0.0;
    g.last_sum_R = hs.sum_R;
    g.last_steps = hs.pair_steps;
    for (float& x : g.last_ms) x = 0.f;
    g.last_ms_kernel = g.last_ms_side = 0.f;
    g.last_side_candidates = 0;
    g.last_steps_side = 0;
    if (g.timing) {
        for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&g.last_ms[i], g.ev[i], g.ev[i + 1]);
        cudaEventElapsedTime(&g.last_ms[5], g.ev[0], g.ev[5]);
        g.last_ms_kernel = g.last_ms[2];
    }
    if (hs.err & kErrBudget)
        return fail(ESIM_EBUDGET, "sum of R(k) = " + std::to_string((double)hs.sum_R) + " exceeds the pair budget");
    return ESIM_OK;
}

}  // namespace

int esim::set_error(int status, const std::string& message) {
    t_err = message;
    return status;
}

namespace esim {

Graph* graph_of(::esim_graph* h) { return &h->g; }

int batch_width(int B) { return B <= 16 ? 16 : (B <= 32 ? 32 : 64); }
int batch_wi(int W) { return W == 16 ? 0 : (W == 32 ? 1 : 2); }

int batch_plan(const Graph& g, int32_t B, const int64_t* u, const double* eps, double c, int32_t k, BatchPlan* plan) {
    if (B < 1) return fail(ESIM_EINVAL, "need B >= 1");
    if (B > kBatchMax) return fail(ESIM_ENOTSUP, "B above 64: split the batch");
    if (!u || !eps) return fail(ESIM_EINVAL, "NULL u or eps");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (k > kTopkMax) return fail(ESIM_ENOTSUP, "k above 4096");
    BatchPlan p{};
    p.B = B;
    p.W = batch_width(B);
    p.k = k;
    p.Lmax = 0;
    for (int q = 0; q < kBatchMax; ++q) {
        p.Lq[q] = -1;
        p.Rb[q] = 0.0;
        p.u[q] = -1;
    }
    for (int q = 0; q < B; ++q) {
        if (u[q] < 0 || u[q] >= g.n) return fail(ESIM_EINVAL, "source node out of range");
        if (!valid_c_eps(c, eps[q])) return fail(ESIM_EINVAL, "need 0 < eps < 1");
        p.Lq[q] = esim_levels(c, eps[q]);
        p.Rb[q] = kappa_of(g, c) * log((double)g.n) / (eps[q] * eps[q]);
        p.u[q] = u[q];
        p.Lmax = std::max(p.Lmax, p.Lq[q]);
    }
    *plan = p;
    return ESIM_OK;
}

size_t batch_ws_bytes(const Graph& g, const BatchPlan& p) {
    return bws_layout(g.n, p.W, p.B, p.Lmax, std::max(g.in.nseg, g.out.nseg), p.k, nullptr, nullptr);
}

// Enqueue the whole batch on view.stream using the arena `ws`; results go to the
// given device or host buffers (host copies are asynchronous).  The status block
// view.status is reset first and copied to view.status_host last.
int batch_enqueue(Graph& tuner, const Graph& view, const BatchPlan& p, void* ws, uint64_t seed, double c,
                  double* s_dev, double* s_host, int32_t* ids_dev, double* vals_dev, int32_t* ids_host,
                  double* vals_host, bool allow_tune) {
    BWs w;
    bws_layout(view.n, p.W, p.B, p.Lmax, std::max(view.in.nseg, view.out.nseg), p.k, (char*)ws, &w);
    const int W = p.W, B = p.B, k = p.k;
    const int32_t Lmax = p.Lmax;
    const size_t nw = (size_t)view.n * W;
    const int64_t N = view.n * (int64_t)B;
    const cudaStream_t stream = view.stream;
    const bool timing = view.timing && view.ev[0];
    ESIM_CUDA_TRY(cudaMemsetAsync(view.status, 0, sizeof(Status), stream), "reset status");
    ESIM_CUDA_TRY(cudaMemcpyAsync(w.u, p.u, sizeof(int64_t) * W, cudaMemcpyHostToDevice, stream), "upload sources");
    ESIM_CUDA_TRY(cudaMemcpyAsync(w.L, p.Lq, sizeof(int32_t) * W, cudaMemcpyHostToDevice, stream), "upload depths");
    ESIM_CUDA_TRY(cudaMemcpyAsync(w.Rb, p.Rb, sizeof(double) * W, cudaMemcpyHostToDevice, stream), "upload R_b");
    if (timing) cudaEventRecord(view.ev[0], stream);
    ESIM_CUDA_TRY(launch_batch_forward_init(view, W, B, w.u, c, w.hist, w.xa), "batch forward init");
    const int wi = batch_wi(W);
    if (Lmax >= 1 && allow_tune) {
        esim_status ts = (esim_status)tune_batch_tiles(tuner, view, W, B, c, w);
        if (ts != ESIM_OK) return ts;
    }
    const int tf = tuner.batch_tile_fwd[wi] < 0 ? 0 : tuner.batch_tile_fwd[wi];
    const int tr = tuner.batch_tile_rev[wi] < 0 ? 0 : tuner.batch_tile_rev[wi];
    float* x[2] = {w.xa, w.xb};
    for (int32_t l = 1; l <= Lmax; ++l)
        ESIM_CUDA_TRY(launch_batch_forward_level(view, W, tf, l, c, w.L, x[(l - 1) & 1], w.hist + (size_t)l * nw,
                                                 x[l & 1], w.partial),
                      "batch forward level");
    if (timing) cudaEventRecord(view.ev[1], stream);
    ESIM_CUDA_TRY(launch_batch_alloc(view, W, B, w.hist, Lmax, w.Rb, view.alloc_mode, w.R), "batch allocation");
    if (view.shared_walks) {
        // one walk set per node: intervals between the distinct R_q(k), sampled once
        ESIM_CUDA_TRY(launch_shared_plan(view, B, w.R, w.scount, w.rbase), "shared walk plan");
        ESIM_CUDA_TRY(launch_scan_R(view, N, w.scount, w.off, w.part_R, w.part_norm, w.part_Rd), "shared walk scan");
        if (timing) cudaEventRecord(view.ev[2], stream);
        ESIM_CUDA_TRY(launch_sample_segments(view, N, w.off, c, seed, w.scount, nullptr, nullptr, B, w.rbase),
                      "batch walk pairs (shared)");
        if (timing) cudaEventRecord(view.ev[3], stream);
        ESIM_CUDA_TRY(launch_shared_columns(view, B, w.R, w.rbase, w.off, w.scount, w.nonmeet), "shared walk counts");
        ESIM_CUDA_TRY(launch_dhat_from_R(view, N, w.nonmeet, w.R, w.dhat), "batch dhat");
    } else {
        ESIM_CUDA_TRY(launch_scan_R(view, N, w.R, w.off, w.part_R, w.part_norm, w.part_Rd), "batch scan");
        if (timing) cudaEventRecord(view.ev[2], stream);
        ESIM_CUDA_TRY(launch_sample_segments(view, N, w.off, c, seed, w.nonmeet, nullptr), "batch walk pairs");
        if (timing) cudaEventRecord(view.ev[3], stream);
        ESIM_CUDA_TRY(launch_dhat_segments(view, N, w.nonmeet, w.off, w.dhat), "batch dhat");
    }
    double* s = s_dev ? s_dev : w.s;
    ESIM_CUDA_TRY(launch_batch_reverse_init(view, W, B, w.dhat, c, w.hist + (size_t)Lmax * nw, w.w, w.sa,
                                            Lmax == 0 ? s : nullptr),
                  "batch reverse init");
    float2* sb[2] = {w.sa, w.sb};
    for (int32_t l = 1; l <= Lmax; ++l)
        ESIM_CUDA_TRY(launch_batch_reverse_level(view, W, B, tr, l == Lmax, c, w.w, w.hist + (size_t)(Lmax - l) * nw,
                                                 sb[(l - 1) & 1], sb[l & 1], s, w.partial),
                      "batch reverse level");
    if (timing) cudaEventRecord(view.ev[4], stream);
    if (k > 0) {
        int32_t* ids = ids_dev ? ids_dev : w.ids;
        double* vals = vals_dev ? vals_dev : w.vals;
        ESIM_CUDA_TRY(launch_topk_batch(view, B, s, view.exclude_source ? w.u : nullptr, k, ids, vals, w.topk),
                      "batch top-k");
        if (ids_host) {
            ESIM_CUDA_TRY(cudaMemcpyAsync(ids_host, ids, sizeof(int32_t) * (size_t)B * k, cudaMemcpyDeviceToHost,
                                          stream), "copy ids");
            ESIM_CUDA_TRY(cudaMemcpyAsync(vals_host, vals, sizeof(double) * (size_t)B * k, cudaMemcpyDeviceToHost,
                                          stream), "copy scores");
        }
    }
    if (timing) cudaEventRecord(view.ev[5], stream);
    if (s_host)
        ESIM_CUDA_TRY(cudaMemcpyAsync(s_host, s, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, stream),
                      "copy scores");
    ESIM_CUDA_TRY(cudaMemcpyAsync(view.status_host, view.status, sizeof(Status), cudaMemcpyDeviceToHost, stream),
                  "copy status");
    return ESIM_OK;
}

}  // namespace esim

extern "C" {

const char* esim_version(void) { return "exactsim-gb300 0.1 (sm_103a)"; }

const char* esim_last_error(void) { return t_err.c_str(); }

int32_t esim_levels(double c, double eps) {
    if (!valid_c_eps(c, eps)) return -1;
    return (int32_t)ceil(log(2.0 / eps) / log(1.0 / c));
}

double esim_sample_base(int64_t n, double c, double eps, double kappa) {
    if (n < 1 || !valid_c_eps(c, eps)) return -1.0;
    if (kappa <= 0.0) {
        const double a = 1.0 - sqrt(c);
        kappa = 6.0 / (a * a * a * a);
    }
    return kappa * log((double)n) / (eps * eps);
}

uint32_t esim_walk_threshold(double c) { return walk_threshold(c); }

esim_status esim_load_graph(int64_t n, const int64_t* in_rowptr, const int32_t* in_col, esim_graph** out) {
    if (!out) return fail(ESIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t)1 << 31) return fail(ESIM_EINVAL, "need 1 <= n < 2^31");
    if (!in_rowptr) return fail(ESIM_EINVAL, "in_rowptr is NULL");
    if (in_rowptr[0] != 0) return fail(ESIM_EINVAL, "in_rowptr[0] must be 0");
    for (int64_t j = 0; j < n; ++j)
        if (in_rowptr[j + 1] < in_rowptr[j]) return fail(ESIM_EINVAL, "in_rowptr is not non-decreasing");
    const int64_t m = in_rowptr[n];
    if (m >= ((int64_t)1 << 32) - 4096) return fail(ESIM_EINVAL, "need m < 2^32 - 4096");
    if (m > 0 && !in_col) return fail(ESIM_EINVAL, "in_col is NULL");
    for (int64_t p = 0; p < m; ++p)
        if (in_col[p] < 0 || (int64_t)in_col[p] >= n) return fail(ESIM_EINVAL, "in_col entry out of range");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice (no usable CUDA device)");
    cudaDeviceProp prop;
    ESIM_CUDA_TRY(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");

    esim_graph* h = new (std::nothrow) esim_graph();
    if (!h) return fail(ESIM_ENOMEM, "host allocation");
    Graph& g = h->g;
    g.device = dev;
    g.sm_count = prop.multiProcessorCount;
    g.n = n;
    g.m = m;

    // host: 32-bit in-CSR, and the out-CSR by a stable counting sort (rows of the
    // out-CSR list targets j in increasing order)
    std::vector<uint32_t> in_rp((size_t)n + 1), out_rp((size_t)n + 1, 0);
    for (int64_t j = 0; j <= n; ++j) in_rp[j] = (uint32_t)in_rowptr[j];
    std::vector<int32_t> in_c(in_col, in_col + m), out_c((size_t)m);
    for (int64_t p = 0; p < m; ++p) out_rp[(size_t)in_col[p] + 1]++;
    for (int64_t i = 0; i < n; ++i) out_rp[i + 1] += out_rp[i];
    {
        std::vector<uint32_t> cur(out_rp.begin(), out_rp.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t p = in_rowptr[j]; p < in_rowptr[j + 1]; ++p) out_c[cur[in_col[p]]++] = (int32_t)j;
    }
    {
        // repeated in-edges (Algorithm 3 needs a simple graph) and the host in-degrees
        std::vector<int64_t> mark((size_t)n, -1);
        auto din = std::make_shared<std::vector<uint32_t>>((size_t)n);
        for (int64_t j = 0; j < n && !g.has_duplicates; ++j)
            for (int64_t p = in_rowptr[j]; p < in_rowptr[j + 1]; ++p) {
                if (mark[in_col[p]] == j) {
                    g.has_duplicates = true;
                    break;
                }
                mark[in_col[p]] = j;
            }
        for (int64_t j = 0; j < n; ++j) (*din)[j] = (uint32_t)(in_rowptr[j + 1] - in_rowptr[j]);
        g.din_host = din;
    }
    {
        std::vector<double> inv((size_t)n);
        for (int64_t j = 0; j < n; ++j) {
            const int64_t d = in_rowptr[j + 1] - in_rowptr[j];
            inv[j] = d ? 1.0 / (double)d : 0.0;
        }
        std::vector<unsigned long long> magic((size_t)n);
        for (int64_t j = 0; j < n; ++j) {
            const int64_t d = in_rowptr[j + 1] - in_rowptr[j];
            magic[j] = d >= 2 ? ~0ull / (unsigned long long)d : 0ull;
        }
        if (dev_alloc(&g.inv_din, (size_t)n) != cudaSuccess ||
            cudaMemcpy(g.inv_din, inv.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
            dev_alloc(&g.din_magic, (size_t)n) != cudaSuccess ||
            cudaMemcpy(g.din_magic, magic.data(), sizeof(unsigned long long) * (size_t)n, cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            release(g);
            delete h;
            return fail(ESIM_ENOMEM, "device allocation for 1/din");
        }
    }
    esim_status st = upload_csr(n, in_rp, in_c, g.in, true, g.sm_count);
    if (st == ESIM_OK) st = upload_csr(n, out_rp, out_c, g.out, false, g.sm_count);
    if (st != ESIM_OK) {
        release(g);
        delete h;
        return st;
    }
    const int64_t nb = allocate_blocks(n);
    const size_t npart = partial_count(g);
    bool ok = dev_alloc(&g.status, 1) == cudaSuccess && cudaMallocHost((void**)&g.status_host, sizeof(Status)) == cudaSuccess &&
              dev_alloc(&g.partial, npart) == cudaSuccess && dev_alloc(&g.scan_part, (size_t)nb) == cudaSuccess &&
              dev_alloc(&g.norm_part, 2 * (size_t)nb) == cudaSuccess &&
              cudaMalloc(&g.topk_ws, topk_stage_offset(n) + (sizeof(double) + sizeof(int32_t)) * kTopkMax) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g.own_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g.side_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.side_ev[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.side_ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(g);
        delete h;
        return fail(ESIM_ENOMEM, "device allocation for graph workspace");
    }
    g.scan_blocks = nb;
    g.stream = g.own_stream;
    cudaMemset(g.status, 0, sizeof(Status));
    *out = h;
    return ESIM_OK;
}

void esim_free_graph(esim_graph* h) {
    if (!h) return;
    release(h->g);
    delete h;
}

int64_t esim_num_nodes(const esim_graph* h) { return h ? h->g.n : -1; }
int64_t esim_num_edges(const esim_graph* h) { return h ? h->g.m : -1; }

esim_status esim_set_stream(esim_graph* h, void* stream) {
    if (check_graph(h)) return ESIM_EINVAL;
    h->g.stream = stream ? (cudaStream_t)stream : h->g.own_stream;
    return ESIM_OK;
}

esim_status esim_set_option(esim_graph* h, const char* key, double value) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!key) return fail(ESIM_EINVAL, "option key is NULL");
    Graph& g = h->g;
    const std::string k(key);
    if (k == "kappa") {
        if (!(value == value)) return fail(ESIM_EINVAL, "kappa is NaN");
        g.kappa = value;
    } else if (k == "alloc") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "alloc must be 0 (pi^2) or 1 (basic)");
        g.alloc_mode = (int)value;
    } else if (k == "exclude_source") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "exclude_source must be 0 or 1");
        g.exclude_source = (int)value;
    } else if (k == "pair_budget") {
        if (!(value >= 0.0)) return fail(ESIM_EINVAL, "pair_budget must be >= 0");
        g.pair_budget = value;
    } else if (k == "timing") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "timing must be 0 or 1");
        g.timing = (int)value;
    } else if (k == "batch_tile") {
        if (value != -1.0 && value != 0.0 && value != 1.0 && value != 2.0)
            return fail(ESIM_EINVAL, "batch_tile must be -1 (autotune), 0, 1 or 2");
        g.batch_tile_force = (int)value;
        for (int i = 0; i < 3; ++i) g.batch_tile_fwd[i] = g.batch_tile_rev[i] = -1;
    } else if (k == "precision") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "precision must be 0 (FP64) or 1 (FP32c)");
        if (value == 1.0 && g.sparse_hist) return fail(ESIM_ENOTSUP, "sparse_hist needs precision 0 (FP64)");
        g.precision = (int)value;
    } else if (k == "shared_walks") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "shared_walks must be 0 or 1");
        g.shared_walks = (int)value;
    } else if (k == "sparse_hist") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "sparse_hist must be 0 or 1");
        if (value == 1.0 && g.precision != 0) return fail(ESIM_ENOTSUP, "sparse_hist needs precision 0 (FP64)");
        g.sparse_hist = (int)value;
    } else if (k == "diag") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "diag must be 0 (estimated) or 1 (ParSim (1-c) I)");
        g.diag_mode = (int)value;
    } else if (k == "alg3") {
        if (value != 0.0 && value != 1.0) return fail(ESIM_EINVAL, "alg3 must be 0 or 1");
        if (value == 1.0 && g.has_duplicates)
            return fail(ESIM_ENOTSUP, "Algorithm 3 needs a graph without repeated in-edges");
        g.alg3 = (int)value;
    } else if (k == "alg3_rule") {
        if (value != 0.0 && value != 1.0)
            return fail(ESIM_EINVAL, "alg3_rule must be 0 (the paper's explored-edge rule) or 1 (cost model)");
        g.alg3_rule = (int)value;
    } else if (k == "alg3_max_depth") {
        if (!(value >= 1.0 && value <= (double)kAlg3MaxDepth) || value != floor(value))
            return fail(ESIM_EINVAL, "alg3_max_depth must be an integer in [1, 16]");
        g.alg3_max_depth = (int)value;
    } else if (k == "alg3_min_pairs") {
        if (!(value >= 0.0)) return fail(ESIM_EINVAL, "alg3_min_pairs must be >= 0");
        g.alg3_min_pairs = value;
    } else if (k == "alg3_w_last") {
        if (!(value >= 0.0)) return fail(ESIM_EINVAL, "alg3_w_last must be >= 0");
        g.alg3_w_last = value;
    } else if (k == "alg3_w_sweep" || k == "alg3_w_probe" || k == "alg3_w_launch") {
        if (!(value >= 0.0)) return fail(ESIM_EINVAL, k + " must be >= 0");
        (k == "alg3_w_sweep" ? g.alg3_w_sweep : k == "alg3_w_probe" ? g.alg3_w_probe : g.alg3_w_launch) = value;
    } else if (k == "alg3_early_pairs") {
        if (!(value >= 1.0)) return fail(ESIM_EINVAL, "alg3_early_pairs must be >= 1");
        g.alg3_early_pairs = value;
    } else if (k == "alg3_push_div") {
        if (!(value >= 1.0 && value <= 1e6) || value != floor(value))
            return fail(ESIM_EINVAL, "alg3_push_div must be an integer in [1, 1e6]");
        g.alg3_push_div = (int)value;
    } else if (k == "alg3_overlap") {
        if (!(value >= 0.0 && value <= 64.0) || value != floor(value))
            return fail(ESIM_EINVAL, "alg3_overlap must be an integer in [0, 64]");
        g.alg3_overlap = (int)value;
    } else if (k == "alg3_workers") {
        if (!(value >= 1.0 && value <= 16.0) || value != floor(value))
            return fail(ESIM_EINVAL, "alg3_workers must be an integer in [1, 16]");
        g.alg3_workers = (int)value;
    } else if (k == "alg3_max_nodes") {
        if (!(value >= 1.0 && value <= 4096.0)) return fail(ESIM_EINVAL, "alg3_max_nodes must be in [1, 4096]");
        g.alg3_max_nodes = (int)value;
    } else {
        return fail(ESIM_EINVAL, "unknown option '" + k + "'");
    }
    return ESIM_OK;
}

esim_status esim_get_option(const esim_graph* h, const char* key, double* value) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!key || !value) return fail(ESIM_EINVAL, "NULL argument");
    const Graph& g = h->g;
    const std::string k(key);
    if (k == "kappa") *value = g.kappa;
    else if (k == "alloc") *value = g.alloc_mode;
    else if (k == "exclude_source") *value = g.exclude_source;
    else if (k == "pair_budget") *value = g.pair_budget;
    else if (k == "timing") *value = g.timing;
    else if (k == "precision") *value = g.precision;
    else if (k == "diag") *value = g.diag_mode;
    else if (k == "sparse_hist") *value = g.sparse_hist;
    else if (k == "shared_walks") *value = g.shared_walks;
    else if (k == "alg3") *value = g.alg3;
    else if (k == "alg3_rule") *value = g.alg3_rule;
    else if (k == "alg3_max_depth") *value = g.alg3_max_depth;
    else if (k == "alg3_min_pairs") *value = g.alg3_min_pairs;
    else if (k == "alg3_max_nodes") *value = g.alg3_max_nodes;
    else if (k == "alg3_overlap") *value = g.alg3_overlap;
    else if (k == "alg3_push_div") *value = g.alg3_push_div;
    else if (k == "alg3_early_pairs") *value = g.alg3_early_pairs;
    else if (k == "alg3_w_sweep") *value = g.alg3_w_sweep;
    else if (k == "alg3_w_probe") *value = g.alg3_w_probe;
    else if (k == "alg3_w_last") *value = g.alg3_w_last;
    else if (k == "alg3_workers") *value = g.alg3_workers;
    else if (k == "alg3_w_launch") *value = g.alg3_w_launch;
    else if (k == "batch_tile") *value = g.batch_tile_force;
    else if (k == "batch_tile_fwd16") *value = g.batch_tile_fwd[0];
    else if (k == "batch_tile_fwd32") *value = g.batch_tile_fwd[1];
    else if (k == "batch_tile_fwd64") *value = g.batch_tile_fwd[2];
    else if (k == "batch_tile_rev16") *value = g.batch_tile_rev[0];
    else if (k == "batch_tile_rev32") *value = g.batch_tile_rev[1];
    else if (k == "batch_tile_rev64") *value = g.batch_tile_rev[2];
    else return fail(ESIM_EINVAL, "unknown option '" + k + "'");
    return ESIM_OK;
}

esim_status esim_query(esim_graph* h, int64_t u, double c, double eps, uint64_t seed, double* s_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!s_out) return fail(ESIM_EINVAL, "s_out is NULL");
    return run_query(h->g, u, c, eps, seed, nullptr, 0, nullptr, nullptr, s_out, nullptr, nullptr);
}

esim_status esim_query_device(esim_graph* h, int64_t u, double c, double eps, uint64_t seed, double* s_dev) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!s_dev) return fail(ESIM_EINVAL, "s_dev is NULL");
    return run_query(h->g, u, c, eps, seed, s_dev, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
}

esim_status esim_topk(esim_graph* h, int64_t u, double c, double eps, uint64_t seed, int32_t k, int32_t* ids_out,
                      double* scores_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (k < 1) return fail(ESIM_EINVAL, "k must be >= 1");
    if (!ids_out || !scores_out) return fail(ESIM_EINVAL, "NULL output");
    return run_query(h->g, u, c, eps, seed, nullptr, k, nullptr, nullptr, nullptr, ids_out, scores_out);
}

esim_status esim_topk_device(esim_graph* h, int64_t u, double c, double eps, uint64_t seed, int32_t k,
                             int32_t* ids_dev, double* scores_dev) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (k < 1) return fail(ESIM_EINVAL, "k must be >= 1");
    if (!ids_dev || !scores_dev) return fail(ESIM_EINVAL, "NULL output");
    return run_query(h->g, u, c, eps, seed, nullptr, k, ids_dev, scores_dev, nullptr, nullptr, nullptr);
}

esim_status esim_last_stats(const esim_graph* h, esim_query_stats* out) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!out) return fail(ESIM_EINVAL, "out is NULL");
    const Graph& g = h->g;
    memset(out, 0, sizeof(*out));
    out->L = g.last_L;
    out->launches = g.last_launches;
    out->R_b = g.last_R_b;
    out->kappa = g.last_kappa;
    out->pi_norm2 = g.last_norm2;
    out->sum_R = g.last_sum_R;
    out->pair_steps = g.last_steps;
    out->ms_forward = g.last_ms[0];
    out->ms_allocate = g.last_ms[1];
    out->ms_sample = g.last_ms[2];
    out->ms_reverse = g.last_ms[3];
    out->ms_topk = g.last_ms[4];
    out->ms_total = g.last_ms[5];
    out->ms_sample_kernel = g.last_ms_kernel;
    out->ms_sample_side = g.last_ms_side;
    out->pair_steps_side = g.last_steps_side;
    out->side_candidates = g.last_side_candidates;
    out->alg3_nodes = g.last_alg3_nodes;
    out->hist_entries = g.last_hist_entries;
    out->workspace_bytes = g.last_ws_bytes;
    return ESIM_OK;
}

esim_status esim_forward(esim_graph* h, int64_t u, double c, int32_t L, double* hist) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (u < 0 || u >= g.n) return fail(ESIM_EINVAL, "source node out of range");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (!hist) return fail(ESIM_EINVAL, "hist is NULL");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    Ws w;
    esim_status st = ensure_ws(g, 0, 0, w);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(launch_forward(g, u, c, L, hist, w.xa, w.xb), "forward sweeps");
    return ESIM_OK;
}

esim_status esim_allocate(esim_graph* h, const double* hist, int32_t L, double R_b, int32_t mode, double* pi_out,
                          uint64_t* R_out, uint64_t* off) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!hist || !R_out || !off) return fail(ESIM_EINVAL, "NULL argument");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (mode != 0 && mode != 1) return fail(ESIM_EINVAL, "mode must be 0 or 1");
    if (!(R_b >= 0.0)) return fail(ESIM_EINVAL, "need R_b >= 0");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_allocate(g, hist, L, R_b, mode, pi_out, R_out, off), "allocation");
    return ESIM_OK;
}

esim_status esim_sample(esim_graph* h, const uint64_t* off, double c, uint64_t seed, uint64_t* nonmeet,
                        uint64_t* pair_steps) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!off || !nonmeet) return fail(ESIM_EINVAL, "NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_sample(g, off, c, seed, nonmeet, pair_steps), "walk pairs");
    return ESIM_OK;
}

esim_status esim_dhat(esim_graph* h, const uint64_t* nonmeet, const uint64_t* off, double* dhat) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!nonmeet || !off || !dhat) return fail(ESIM_EINVAL, "NULL argument");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_dhat(g, nonmeet, off, dhat), "dhat");
    return ESIM_OK;
}

esim_status esim_reverse(esim_graph* h, const double* hist, int32_t L, double c, const double* dhat, double* s_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!hist || !dhat || !s_out) return fail(ESIM_EINVAL, "NULL argument");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    Ws w;
    esim_status st = ensure_ws(g, 0, 0, w);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(launch_reverse(g, hist, L, c, dhat, s_out, w.xa, w.xb), "reverse sweeps");
    return ESIM_OK;
}

esim_status esim_select_topk(esim_graph* h, const double* scores, int64_t exclude, int32_t k, int32_t* ids_out,
                             double* vals_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!scores || !ids_out || !vals_out) return fail(ESIM_EINVAL, "NULL argument");
    if (k < 1) return fail(ESIM_EINVAL, "k must be >= 1");
    if (k > kTopkMax) return fail(ESIM_ENOTSUP, "k above 4096");
    if (exclude < -1 || exclude >= g.n) return fail(ESIM_EINVAL, "exclude out of range");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_topk(g, scores, exclude, k, ids_out, vals_out, g.topk_ws), "top-k");
    return ESIM_OK;
}

esim_status esim_forward_f32(esim_graph* h, int64_t u, double c, int32_t L, float* hist) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (u < 0 || u >= g.n) return fail(ESIM_EINVAL, "source node out of range");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (!hist) return fail(ESIM_EINVAL, "hist is NULL");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    Ws w;
    esim_status st = ensure_ws(g, 0, 1, w);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(launch_forward32(g, u, c, L, hist, w.xa32, w.xb32), "forward sweeps (FP32c)");
    return ESIM_OK;
}

esim_status esim_allocate_f32(esim_graph* h, const float* hist, int32_t L, double R_b, int32_t mode, double* pi_out,
                              uint64_t* R_out, uint64_t* off) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!hist || !R_out || !off) return fail(ESIM_EINVAL, "NULL argument");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (mode != 0 && mode != 1) return fail(ESIM_EINVAL, "mode must be 0 or 1");
    if (!(R_b >= 0.0)) return fail(ESIM_EINVAL, "need R_b >= 0");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_allocate32(g, hist, L, R_b, mode, pi_out, R_out, off), "allocation (FP32c)");
    return ESIM_OK;
}

esim_status esim_reverse_f32(esim_graph* h, const float* hist, int32_t L, double c, const double* dhat,
                             double* s_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!hist || !dhat || !s_out) return fail(ESIM_EINVAL, "NULL argument");
    if (L < 0 || L > 4096) return fail(ESIM_EINVAL, "need 0 <= L <= 4096");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    Ws w;
    esim_status st = ensure_ws(g, 0, 1, w);
    if (st != ESIM_OK) return st;
    ESIM_CUDA_TRY(launch_reverse32(g, hist, L, c, dhat, s_out, w.w2, w.sa2, w.sb2), "reverse sweeps (FP32c)");
    return ESIM_OK;
}

esim_status esim_query_batch(esim_graph* h, int32_t B, const int64_t* u, const double* eps, uint64_t seed, double c,
                             double* s_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!s_out) return fail(ESIM_EINVAL, "s_out is NULL");
    return run_batch(h->g, B, u, eps, seed, c, nullptr, s_out, 0, nullptr, nullptr, nullptr, nullptr);
}

esim_status esim_query_batch_device(esim_graph* h, int32_t B, const int64_t* u, const double* eps, uint64_t seed,
                                    double c, double* s_dev) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (!s_dev) return fail(ESIM_EINVAL, "s_dev is NULL");
    return run_batch(h->g, B, u, eps, seed, c, s_dev, nullptr, 0, nullptr, nullptr, nullptr, nullptr);
}

esim_status esim_topk_batch(esim_graph* h, int32_t B, const int64_t* u, const double* eps, uint64_t seed, double c,
                            int32_t k, int32_t* ids_out, double* scores_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (k < 1) return fail(ESIM_EINVAL, "k must be >= 1");
    if (!ids_out || !scores_out) return fail(ESIM_EINVAL, "NULL output");
    return run_batch(h->g, B, u, eps, seed, c, nullptr, nullptr, k, nullptr, nullptr, ids_out, scores_out);
}

esim_status esim_topk_batch_device(esim_graph* h, int32_t B, const int64_t* u, const double* eps, uint64_t seed,
                                   double c, int32_t k, int32_t* ids_dev, double* scores_dev) {
    if (check_graph(h)) return ESIM_EINVAL;
    if (k < 1) return fail(ESIM_EINVAL, "k must be >= 1");
    if (!ids_dev || !scores_dev) return fail(ESIM_EINVAL, "NULL output");
    return run_batch(h->g, B, u, eps, seed, c, nullptr, nullptr, k, ids_dev, scores_dev, nullptr, nullptr);
}

esim_status esim_alg3_first_meeting(esim_graph* h, int64_t k, int32_t depth, double c, double* z_out) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (k < 0 || k >= g.n) return fail(ESIM_EINVAL, "node out of range");
    if (depth < 1 || depth > kAlg3MaxDepth) return fail(ESIM_EINVAL, "need 1 <= depth <= 16");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (!z_out) return fail(ESIM_EINVAL, "z_out is NULL");
    if (g.has_duplicates) return fail(ESIM_ENOTSUP, "Algorithm 3 needs a graph without repeated in-edges");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    esim_status a3 = ensure_a3ws(g);
    if (a3 != ESIM_OK) return a3;
    ESIM_CUDA_TRY(alg3_first_meeting(g, k, depth, c, g.a3ws, z_out, nullptr), "Algorithm 3 first meetings");
    return ESIM_OK;
}

esim_status esim_alg3_paper_depth(esim_graph* h, const uint64_t* R, double c, int32_t max_depth, uint8_t* depth) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!R || !depth) return fail(ESIM_EINVAL, "NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (max_depth < 0 || max_depth > kAlg3MaxDepth) return fail(ESIM_EINVAL, "need 0 <= max_depth <= 16");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    esim_status a3 = ensure_a3pws(g);
    if (a3 != ESIM_OK) return a3;
    ESIM_CUDA_TRY(alg3_paper_depths(g, R, c, max_depth, g.a3pws, depth, nullptr), "Algorithm 3 depths (explored edges)");
    return ESIM_OK;
}

esim_status esim_alg3_zsum(esim_graph* h, const uint8_t* depth, double c, double* zsum) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!depth || !zsum) return fail(ESIM_EINVAL, "NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    if (g.has_duplicates) return fail(ESIM_ENOTSUP, "Algorithm 3 needs a graph without repeated in-edges");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    int launches = 0, used = 0;
    return alg3_zsums(g, depth, c, zsum, &launches, &used);
}

int32_t esim_alg3_depth(double v, double c, const uint64_t* supp, int32_t max_depth, int64_t n, int64_t m,
                        double w_sweep, double w_probe, double w_launch, double w_last) {
    if (!supp || !(c > 0.0 && c < 1.0) || max_depth < 0 || max_depth > kAlg3MaxDepth || n < 1 || m < 0 ||
        !(v >= 0.0) || !(w_sweep >= 0.0) || !(w_probe >= 0.0) || !(w_launch >= 0.0) || !(w_last >= 0.0))
        return -1;
    return alg3_depth(v, c, supp, max_depth, n, m, w_sweep, w_probe, w_launch, w_last);
}

esim_status esim_sample_depth(esim_graph* h, const uint64_t* off, const uint8_t* depth, double c, uint64_t seed,
                              uint64_t* counts, uint64_t* pair_steps) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!off || !counts) return fail(ESIM_EINVAL, "NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_sample(g, off, c, seed, counts, pair_steps, depth), "walk pairs");
    return ESIM_OK;
}

esim_status esim_dhat_alg3(esim_graph* h, const uint64_t* counts, const uint64_t* off, const uint8_t* depth,
                           const double* zsum, double c, double* dhat) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    if (!counts || !off || !depth || !zsum || !dhat) return fail(ESIM_EINVAL, "NULL argument");
    if (!(c > 0.0 && c < 1.0)) return fail(ESIM_EINVAL, "need 0 < c < 1");
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(launch_dhat_alg3(g, counts, off, depth, zsum, c, dhat), "dhat (Algorithm 3)");
    return ESIM_OK;
}

esim_status esim_sync(esim_graph* h) {
    if (check_graph(h)) return ESIM_EINVAL;
    Graph& g = h->g;
    ESIM_CUDA_TRY(cudaSetDevice(g.device), "cudaSetDevice");
    ESIM_CUDA_TRY(cudaMemcpyAsync(g.status_host, g.status, sizeof(Status), cudaMemcpyDeviceToHost, g.stream),
                  "copy status");
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "stream synchronize");
    const int err = g.status_host->err;
    ESIM_CUDA_TRY(cudaMemsetAsync(g.status, 0, sizeof(Status), g.stream), "reset status");
    ESIM_CUDA_TRY(cudaStreamSynchronize(g.stream), "stream synchronize");
    if (err & kErrBudget) return fail(ESIM_EBUDGET, "pair budget exceeded or R(k) overflow");
    if (err & kErrTimeout) return fail(ESIM_ETIMEOUT, "device wait timed out");
    return ESIM_OK;
}

}  // extern "C"
