// Internal declarations shared by the library's translation units.
// Not part of the public ABI (that is include/exactsim.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <memory>
#include <vector>

struct esim_graph;

namespace esim {

// Device-side error bits, accumulated in Status::err.
enum : int {
    kErrBudget = 1,   // sum of R(k) above the pair budget, or R(k) overflow
    kErrTimeout = 2,  // a bounded wait ran out
    kErrCapacity = 4, // the sparse history outgrew its (pigeonhole) capacity
};

// Per-query device status block (one per graph handle).
struct Status {
    unsigned long long sum_R;
    unsigned long long pair_steps;
    double pi_norm2;
    int err;
    unsigned int ticket;             // last-block ticket of the sparse-history compaction
    unsigned long long hist_count;   // sparse history entries so far
    unsigned long long pair_steps_side;  // pair-steps of the side-stream sampler launch
};

// Sparse history of one query (sparse linearization): entries [lvl[l], lvl[l+1]) are
// the kept (node, pi^l(node)) of level l.
struct SparseHist {
    int32_t* idx;
    double* val;
    uint64_t* lvl;   // L + 2
    uint64_t cap;
};

// One segment of a long CSR row: entries [beg, end) of row `row`.
struct Segment {
    int32_t row;
    uint32_t beg;
    uint32_t end;
    uint32_t first;  // index of the row's first segment (rows own consecutive segments)
};

// A CSR resident on the device, with the row-split table for rows whose length
// is at least `long_min`.  Long rows are cut into segments of `seg_len` entries.
struct DevCsr {
    uint32_t* rp = nullptr;      // n+1
    int32_t* col = nullptr;      // m
    uint2* info = nullptr;       // n: (rp[i], rp[i+1] - rp[i]), one 8-byte load per row (walks)
    Segment* seg = nullptr;      // nseg
    int32_t* long_rows = nullptr;  // nlong row ids
    int32_t* long_first = nullptr; // nlong+1: first segment of each long row
    int64_t nseg = 0;
    int64_t nlong = 0;
    uint32_t long_min = 0;
    int group = 8;               // threads per short row
    // The single-vector sweeps' tiles: tile t covers rows [tiles[t], tiles[t+1]) with at
    // most tile_cap entries in all, or one row longer than that; rows longer than
    // kSweepTile are cut into segments of their own table (tseg, tlong_rows, tlong_first).
    uint32_t* tiles = nullptr;   // ntiles + 1
    int64_t ntiles = 0;
    uint32_t tile_cap = 0;       // entries per tile, <= kSweepTile (smaller on small graphs)
    Segment* tseg = nullptr;
    int32_t* tlong_rows = nullptr;
    int32_t* tlong_first = nullptr;
    int64_t tnseg = 0;
    int64_t tnlong = 0;
};

constexpr uint32_t kSweepTile = 512;        // entries a warp gathers into shared memory per tile, at most
constexpr uint32_t kSweepTileRows = 256;    // rows per tile at most (runs of empty rows)

struct Graph {
    int device = 0;
    int sm_count = 0;
    int64_t n = 0, m = 0;
    DevCsr in;    // rows = nodes, entries = in-neighbours (walks, reverse sweep)
    DevCsr out;   // rows = nodes, entries = out-neighbours (forward sweep)
    double* inv_din = nullptr;  // n: 1/din(i) (0 where din = 0), for the FP64 sweeps
    unsigned long long* din_magic = nullptr;  // n: floor((2^64 - 1) / din(i)) (0 where din <= 1), exact division
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t side_stream = nullptr;  // Algorithm 3: walks of the other nodes during the planning
    cudaEvent_t side_ev[2] = {};
    int side_candidates = 0;             // Algorithm 3 candidates walked by the side sampler
    cudaEvent_t side_tev[2] = {};        // timing of the side sampler (option timing)
    int sample_block_cap = 0;            // sampler blocks per SM (0: as many as fit)
    int alg3_overlap = 4;                // side sampler blocks per SM during the planning (0: no overlap)
    int alg3_push_div = 4;               // probe steps push while the frontier's in-edges <= (m+n)/this
    double alg3_early_pairs = 16777216.0; // a planned candidate with this many pairs walks at once
    // options
    double kappa = 0.0;
    int alloc_mode = 0;
    int exclude_source = 1;
    double pair_budget = 1e15;
    int timing = 0;
    int precision = 0;            // 0: FP64 sweeps; 1: FP32 storage with two-float sums (FP32c)
    int sparse_hist = 0;          // 1: sparse linearization (FP64 only; the query runs at eps/2)
    // Algorithm 3 (local deterministic exploitation)
    int alg3 = 0;
    int diag_mode = 0;  // 0: D^ from walk pairs (Algorithm 2 / 3); 1: ParSim's D = (1-c) I
    int alg3_rule = 0;       // 0: the paper's depth (explored edges reach 2 R(k)/sqrt c); 1: cost model
    int alg3_max_depth = 16;
    double alg3_min_pairs = 1e6;
    int alg3_max_nodes = 64;
    // Algorithm 3's cost model (pair-steps per sweep entry, per probe entry and column, per launch)
    double alg3_w_sweep = 4.0;
    double alg3_w_probe = 0.2;
    double alg3_w_launch = 524288.0;
    double alg3_w_last = 0.0625;         // the last probe level's share of a dense probe
    bool has_duplicates = false;  // repeated in-edges (Algorithm 3 needs a simple graph)
    std::shared_ptr<std::vector<uint32_t>> din_host;  // in-degrees, for the exploitation plan
    void* a3ws = nullptr;         // Algorithm 3 scratch (FP64 vectors, dot partials)
    size_t a3ws_bytes = 0;
    void* a3pws = nullptr;        // the paper's depth rule: support bit sets and edge tables
    size_t a3pws_bytes = 0;
    // Algorithm 3: extra workers for the one-node Lemma 5 computations, each with its own
    // stream, workspace and sweep/scan scratch (worker 0 is the query's own stream)
    struct A3Worker {
        cudaStream_t stream = nullptr;
        void* ws = nullptr;
        double* partial = nullptr;
        unsigned long long* scan_part = nullptr;
        double* norm_part = nullptr;
    };
    std::vector<A3Worker> a3workers;
    size_t a3worker_ws_bytes = 0;
    int alg3_workers = 4;         // concurrent one-node Lemma 5 computations
    void* zstage = nullptr;       // Algorithm 3: depth-2 node ids and their gathered Z sums
    size_t zstage_bytes = 0;
    int32_t last_alg3_nodes = 0;
    int32_t last_side_candidates = 0;
    uint64_t last_hist_entries = 0;
    uint64_t last_ws_bytes = 0;
    // batched queries: their own workspace, and the autotuned tile per width (W = 32, 64)
    void* bws = nullptr;
    size_t bws_bytes = 0;
    int batch_tile_fwd[3] = {-1, -1, -1};  // per width W = 16, 32, 64
    int batch_tile_rev[3] = {-1, -1, -1};
    int batch_tile_force = -1;    // option "batch_tile": -1 autotune, else 0..2
    int shared_walks = 1;         // batches: one walk set per node for all columns
    float batch_tune_ms[3][2][3] = {};
    // workspace
    Status* status = nullptr;     // device
    Status* status_host = nullptr; // pinned host copy
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* partial = nullptr;    // long-row partial sums (max nseg of in/out)
    unsigned long long* scan_part = nullptr;  // scan partials
    double* norm_part = nullptr;
    int64_t scan_blocks = 0;
    void* topk_ws = nullptr;
    // timing events
    cudaEvent_t ev[8] = {};
    // last stats
    int32_t last_L = 0;
    int32_t last_launches = 0;
    double last_R_b = 0, last_kappa = 0, last_norm2 = 0;
    unsigned long long last_sum_R = 0, last_steps = 0;
    float last_ms[6] = {};
    float last_ms_kernel = 0.f, last_ms_side = 0.f;  // sampler launches alone (main, side)
    unsigned long long last_steps_side = 0;
};

// sweep.cu
cudaError_t launch_forward(const Graph& g, int64_t u, double c, int32_t L, double* hist, double* xa, double* xb);
cudaError_t launch_reverse(const Graph& g, const double* hist, int32_t L, double c, const double* dhat, double* s_out,
                           double* sa, double* sb);
cudaError_t launch_forward32(const Graph& g, int64_t u, double c, int32_t L, float* hist, float* xa, float* xb);
cudaError_t launch_walk_distributions(const Graph& g, int64_t u, int steps, double* H, double* xa, double* xb);
cudaError_t launch_pull_sum(const Graph& g, const float2* x, double* out);
cudaError_t launch_reverse32(const Graph& g, const float* hist, int32_t L, double c, const double* dhat,
                             double* s_out, float2* w, float2* sa, float2* sb);
cudaError_t launch_forward_sparse(const Graph& g, int64_t u, double c, int32_t L, double theta, const SparseHist& h,
                                  double* lev, double* pi_run, double* xa, double* xb);
cudaError_t launch_reverse_sparse(const Graph& g, const SparseHist& h, int32_t L, double c, const double* dhat,
                                  double* s_out, double* sa);

// sample.cu
int64_t allocate_blocks(int64_t n);
cudaError_t launch_allocate(const Graph& g, const double* hist, int32_t L, double R_b, int mode, double* pi_out,
                            uint64_t* R_out, uint64_t* off);
cudaError_t launch_allocate32(const Graph& g, const float* hist, int32_t L, double R_b, int mode, double* pi_out,
                              uint64_t* R_out, uint64_t* off);
cudaError_t launch_sample(const Graph& g, const uint64_t* off, double c, uint64_t seed, uint64_t* nonmeet,
                          uint64_t* pair_steps, const uint8_t* depth = nullptr);
cudaError_t launch_dhat(const Graph& g, const uint64_t* nonmeet, const uint64_t* off, double* dhat);
cudaError_t launch_fill(const Graph& g, int64_t n, double value, double* out);
// R_out(k) = R(k) where bit keep(k) of want_mask is set (keep(k) < 8), else 0
cudaError_t launch_mask_R(const Graph& g, const uint64_t* R, const uint8_t* keep, uint8_t want_mask, uint64_t* R_out);
// counts(k) = side(k) where cand(k) != 1 (the nodes the side sampler walked)
cudaError_t launch_merge_counts(const Graph& g, const uint8_t* cand, const uint64_t* side, uint64_t* counts);
// cand(k) = 1 for the listed nodes
cudaError_t launch_mark(const Graph& g, const int32_t* ids, int count, uint8_t* mark);
// batches: nseg = B * n segments, segment q*n + k = node k of column q
// shared_B > 0 with rbase: segment s covers pairs [rbase[s], rbase[s] + len) of node s / shared_B
cudaError_t launch_sample_segments(const Graph& g, int64_t nseg, const uint64_t* off, double c, uint64_t seed,
                                   uint64_t* nonmeet, uint64_t* pair_steps, const uint8_t* depth = nullptr,
                                   int shared_B = 0, const uint64_t* rbase = nullptr, bool zero_counts = true);
// One planned Algorithm 3 candidate: depth >= 1 sets R(k) and depth(k); early marks
// cand(k) = 2 (its walks run on the side stream during the rest of the planning)
struct PlanEntry {
    int32_t k;
    uint8_t depth;
    uint8_t early;
    uint16_t pad;
    uint64_t R;
};
cudaError_t launch_plan_scatter(const Graph& g, const PlanEntry* plan, int count, uint64_t* R, uint8_t* depth,
                                uint8_t* cand);
cudaError_t launch_dhat_segments(const Graph& g, int64_t nseg, const uint64_t* nonmeet, const uint64_t* off,
                                 double* dhat);
// record = false: an auxiliary scan that leaves the status block (sum of R, budget) alone
cudaError_t launch_scan_R(const Graph& g, int64_t N, const uint64_t* R, uint64_t* off, unsigned long long* part_R,
                          double* part_norm, double* part_Rd, bool record = true);
uint32_t walk_threshold(double c);

// capi.cu: record a message for esim_last_error() and return `status` (as an esim_status int)
int set_error(int status, const std::string& message);

// batch.cu
int batch_tile_count();
int batch_tile_lpr(int tile);
cudaError_t launch_batch_forward_init(const Graph& g, int W, int B, const int64_t* u, double c, float* hist0, float* x0);
cudaError_t launch_batch_forward_level(const Graph& g, int W, int tile, int level, double c, const int32_t* Lq,
                                       const float* x_prev, float* hist_l, float* x_next, void* partial);
cudaError_t launch_batch_alloc(const Graph& g, int W, int B, const float* hist, int32_t Lmax, const double* Rb,
                               int mode, uint64_t* R);
cudaError_t launch_batch_reverse_init(const Graph& g, int W, int B, const double* dhat, double c, const float* hL,
                                      float2* w, float2* s0, double* s_out_if_final);
// walks shared across a batch's columns (node-major intervals between the distinct R_q(k))
cudaError_t launch_shared_plan(const Graph& g, int B, const uint64_t* R, uint64_t* len, uint64_t* rbase);
cudaError_t launch_shared_columns(const Graph& g, int B, const uint64_t* R, const uint64_t* rbase, const uint64_t* soff,
                                  const uint64_t* scount, uint64_t* nonmeet);
cudaError_t launch_dhat_from_R(const Graph& g, int64_t N, const uint64_t* nonmeet, const uint64_t* R, double* dhat);
cudaError_t launch_batch_reverse_level(const Graph& g, int W, int B, int tile, bool final_level, double c,
                                       const float2* w, const float* h, const float2* s_prev, float2* s_next,
                                       double* s_out, void* partial);

// alg3.cu
constexpr int kAlg3MaxDepth = 16;
size_t alg3_workspace_bytes(const Graph& g);
// supp_out[c * (kAlg3MaxDepth + 1) + i] = number of nodes with (P^T)^i(ks[c], .) != 0, for
// i = 0..levels (levels <= kAlg3MaxDepth) and the count nodes ks (host); synchronises g.stream.
cudaError_t alg3_supports(const Graph& g, const int32_t* ks, int count, int levels, void* ws, uint64_t* supp_out,
                          int* launches);
// Z_1..Z_depth of node k (Lemma 5) into z_out (host), depth <= kAlg3MaxDepth; synchronises g.stream.
cudaError_t alg3_first_meeting(const Graph& g, int64_t k, int depth, double c, void* ws, double* z_out,
                               int* launches);
cudaError_t launch_dhat_alg3(const Graph& g, const uint64_t* counts, const uint64_t* off, const uint8_t* depth,
                             const double* zsum, double c, double* dhat);

// alg3_paper.cu: the paper's adaptive depth (Algorithm 3).  depth[k] for every node with
// R(k) > 0 (device arrays; the others get 0); synchronises g.stream once per level.
size_t alg3_paper_bytes(int64_t n, int max_depth);
bool alg3_paper_fits(int64_t n);
cudaError_t alg3_paper_depths(const Graph& g, const uint64_t* R, double c, int max_depth, void* ws, uint8_t* depth,
                              int* launches);
// zsum(k) = Z_1(k) = c / din(k) for the nodes of depth 1 (others untouched)
cudaError_t alg3_paper_z1(const Graph& g, const uint8_t* depth, double c, double* zsum);
// zsum(k) = Z_1(k) + Z_2(k) for the listed nodes (device ids), by the closed form of depth 2;
// NaN where the two-hop neighbourhood is too large for the kernel's table
cudaError_t alg3_paper_z2(const Graph& g, const int32_t* ids, int count, double c, double* zsum);
// dst[i] = src[ids[i]] for i < count (device arrays)
cudaError_t alg3_gather_f64(const Graph& g, const int32_t* ids, int count, const double* src, double* dst);

// topk.cu
constexpr int kTopkMax = 4096;

// capi.cu: batch planning and enqueueing (shared by the batch calls and the server)
constexpr int kBatchMax = 64;
struct BatchPlan {
    int W, B, k;
    int32_t Lmax;
    int32_t Lq[kBatchMax];
    double Rb[kBatchMax];
    int64_t u[kBatchMax];
};
int batch_width(int B);
int batch_wi(int W);
int batch_plan(const Graph& g, int32_t B, const int64_t* u, const double* eps, double c, int32_t k, BatchPlan* plan);
size_t batch_ws_bytes(const Graph& g, const BatchPlan& p);
// the Graph behind a public handle
Graph* graph_of(struct ::esim_graph* h);
int batch_enqueue(Graph& tuner, const Graph& view, const BatchPlan& p, void* ws, uint64_t seed, double c,
                  double* s_dev, double* s_host, int32_t* ids_dev, double* vals_dev, int32_t* ids_host,
                  double* vals_host, bool allow_tune);
size_t topk_workspace_bytes(int64_t n);
cudaError_t launch_topk(const Graph& g, const double* scores, int64_t exclude, int32_t k, int32_t* ids_out,
                        double* vals_out, void* ws);
size_t topk_batch_workspace_bytes(int32_t B);
cudaError_t launch_topk_batch(const Graph& g, int32_t B, const double* scores, const int64_t* exclude, int32_t k,
                              int32_t* ids_out, double* vals_out, void* ws);

}  // namespace esim
