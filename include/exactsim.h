/*
 * exactsim.h -- C ABI of the GB300 (sm_103a) ExactSim single-source SimRank library.
 *
 * Method: Wang, Wei, Yuan, Du, Wen, "Exact Single-Source SimRank Computation on
 * Large Graphs" (SIGMOD 2020, arXiv:2004.03493).  A single-source query for
 * node u returns s(v) ~ S(u, v) for every node v (Sec. 1); a top-k query returns
 * the k nodes with the largest similarities (Sec. 1).  The query runs Algorithm 1
 * (Basic ExactSim) with Algorithm 2 as its estimator of the diagonal correction
 * D and the pi(k)^2 sample allocation of Lemma 4:
 *
 *   1. L = ceil(log_{1/c}(2/eps))                                   (Algorithm 1)
 *   2. pi^0 = (1-sqrt c) e_u,  pi^l = sqrt(c) P pi^{l-1},  l = 1..L   (Algorithm 1)
 *   3. pi = sum_l pi^l;  R(k) = ceil(R_b pi(k)^2),  R_b = kappa ln(n) / eps^2
 *                                                  (Lemma 4; kappa = 6/(1-sqrt c)^4)
 *   4. D^(k) = fraction of R(k) sqrt(c)-walk pairs from k that never meet
 *                                                  (Algorithm 2, Eq. scwwalk)
 *   5. s^0 = D^ pi^L / (1-sqrt c);  s^l = sqrt(c) P^T s^{l-1} + D^ pi^{L-l} / (1-sqrt c)
 *      and s = s^L                                 (Algorithm 1, Eq. sL)
 *   6. top-k of s, ordered (score desc, node id asc), the source excluded
 *
 * P is the reverse transition matrix of Sec. 2.2: P(i, j) = 1/din(j) for every
 * in-neighbour i of j.  The graph is given as an in-edge CSR: row j lists the
 * in-neighbours I(j) of node j.  A repeated in-edge counts with its multiplicity.
 *
 * Random numbers (the paper names none): Philox-4x32-10 (Salmon et al., SC'11)
 * with key = (seed low 32 bits, seed high 32 bits) and counter (r_lo, r_hi, k, t)
 * for pair r of node k at step t.  One call per step gives (w0, w1, w2, w3); with
 * T = floor(sqrt(c) 2^32) walk A moves iff w0 < T and din > 0 and goes to
 * in-neighbour number (w1 * din) >> 32, exactly uniform by Lemire's rejection: when
 * the low 32 bits of w1 * din fall below (2^32 - din) mod din, the word is redrawn
 * from the side stream, counter (r_lo, r_hi, k, 2^31 | W 2^30 | j 2^16 | t) for the
 * j-th block of redraws of walk W (A = 0, B = 1); walk B likewise with w2, w3.  A
 * pair ends as "no meeting" as soon as either walk stops, and as "meeting" when
 * both move to the same node.  A pair still running after 65536 steps ends as "no
 * meeting".  With Algorithm 3 a node of depth d moves its pairs for d steps without
 * the continuation test.  A walk pair therefore depends only on (seed, k, r), not on
 * the query, its batch or the launch that runs it.
 *
 * Conventions
 *  - Every call returns an esim_status; ESIM_OK is 0.  On failure
 *    esim_last_error() gives a message (thread-local, valid until the next call
 *    on the same thread).
 *  - "host" pointers are ordinary CPU memory owned by the caller.  "device"
 *    pointers are CUDA global memory on the graph's device, owned by the caller.
 *  - Whole-query calls (esim_query, esim_topk and their _device forms) return
 *    after the work has finished on the GPU.  Step calls (esim_forward ...
 *    esim_select_topk) only enqueue work on the graph's stream; call esim_sync
 *    to wait and to collect device-side errors.
 *  - No call falls back to the CPU.  Without a usable CUDA device every call
 *    that needs one returns ESIM_ECUDA.
 *  - Node ids are int32 in [0, n); n < 2^31 and m < 2^32.
 *  - One graph handle serves one call at a time: calls on the same handle from
 *    several threads must be serialised by the caller (the server has its own
 *    scheduler thread and takes requests from any thread).  Several handles may
 *    share a device.
 */
#ifndef EXACTSIM_H
#define EXACTSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esim_graph esim_graph; /* opaque; owned by the library */

typedef enum {
    ESIM_OK = 0,
    ESIM_EINVAL = -1,   /* an argument is out of range or inconsistent */
    ESIM_ENOMEM = -2,   /* device or host allocation failed */
    ESIM_ECUDA = -3,    /* a CUDA call failed, or no usable device */
    ESIM_ETIMEOUT = -4, /* a bounded device-side wait ran out */
    ESIM_EBUDGET = -5,  /* the sum of R(k) exceeds the pair budget; no walks were run */
    ESIM_ENOTSUP = -6   /* a size the library does not handle (e.g. k above the top-k limit) */
} esim_status;

/* Statistics of the last whole query on a graph handle. */
typedef struct {
    int32_t L;            /* depth ceil(log_{1/c}(2/eps)) */
    int32_t launches;     /* kernels the library launched for the query */
    double R_b;           /* kappa ln(n) / eps^2 */
    double kappa;         /* the constant used */
    double pi_norm2;      /* ||pi||^2 = sum_k pi(k)^2 */
    uint64_t sum_R;       /* number of walk pairs, sum_k R(k) */
    uint64_t pair_steps;  /* Philox calls made by the sampler (one per pair step) */
    float ms_forward;     /* phase durations (CUDA events) when option "timing" is 1, else 0 */
    float ms_allocate;
    float ms_sample;
    float ms_reverse;
    float ms_topk;
    float ms_total;
    int32_t alg3_nodes;   /* nodes exploited by Algorithm 3 in the last query */
    int32_t reserved2;
    uint64_t hist_entries;    /* stored history entries: (L+1) n dense, kept entries sparse */
    uint64_t workspace_bytes; /* device bytes of the last query's workspace layout */
    /* With Algorithm 3 a second stream walks, in one sampler launch during the planning,
     * the nodes whose R(k) and depth are final: under the cost-model rule every node that
     * is not an exploitation candidate and the candidates with at least "alg3_early_pairs"
     * pairs, once every depth is chosen (before the first-meeting terms); under the
     * paper's rule every node, once the depths are known.  The other candidates walk on
     * the main stream after the planning.  ms_sample_kernel is the main sampler launch
     * alone and ms_sample_side the side launch (with option timing); pair_steps_side is
     * the side launch's share of pair_steps, which counts every launch; side_candidates
     * is the number of candidates the side launch walked. */
    float ms_sample_kernel;
    float ms_sample_side;
    uint64_t pair_steps_side;
    int32_t side_candidates;
    int32_t reserved3;
} esim_query_stats;

/* ------------------------------------------------------------------ library */

/* Version string of the library. */
const char* esim_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* esim_last_error(void);

/* Parameters of Algorithm 1.  esim_levels returns L = ceil(log(2/eps)/log(1/c)),
 * or -1 unless 0 < c < 1 and 0 < eps < 1.  esim_sample_base returns
 * R_b = kappa * log(n) / (eps * eps), kappa <= 0 meaning the paper's
 * 6 / ((1 - sqrt c)^4), or -1 on bad input.  esim_walk_threshold returns
 * T = floor(sqrt(c) * 2^32). */
int32_t esim_levels(double c, double eps);
double esim_sample_base(int64_t n, double c, double eps, double kappa);
uint32_t esim_walk_threshold(double c);

/* ------------------------------------------------------------------ graph */

/* Load a graph from a host in-edge CSR: in_rowptr[n+1] (in_rowptr[0] = 0,
 * non-decreasing, in_rowptr[n] = m), in_col[m] with 0 <= in_col[p] < n.
 * The library copies both arrays to the current CUDA device, builds the
 * out-edge CSR (its transpose) and the row-split tables, and keeps them until
 * esim_free_graph.  The caller may free its arrays after the call.
 * Errors: ESIM_EINVAL (bad CSR, n < 1, n >= 2^31, m >= 2^32), ESIM_ENOMEM,
 * ESIM_ECUDA. */
esim_status esim_load_graph(int64_t n, const int64_t* in_rowptr, const int32_t* in_col, esim_graph** out);

/* Release the graph and every device buffer the library holds for it. */
void esim_free_graph(esim_graph* g);

int64_t esim_num_nodes(const esim_graph* g);
int64_t esim_num_edges(const esim_graph* g);

/* Run the graph's work on `stream` (a cudaStream_t of the graph's device; NULL
 * restores the library's own stream).  The library does not take ownership. */
esim_status esim_set_stream(esim_graph* g, void* stream);

/* Options (per graph handle):
 *   "kappa"          sample constant; <= 0 means 6/(1-sqrt c)^4 (default 0)
 *   "alloc"          0: R(k) = ceil(R_b pi(k)^2) (Lemma 4, default);
 *                    1: R(k) = ceil(R_b pi(k)) (Algorithm 1, basic)
 *   "exclude_source" 1: top-k leaves out the source (default); 0: keeps it
 *   "pair_budget"    largest allowed sum of R(k) (default 1e15); above it a
 *                    query returns ESIM_EBUDGET without running walks
 *   "timing"         1: record per-phase CUDA event times in the stats
 *   "shared_walks"   batches and the server: 1 (default) samples each node's walk pairs once
 *                    for all columns -- max_q R_q(k) pairs cut at the distinct R_q(k), each
 *                    column counting the intervals below its own R_q(k); the walk spec keys
 *                    pairs by (seed, k, r) only, so every column's counts are the same
 *                    integers as with 0 (each column sampled on its own)
 *   "sparse_hist"    1: sparse linearization (Section 3.2; FP64 only): the query runs
 *                    at eps/2 (L and R_b) and keeps only the history entries
 *                    pi^l(k) > (1-sqrt c)^2 eps/2 -- fewer than 1/that many, whatever n --
 *                    which adds at most eps/2 to the error; pi for the allocation is
 *                    still the dense sum.  A counting pass of the forward sweeps sizes
 *                    the workspace to the kept entries.  0: dense history (default)
 *   "diag"           0: D^ estimated by walk pairs (default); 1: ParSim's approximation
 *                    D = (1-c) I (Section 2, related work), no allocation and no walk pairs -- the
 *                    baseline of the paper's comparison of diagonal corrections
 *   "alg3"           1: Algorithm 3 (local deterministic exploitation); nodes with
 *                    din <= 1 take the exact D (1 at din 0, 1-c at din 1) and no walk
 *                    pairs.  An exploited node k of depth d gets the exact Z_1..Z_d
 *                    (Lemma 5) and special pairs that move for d steps without the
 *                    continuation draw; D^(k) = 1 - sum Z - c^d (pairs meeting after step
 *                    d)/R.  How d and the pair count are chosen is option "alg3_rule".
 *                    Needs a graph without repeated in-edges (else ESIM_ENOTSUP).
 *   "alg3_rule"      0 (default): the paper's adaptive depth (Algorithm 3).  Every node
 *                    with R(k) > 0 explores level by level, counting each edge the
 *                    listing traverses when it extends a walk distribution
 *                    (P^T)^(l')(q', .) by one step, and stops at the level during which
 *                    the count reaches 2 R(k)/sqrt(c), at a level that adds no edge, or at
 *                    alg3_max_depth; it keeps its R(k) pairs.  The count keeps n x n
 *                    support bit sets: graphs with 2 n ceil(n/32) 4-byte words above
 *                    4 GiB (n > 131072) return ESIM_ENOTSUP.
 *                    1: a cost model for speed -- only the heaviest nodes (by pi, at most
 *                    alg3_max_nodes, with din >= 2 and an Algorithm 2 count of at least
 *                    alg3_min_pairs) are exploited, at the depth that minimises an
 *                    estimate of the GPU work (walks plus the sweeps of Lemma 5, which
 *                    grow with the supports of (P^T)^i(k, .)), with
 *                    max(1, ceil(R_b pi(k)^2 c^(2d))) pairs: the tail estimator's variance
 *                    bound at depth d is c^(2d) times Algorithm 2's, so the variance bound
 *                    of R(k) Algorithm 2 pairs is kept; depth 0 leaves a node to Algorithm 2
 *   "alg3_max_nodes" cost model: heaviest nodes (by pi) considered, 1..4096 (default 64)
 *   "alg3_min_pairs" cost model: smallest Algorithm 2 pair count worth considering (default 1e6)
 *   "alg3_max_depth" deepest exploitation, 1..16 (default 16)
 *   "alg3_workers"   one-node Lemma 5 computations run at once, 1..16 (default 4): each
 *                    extra worker has its own stream and Algorithm 3 workspace (about
 *                    0.7 GB at n = 1e5, a few GB at n = 4e6; fewer workers when the device
 *                    cannot hold them).  Results do not depend on it.
 *   "alg3_push_div"  a probe step pushes from its frontier while the frontier's in-edges are
 *                    at most (m+n)/alg3_push_div, else pulls over all rows (default 4);
 *                    both give the same integers
 *   "alg3_overlap"   sampler blocks per SM of the side launch, which walks the nodes
 *                    whose plan is final on a second stream during the planning (default
 *                    4; 0: all walks after the planning).  Counts do not depend on it.
 *   "alg3_early_pairs"  with "alg3_overlap" > 0, the candidates with at least this many
 *                    pairs (default 2^24) walk in the side launch, with the other nodes,
 *                    as soon as every depth is chosen, while the first-meeting terms are
 *                    computed; the others after the planning.  Counts do not depend on it.
 *   "alg3_w_sweep", "alg3_w_probe", "alg3_w_launch", "alg3_w_last"  weights of the cost
 *                    model, in walk pair-steps: per entry of a single-vector sweep
 *                    (default 4), per entry and column of a 32-column probe sweep (0.2),
 *                    per kernel launch (2^19), and the last two probe levels' share of a
 *                    dense probe (1/16: one warp per node over its two- and three-hop
 *                    neighbourhood).  The estimate of depth d is R_d (d + 1/(1-c)) walks
 *                    plus w_sweep (m+n)(2d-1) + w_probe (m+n) (sum_{i<=d-4} |supp h_i|(d-i)
 *                    + w_last sum_{i=max(1,d-3)}^{d-2} (d-i)|supp h_i|) + w_launch (3(2d-1)
 *                    + sum_{i<=d-4} ceil(|supp h_i|/32)(3(d-i)+2) + 2 per level i >= d-3)
 *   "batch_tile"     -1: batched sweeps pick their tile by timing (default);
 *                    0, 1, 2: force 32, 16 or 8 lanes per row (results do not change)
 *   "precision"      0: FP64 sweeps (default);
 *                    1: FP32c, the precision form -- pi^l and x^l stored in FP32
 *                    with two-float (compensated) row sums, s^l stored and summed
 *                    as two-floats, FP64 only for the final s and for D^
 * Errors: ESIM_EINVAL for an unknown key or a bad value. */
esim_status esim_set_option(esim_graph* g, const char* key, double value);
esim_status esim_get_option(const esim_graph* g, const char* key, double* value);

/* ------------------------------------------------------------------ queries */

/* Single-source query of node u (Algorithm 1): s_out[n] (host) receives s(v)
 * for every node v.  c and eps in (0, 1); seed selects the walk stream.
 * Errors: ESIM_EINVAL, ESIM_EBUDGET, ESIM_ENOMEM, ESIM_ECUDA. */
esim_status esim_query(esim_graph* g, int64_t u, double c, double eps, uint64_t seed, double* s_out);

/* As esim_query, with s_dev[n] in device memory. */
esim_status esim_query_device(esim_graph* g, int64_t u, double c, double eps, uint64_t seed, double* s_dev);

/* Top-k query: the k nodes with the largest s(v), ordered (score desc, id asc),
 * the source left out unless option "exclude_source" is 0.  ids_out[k] and
 * scores_out[k] are host arrays.  If fewer than k nodes are eligible the
 * remaining slots get id -1 and score 0.  1 <= k <= 4096, else ESIM_ENOTSUP
 * (k > 4096) or ESIM_EINVAL (k < 1). */
esim_status esim_topk(esim_graph* g, int64_t u, double c, double eps, uint64_t seed, int32_t k,
                      int32_t* ids_out, double* scores_out);

/* As esim_topk with device outputs. */
esim_status esim_topk_device(esim_graph* g, int64_t u, double c, double eps, uint64_t seed, int32_t k,
                             int32_t* ids_dev, double* scores_dev);

/* Batched queries (B <= 64 sources, each with its own eps, one launch sequence).
 * The sweeps become sparse-matrix x dense-matrix products over an n x W block
 * (W = 32 for B <= 32, else 64), in the precision form (FP32 storage, two-float
 * sums, FP64 output).  Column q runs Algorithm 1 with its own depth
 * L_q = ceil(log_{1/c}(2/eps[q])) (levels above L_q are zero) and its own
 * R_b = kappa ln(n)/eps[q]^2.  All columns draw their walk pairs from the one
 * seed: pair r of node k is the same pair in every column and in a single query
 * with that seed.  A column's result does not depend on the other columns of the
 * batch (each column sums a row's entries in the same fixed order whatever the
 * batch or the tile shape), so a query gives bit-identical results alone (B = 1)
 * and in any mix.  s_out[B * n] is query-major: s_out[q * n + v].
 * Errors: ESIM_EINVAL, ESIM_ENOTSUP (B > 64, k > 4096), ESIM_EBUDGET, ESIM_ENOMEM,
 * ESIM_ECUDA. */
esim_status esim_query_batch(esim_graph* g, int32_t B, const int64_t* u, const double* eps, uint64_t seed, double c,
                             double* s_out);
esim_status esim_query_batch_device(esim_graph* g, int32_t B, const int64_t* u, const double* eps, uint64_t seed,
                                    double c, double* s_dev);
/* Batched top-k: ids_out[B * k], scores_out[B * k] (row q holds query q's top-k,
 * ordered (score desc, id asc), its source left out unless "exclude_source" is 0). */
esim_status esim_topk_batch(esim_graph* g, int32_t B, const int64_t* u, const double* eps, uint64_t seed, double c,
                            int32_t k, int32_t* ids_out, double* scores_out);
esim_status esim_topk_batch_device(esim_graph* g, int32_t B, const int64_t* u, const double* eps, uint64_t seed,
                                   double c, int32_t k, int32_t* ids_dev, double* scores_dev);

/* ------------------------------------------------------------------ serving
 * A request loop over one resident graph with continuous batching.  Requests
 * (u, eps) enter a queue; a scheduler thread forms waves of up to max_batch
 * requests and runs each wave as a batched query (esim_topk_batch) on its own
 * CUDA stream and workspace.  Up to max_waves waves are in flight, admitted while
 * their workspaces fit mem_budget_bytes; when a wave completes its slots and
 * memory go to the next queued requests, so requests that arrive while others
 * run start as soon as a slot set frees, and the waves' kernels overlap on the
 * device.  A request's result is bit-identical to the same request served alone.
 * While a server runs it owns the graph: make no other call on that graph handle.
 * Every wait is bounded; no device-side wait exists. */
typedef struct esim_server esim_server;

typedef struct {
    double c;                /* decay factor, 0 < c < 1 */
    double kappa;            /* sample constant to set on the graph; 0 keeps the graph's option */
    uint64_t seed;           /* walk stream shared by all requests */
    int32_t k;               /* top-k of every request, 1..4096 */
    int32_t max_batch;       /* requests per wave, 1..64 */
    int32_t max_waves;       /* waves in flight, 1..8 (one CUDA stream each) */
    int32_t reserved;
    double mem_budget_bytes; /* device memory for wave workspaces; <= 0: 80 % of the free memory */
} esim_server_config;

typedef struct {
    uint64_t completed;      /* requests answered */
    uint64_t failed;         /* requests that ended with an error (or were cancelled) */
    uint64_t waves;          /* waves launched */
    double mean_batch;       /* requests per wave */
    double p50_ms;           /* latency from submit to completion, over completed requests */
    double p99_ms;
    double max_ms;
    int32_t max_running;     /* most requests on the GPU at once */
    int32_t queued;          /* requests waiting now */
} esim_server_stats;

esim_status esim_server_create(esim_graph* g, const esim_server_config* cfg, esim_server** out);
/* Queue a top-k query of source u with error eps; *id_out identifies it. */
esim_status esim_server_submit(esim_server* s, int64_t u, double eps, uint64_t* id_out);
/* *state: 0 queued, 1 running, 2 done, 3 failed. */
esim_status esim_server_poll(esim_server* s, uint64_t id, int32_t* state);
/* Wait up to timeout_ms for request id; on success copies its k ids and scores
 * (either may be NULL) and its latency, and forgets the request.  ESIM_ETIMEOUT
 * if it is not finished in time (it stays known); the request's own error if it
 * failed. */
esim_status esim_server_wait(esim_server* s, uint64_t id, int32_t timeout_ms, int32_t* ids_out, double* scores_out,
                             double* latency_ms);
esim_status esim_server_get_stats(esim_server* s, esim_server_stats* out);
/* Cancel queued requests, let running waves finish, release everything. */
void esim_server_destroy(esim_server* s);

/* Statistics of the last whole query on g. */
esim_status esim_last_stats(const esim_graph* g, esim_query_stats* out);

/* ------------------------------------------------------------------ steps
 * The steps of the query, exposed for testing and composition.  All pointers
 * are device pointers; all calls enqueue on the graph's stream. */

/* Forward sweeps (Algorithm 1): hist[(L+1) * n] receives pi^0 .. pi^L, level l
 * at hist + l*n.  0 <= u < n, 0 < c < 1, 0 <= L <= 4096. */
esim_status esim_forward(esim_graph* g, int64_t u, double c, int32_t L, double* hist);

/* Allocation (Lemma 4 / Algorithm 1): pi(k) = sum_{l=0..L} hist[l*n + k] added in
 * level order; R(k) = ceil(R_b * (pi(k) * pi(k))) (mode 0) or ceil(R_b * pi(k))
 * (mode 1); off[0] = 0, off[k+1] = off[k] + R(k).  pi_out may be NULL.
 * R_out[n], off[n+1] (uint64).  With option "alg3" = 1 the nodes with din <= 1 get
 * R(k) = 0 (Algorithm 3 gives their D exactly: 1 at din 0, 1-c at din 1).  A value of
 * R_b * pi^2 at or above 2^63 makes esim_sync return ESIM_EBUDGET. */
esim_status esim_allocate(esim_graph* g, const double* hist, int32_t L, double R_b, int32_t mode,
                          double* pi_out, uint64_t* R_out, uint64_t* off);

/* Walk pairs (Algorithm 2): nonmeet[n] (uint64) receives, for each k, how many
 * of its off[k+1] - off[k] pairs never meet.  pair_steps (one uint64, may be
 * NULL) receives the number of Philox calls.  If off[n] exceeds the option
 * "pair_budget" no walk runs and esim_sync returns ESIM_EBUDGET.
 * off[n+1] must be nondecreasing with off[0] = 0, as esim_allocate writes it.  The
 * library does not check this on the device: other arrays give undefined results,
 * including reads past the end of off.  The same holds for every step call below
 * that takes off. */
esim_status esim_sample(esim_graph* g, const uint64_t* off, double c, uint64_t seed, uint64_t* nonmeet,
                        uint64_t* pair_steps);

/* D^(k) = nonmeet[k] / (off[k+1] - off[k]), 0 where the count is 0 (Algorithm 2). */
esim_status esim_dhat(esim_graph* g, const uint64_t* nonmeet, const uint64_t* off, double* dhat);

/* Reverse accumulation (Algorithm 1, Eq. sL) from hist[(L+1)*n] and D^[n]:
 * s_out[n] = s^L. */
esim_status esim_reverse(esim_graph* g, const double* hist, int32_t L, double c, const double* dhat,
                         double* s_out);

/* Precision-form steps (FP32c, see option "precision").  esim_forward_f32 writes
 * pi^0 .. pi^L as FP32 into hist[(L+1) * n] (each row sum formed in two-float and
 * rounded once).  esim_allocate_f32 is esim_allocate over an FP32 history, the
 * level sums taken in two-float and rounded to FP64 before R(k) is decided.
 * esim_reverse_f32 runs the reverse accumulation from an FP32 history with
 * two-float vectors and writes s^L in FP64. */
esim_status esim_forward_f32(esim_graph* g, int64_t u, double c, int32_t L, float* hist);
esim_status esim_allocate_f32(esim_graph* g, const float* hist, int32_t L, double R_b, int32_t mode,
                              double* pi_out, uint64_t* R_out, uint64_t* off);
esim_status esim_reverse_f32(esim_graph* g, const float* hist, int32_t L, double c, const double* dhat,
                             double* s_out);

/* Algorithm 3 steps.  esim_alg3_first_meeting writes Z_1..Z_depth of node k
 * (1 <= depth <= 16) into z_out (host): Z_l(k) = c^l * the probability that two
 * non-stop walks from k first meet at step l (Lemma 5, summed over the meeting
 * node); synchronous.  esim_sample_depth is esim_sample with depth[n] (device,
 * uint8, may be NULL): for a node of depth d > 0 its pairs move without the
 * continuation draw for d steps and counts[k] is the number that first meet after
 * step d.  esim_dhat_alg3 gives D^ = counts/R for depth 0, 1 - zsum - c^d counts/R
 * for depth d > 0, and 1 (din 0) or 1-c (din 1) exactly. */
esim_status esim_alg3_first_meeting(esim_graph* g, int64_t k, int32_t depth, double c, double* z_out);
/* Algorithm 3's depth choice for one node, host arithmetic only (no device): the d in
 * 0..max_depth (<= 16) of least estimated work R_d (d + 1/(1-c)) + w_sweep (m+n)(2d-1) +
 * w_probe (m+n) (sum_{i=1}^{d-4} supp[i](d-i) + w_last sum_{i=max(1,d-3)}^{d-2}
 * (d-i) supp[i]) + w_launch launches(d), R_d = max(1, ceil(v c^(2d))), v = R_b pi(k)^2 (R_b pi(k) for the
 * basic allocation), supp[i] = |supp (P^T)^i(k, .)| for i = 0..max(0, max_depth-2); the
 * first on ties (the options "alg3_w_*" give the weights).  Option "alg3_rule" = 1
 * decides every candidate with it.  Returns -1 on invalid arguments. */
int32_t esim_alg3_depth(double v, double c, const uint64_t* supp, int32_t max_depth, int64_t n, int64_t m,
                        double w_sweep, double w_probe, double w_launch, double w_last);
/* Algorithm 3's adaptive depth as the paper gives it ("Local deterministic exploitation
 * for D"): depth[n] (device, uint8) receives, for every node with R[k] > 0 (R: device,
 * uint64[n]), the level l during which its explored-edge count E_k reaches
 * 2 R(k)/sqrt(c), compared in FP64; a level that adds no edge, or max_depth
 * (0..16), ends the exploration earlier.  E_k adds, at level l, for every l' = 0..l and
 * every q' in supp (P^T)^(l-l')(k, .), the in-degrees of the nodes in
 * supp (P^T)^(l')(q', .): the edges the listing traverses when it extends that walk
 * distribution by one step.  Nodes with R[k] = 0 get depth 0.  Synchronises the
 * graph's stream once per level.  Errors: ESIM_ENOTSUP for n > 131072 (the support
 * bit sets), ESIM_EINVAL, ESIM_ENOMEM, ESIM_ECUDA. */
esim_status esim_alg3_paper_depth(esim_graph* g, const uint64_t* R, double c, int32_t max_depth, uint8_t* depth);
/* Algorithm 3's exact part for given depths (Lemma 5): zsum[k] = Z_1(k) + ... + Z_d(k) with
 * d = depth[k] (device uint8[n], 0..16), 0 where d = 0; zsum is device double[n].  Depth 1
 * is c/din(k); depth 2 uses Lemma 5's closed form over the two-hop neighbourhood (one warp
 * per node, 63-bit fixed point); deeper nodes, and depth-2 nodes with more than 512
 * two-hop entries, run esim_alg3_first_meeting's kernels, "alg3_workers" nodes at a time.
 * The query with option "alg3_rule" = 0 uses this for the depths esim_alg3_paper_depth
 * gives, and the cost-model rule for its plan.  Synchronous.  Needs a graph without
 * repeated in-edges (else ESIM_ENOTSUP); ESIM_ENOMEM, ESIM_ECUDA. */
esim_status esim_alg3_zsum(esim_graph* g, const uint8_t* depth, double c, double* zsum);
esim_status esim_sample_depth(esim_graph* g, const uint64_t* off, const uint8_t* depth, double c, uint64_t seed,
                              uint64_t* counts, uint64_t* pair_steps);
esim_status esim_dhat_alg3(esim_graph* g, const uint64_t* counts, const uint64_t* off, const uint8_t* depth,
                           const double* zsum, double c, double* dhat);

/* Top-k selection over scores[n] (device): ids_out[k], vals_out[k] (device),
 * ordered (score desc, id asc); exclude = -1 keeps every node.  1 <= k <= 4096. */
esim_status esim_select_topk(esim_graph* g, const double* scores, int64_t exclude, int32_t k,
                             int32_t* ids_out, double* vals_out);

/* Top-k selection that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code running
 * inside a host framework that owns all device memory (a fixed arena, a
 * memory-capped serving process) and latency-critical threads that must not
 * take the device synchronisation an allocation or free may cause.
 * Same result as esim_select_topk: ids_out[k], vals_out[k] (device) receive the k
 * largest scores[n] (device), ordered (score desc, id asc); exclude = -1 keeps
 * every node; slots beyond the eligible nodes get id -1 and score 0.  Needs no
 * graph handle; work is enqueued on `stream` (a cudaStream_t of the current
 * device, NULL for the legacy default stream) and the call returns without
 * waiting.  Scratch: a static device array of about 66 KB (the radix-select state
 * and 4096 candidates), resident on every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  The address is kept with the id of the CUDA context it was
 * taken in; after a device reset (a new context) the next call looks it up again.
 * All calls share the array: calls whose work overlaps on
 * the GPU race and must be serialised by the caller.  Limits: 1 <= k <= 4096
 * (ESIM_ENOTSUP above), 1 <= n < 2^31.  Calls no cudaMalloc or cudaFree. */
esim_status esim_select_topk_static(const double* scores, int64_t n, int64_t exclude, int32_t k, int32_t* ids_out,
                                    double* vals_out, void* stream);

/* Wait for the graph's stream; returns the first device-side error recorded
 * since the last esim_sync (ESIM_EBUDGET, ESIM_ETIMEOUT) or ESIM_ECUDA. */
esim_status esim_sync(esim_graph* g);

#ifdef __cplusplus
}
#endif

#endif /* EXACTSIM_H */
