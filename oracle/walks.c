/*
 * O3: CPU walk-pair sampler for the diagonal correction estimate (Algorithm 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by oracle/walks.py for tests/, for
 * __graft_entry__.smoke() and for bench.py's cpu_baseline / reference legs.
 * The CUDA library never links or includes this file and has its own sampler.
 *
 * What it computes (Algorithm 2; walk semantics of Eq. scwwalk): for every node k
 * with R(k) > 0, R(k) pairs of independent sqrt(c)-walks start at k.  A step
 * moves a walk to a uniform in-neighbour with probability sqrt(c); otherwise the
 * walk stops.  nonmeet(k) counts the pairs whose walks never visit the same node
 * at the same step t >= 1.
 *
 * Random numbers.  The paper names no generator.  Both this file and the
 * library draw from Philox-4x32-10, written here from its definition in
 * Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3"
 * (SC'11):
 *   round:  (X0, X1, X2, X3) -> (hi(M1*X2) ^ X1 ^ K0, lo(M1*X2),
 *                                hi(M0*X0) ^ X3 ^ K1, lo(M0*X0))
 *   with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key (K0, K1) grows by the Weyl
 *   constants (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.
 *
 * Walk specification shared by both sides:
 *   key      = (seed low 32 bits, seed high 32 bits)
 *   counter  = (r low 32 bits, r high 32 bits, k, t) for pair r of node k, step t
 *   (w0, w1, w2, w3) = Philox(counter, key)
 *   T        = floor(sqrt(c) * 2^32)
 *   walk A moves iff w0 < T and din(xA) > 0; walk B moves iff w2 < T and din(xB) > 0
 *   if either does not move, the pair ends without meeting
 *   otherwise xA <- I(xA)[pick(w1, din(xA), A)], xB <- I(xB)[pick(w3, din(xB), B)]
 *   if xA == xB the pair ends as a meeting; else t <- t + 1
 *   a pair that reaches t = 65536 steps ends without meeting (probability c^65536)
 *
 * pick(x, d, W) is an exactly uniform index in [0, d): Lemire's multiply-shift with
 * rejection (D. Lemire, "Fast Random Integer Generation in an Interval", ACM TOMS
 * 2019): with p = x * d (64 bits), accept p >> 32 unless low32(p) < (2^32 mod d);
 * a rejected word is replaced by the next word of walk W's side stream, the words
 * z0..z3 of Philox(counter (r_lo, r_hi, k, 2^31 | W 2^30 | j 2^16 | t)) for
 * j = 0, 1, ..., W = 0 for walk A and 1 for walk B.  After 2^14 side blocks the
 * last index is kept (probability below 2^-65536).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u
#define WALK_T_MAX 65536u

static void philox_round(uint32_t x[4], uint32_t k0, uint32_t k1) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k0;
    uint32_t y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
}

static void philox4x32_10(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        philox_round(x, k0, k1);
    }
    memcpy(out, x, sizeof(x));
}

/* Philox-4x32-10 of `count` counters (4 words each) under one 64-bit seed. */
void oracle_philox_many(int64_t count, const uint32_t* ctr, uint64_t seed, uint32_t* out) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t i = 0; i < count; ++i) philox4x32_10(ctr + 4 * i, k0, k1, out + 4 * i);
}

uint32_t oracle_walk_threshold(double c) {
    double v = floor(sqrt(c) * 4294967296.0);
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

/* Exactly uniform index in [0, d) (Lemire's method, side stream on rejection). */
static uint32_t pick(uint32_t x, uint32_t d, uint32_t rlo, uint32_t rhi, uint32_t k, uint32_t tag,
                     uint32_t k0, uint32_t k1) {
    uint64_t m = (uint64_t)x * (uint64_t)d;
    uint32_t l = (uint32_t)m;
    if (l < d) {
        const uint32_t thr = (uint32_t)(0u - d) % d;
        uint32_t j = 0, z[4];
        int used = 4;
        while (l < thr) {
            if (used == 4) {
                if (j == (1u << 14)) break;
                uint32_t ctr[4] = {rlo, rhi, k, tag | (j << 16)};
                philox4x32_10(ctr, k0, k1, z);
                ++j;
                used = 0;
            }
            x = z[used++];
            m = (uint64_t)x * (uint64_t)d;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* pick() for `count` words x[i] with one d (test hook for the rejection path). */
void oracle_pick_many(int64_t count, const uint32_t* x, uint32_t d, uint64_t seed, uint32_t* out) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int64_t i = 0; i < count; ++i) out[i] = pick(x[i], d, (uint32_t)i, 0u, 0u, 0x80000000u, k0, k1);
}

/* One walk pair.  Depth 0 (Algorithm 2): returns 1 if the walks never meet.
 * Depth d > 0 (Algorithm 3's special pair): the first d steps move without the
 * continuation draw (non-stop walks); returns 1 if the walks first meet at a step
 * after d, 0 otherwise (a meeting within the first d steps is already counted in
 * the exact first-meeting probabilities).  *steps counts main-stream Philox calls. */
static int walk_pair(const int64_t* rp, const int32_t* col, uint32_t k, uint64_t r,
                     uint32_t T, uint32_t k0, uint32_t k1, uint32_t depth, uint64_t* steps) {
    uint32_t xa = k, xb = k;
    const uint32_t rlo = (uint32_t)r, rhi = (uint32_t)(r >> 32);
    for (uint32_t t = 0; t < WALK_T_MAX; ++t) {
        uint32_t ctr[4] = {rlo, rhi, k, t};
        uint32_t w[4];
        philox4x32_10(ctr, k0, k1, w);
        *steps += 1;
        uint64_t da = (uint64_t)(rp[xa + 1] - rp[xa]);
        uint64_t db = (uint64_t)(rp[xb + 1] - rp[xb]);
        int forced = t < depth;
        int move_a = (forced || w[0] < T) && (da > 0);
        int move_b = (forced || w[2] < T) && (db > 0);
        if (!(move_a && move_b)) return depth ? 0 : 1;
        uint32_t ia = pick(w[1], (uint32_t)da, rlo, rhi, k, 0x80000000u | t, k0, k1);
        uint32_t ib = pick(w[3], (uint32_t)db, rlo, rhi, k, 0xC0000000u | t, k0, k1);
        uint32_t na = (uint32_t)col[rp[xa] + (int64_t)ia];
        uint32_t nb = (uint32_t)col[rp[xb] + (int64_t)ib];
        if (na == nb) return depth ? (t >= depth ? 1 : 0) : 0;
        xa = na;
        xb = nb;
    }
    return depth ? 0 : 1;
}

/*
 * nonmeet[k] <- number of non-meeting pairs among the R[k] pairs of node k.
 * Returns the total number of Philox calls (pair-steps), or -1 on bad input.
 * nthreads <= 0 uses the OpenMP default.
 */
int64_t oracle_walk_pairs_depth(int64_t n, const int64_t* in_rowptr, const int32_t* in_col,
                                const uint64_t* R, const uint8_t* depth, double c, uint64_t seed,
                                uint64_t* nonmeet, int nthreads);

int64_t oracle_walk_pairs(int64_t n, const int64_t* in_rowptr, const int32_t* in_col,
                          const uint64_t* R, double c, uint64_t seed, uint64_t* nonmeet,
                          int nthreads) {
    return oracle_walk_pairs_depth(n, in_rowptr, in_col, R, NULL, c, seed, nonmeet, nthreads);
}

/*
 * As oracle_walk_pairs, with depth[k] (may be NULL) selecting Algorithm 3's special
 * pairs for node k: counts[k] is then the number of pairs that first meet after
 * step depth[k].
 */
int64_t oracle_walk_pairs_depth(int64_t n, const int64_t* in_rowptr, const int32_t* in_col,
                                const uint64_t* R, const uint8_t* depth, double c, uint64_t seed,
                                uint64_t* nonmeet, int nthreads) {
    if (n <= 0 || n > 0xFFFFFFFFll) return -1;
    uint32_t T = oracle_walk_threshold(c);
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint64_t* off = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    if (!off) return -1;
    off[0] = 0;
    for (int64_t k = 0; k < n; ++k) off[k + 1] = off[k] + R[k];
    memset(nonmeet, 0, sizeof(uint64_t) * (size_t)n);
    const uint64_t total = off[n];
    const uint64_t chunk = 1u << 15;
    const int64_t nchunks = (int64_t)((total + chunk - 1) / chunk);
    uint64_t steps_total = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : steps_total)
#endif
    for (int64_t ch = 0; ch < nchunks; ++ch) {
        uint64_t g = (uint64_t)ch * chunk;
        uint64_t end = g + chunk < total ? g + chunk : total;
        /* node of global pair g: largest k with off[k] <= g and R[k] > 0 */
        int64_t lo = 0, hi = n;  /* off[lo] <= g < off[hi] */
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (off[mid] <= g) lo = mid; else hi = mid;
        }
        int64_t k = lo;
        uint64_t local = 0, steps = 0;
        while (g < end) {
            while (off[k + 1] <= g) ++k;
            uint64_t kend = off[k + 1] < end ? off[k + 1] : end;
            local = 0;
            const uint32_t d = depth ? depth[k] : 0u;
            for (; g < kend; ++g)
                local += (uint64_t)walk_pair(in_rowptr, in_col, (uint32_t)k, g - off[k], T, k0, k1, d, &steps);
#ifdef _OPENMP
#pragma omp atomic
#endif
            nonmeet[k] += local;
        }
        steps_total += steps;
    }
    free(off);
    return (int64_t)steps_total;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
