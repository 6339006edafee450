"""Pins of the oracle's Algorithm 3 (local deterministic exploitation).

* Lemma 5's recursion against exact rational first-meeting probabilities of two
  non-stop walks (brute force over pairs of nodes).
* The truncated sum of Z_l(k) stays below 1 - D(k) of the Power Method, and the
  special tail walks estimate the remainder without bias (z-test).
* The counter E_k of the adaptive depth against the listing's loops written out and
  against its closed form on the complete digraph; the depth rule (the level where
  E_k reaches 2 R(k)/sqrt(c)); an exploration that runs out of edges gives the Power
  Method's exact D; the whole Algorithm 3 query within eps of the Power Method.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import alg3 as a3
from oracle import exactsim, power
from oracle import linearization as lin

C = 0.6


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_lemma5_matches_bruteforce(seed):
    n = 7 if seed % 2 else 8
    g = synth.random_small(n, p=0.45, seed=seed)
    nn, rp, col = g
    din = np.diff(rp)
    for k in range(n):
        if din[k] == 0:
            continue
        z = a3.first_meeting_lemma5(nn, rp, col, k, C, 8)
        zb = [float(x) for x in a3.first_meeting_bruteforce(nn, rp, col, k, Fraction(3, 5), 8)]
        assert np.max(np.abs(np.array(z) - np.array(zb))) < 1e-14, (k, z, zb)


def test_truncated_meeting_mass_is_below_one_minus_D():
    g = synth.chung_lu(80, 600, gamma=2.1, seed=5)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    din = np.diff(rp)
    for k in np.nonzero(din >= 2)[0][:12]:
        z = a3.first_meeting_lemma5(n, rp, col, int(k), C, 3)
        assert all(x >= -1e-15 for x in z)
        assert sum(z) <= 1 - D[k] + 1e-12
        # one step: Z_1 = c * sum_a (1/din)^2 = c / din for a simple graph
        assert z[0] == pytest.approx(C / din[k], rel=1e-12)


def test_tail_walks_estimate_the_remainder(oracle_walks):
    g = synth.chung_lu(60, 500, gamma=2.1, seed=6)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    din = np.diff(rp)
    ks = [int(k) for k in np.nonzero(din >= 2)[0][:8]]
    R = np.zeros(n, dtype=np.uint64)
    depth = np.zeros(n, dtype=np.uint8)
    zsum = np.zeros(n)
    for i, k in enumerate(ks):
        d = 1 + i  # depths 1..8
        depth[k] = d
        R[k] = 300_000
        zsum[k] = sum(a3.first_meeting_lemma5(n, rp, col, k, C, d))
    counts, _ = oracle_walks.walk_pairs_depth(n, rp, col, R, depth, C, seed=3)
    Dh = a3.dhat_alg3(counts, R, depth, zsum, din, C)
    for k in ks:
        d = int(depth[k])
        p = (1 - D[k] - zsum[k]) / C ** d  # probability of a tail meeting
        sd = C ** d * np.sqrt(max(p * (1 - p), 1e-300) / 300_000)
        assert abs(Dh[k] - D[k]) < 5 * sd + 1e-12, (k, d, Dh[k], D[k])
    # depth 0 everywhere is Algorithm 2
    c0, _ = oracle_walks.walk_pairs_depth(n, rp, col, R, np.zeros(n, dtype=np.uint8), C, seed=3)
    c1, _ = oracle_walks.walk_pairs(n, rp, col, R, C, seed=3)
    assert np.array_equal(c0, c1)


def test_explored_edges_match_the_listing():
    """The vectorised counter equals the listing's loops written out, level by level."""
    for seed in range(1, 7):
        n, rp, col = synth.random_small(9, p=0.3 + 0.03 * seed, seed=seed)
        E = a3.explored_edges(n, rp, col, 6)
        for k in range(n):
            assert list(E[:, k]) == a3.explored_edges_literal(n, rp, col, k, 6), (seed, k)


def _complete_digraph(n):
    rp = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int64)
    col = np.array([i for j in range(n) for i in range(n) if i != j], dtype=np.int32)
    return n, rp, col


@pytest.mark.parametrize("n", [3, 4, 6])
def test_explored_edges_closed_form_complete_digraph(n):
    """K_n: supports |supp h_0| = 1, |supp h_1| = n-1, |supp h_j| = n (j >= 2), so the
    edges of one extension are e_0 = n-1, e_1 = (n-1)^2, e_j = n(n-1); level l adds
    sum_{l'} |supp h_(l-l')| e_l'."""
    _, rp, col = _complete_digraph(n)
    size = lambda j: 1 if j == 0 else (n - 1 if j == 1 else n)
    e = lambda j: n - 1 if j == 0 else ((n - 1) ** 2 if j == 1 else n * (n - 1))
    run, want = 0, []
    for ell in range(7):
        run += sum(size(ell - lp) * e(lp) for lp in range(ell + 1))
        want.append(run)
    E = a3.explored_edges(n, rp, col, 6)
    for k in range(n):
        assert list(E[:, k]) == want


def test_depth_rule_is_the_level_where_the_count_reaches_the_walk_work():
    """l(k) is the first level whose count reaches 2 R(k)/sqrt(c), capped by max_depth."""
    n, rp, col = _complete_digraph(5)
    E = a3.explored_edges(n, rp, col, 8)[:, 0]  # 4, 36, 96, ...
    T = lambda R: 2.0 * R / np.sqrt(C)
    for R in (1, 2, 3, 13, 14, 40, 10 ** 4, 10 ** 9):
        d = a3.paper_depth(E, R, C, 8)
        want = next((ell for ell in range(9) if E[ell] >= T(R)), 8)
        assert d == want, (R, d, want)
    assert a3.paper_depth(E, 10 ** 9, C, 3) == 3  # the cap
    # the threshold carries 1/sqrt(c): R = 14 needs 36.1 edges, which level 1 (36) misses
    assert a3.paper_depth(E, 14, C, 8) == 2 and a3.paper_depth(E, 13, C, 8) == 1


def test_exhausted_exploration_gives_the_exact_diagonal(oracle_walks):
    """Node 0 <- {1, 2}; 1 <- {3}; 2 <- {3, 4}; 3 and 4 have no in-edges.  Level 2 adds no
    edge, so the exploration stops there at any R: D^(0) = 1 - Z_1 - Z_2 with no tail
    meetings, equal to the Power Method's D(0)."""
    n = 5
    rp = np.array([0, 2, 3, 5, 5, 5], dtype=np.int64)
    col = np.array([1, 2, 3, 3, 4], dtype=np.int32)
    assert a3.explored_edges_literal(n, rp, col, 0, 4) == [2, 8, 8, 8, 8]
    E = a3.explored_edges(n, rp, col, 6)
    assert a3.paper_depth(E[:, 0], 10 ** 12, C, 16) == 2
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    pi = np.array([0.5, 0.2, 0.2, 0.05, 0.05])
    depth, R = a3.exploitation_plan(n, rp, col, pi, 1e8, C, max_depth=16)
    assert depth[0] == 2 and R[0] == int(np.ceil(1e8 * 0.25))
    assert np.all(R[[1, 3, 4]] == 0) and depth[1] == 0  # din 1 and 0: exact D, no pairs
    zsum = a3.first_meeting_sums(n, rp, col, depth, C)
    counts, _ = oracle_walks.walk_pairs_depth(n, rp, col, R, depth, C, seed=5)
    assert counts[0] == 0
    Dh = a3.dhat_alg3(counts, R, depth, zsum, np.diff(rp), C)
    assert abs(Dh[0] - D[0]) < 1e-15
    assert Dh[1] == 1 - C and Dh[3] == 1.0


def test_paper_plan_rules():
    n, rp, col = synth.chung_lu(300, 2400, gamma=2.1, seed=7)
    din = np.diff(rp)
    rng = np.random.default_rng(1)
    pi = rng.random(n) * 0.1
    pi[rng.random(n) < 0.1] = 0.0
    E = a3.explored_edges(n, rp, col, 12)
    for R_b, mode in ((1e6, "pi2"), (1e12, "pi2"), (1e7, "basic")):
        depth, R = a3.exploitation_plan(n, rp, col, pi, R_b, C, max_depth=12, mode=mode)
        R2 = lin.allocate(pi, R_b, mode)
        assert np.all(R[din <= 1] == 0) and np.all(depth[din <= 1] == 0)
        keep = din >= 2
        assert np.array_equal(R[keep], R2[keep])  # the paper keeps R(k) pairs
        assert np.all(depth[R == 0] == 0)
        for k in np.nonzero(R)[0]:
            T = 2.0 * float(R[k]) / np.sqrt(C)
            d = int(depth[k])
            assert E[d, k] >= T or d == 12 or (d > 0 and E[d, k] == E[d - 1, k])
            assert d == 0 or E[d - 1, k] < T
    # more pairs never explore less
    d_lo, _ = a3.exploitation_plan(n, rp, col, pi, 1e6, C, max_depth=12)
    d_hi, _ = a3.exploitation_plan(n, rp, col, pi, 1e12, C, max_depth=12)
    assert np.all(d_hi >= d_lo) and d_hi.max() > d_lo.max()


def test_first_meeting_sums_match_lemma5_term_by_term():
    for g, depth_max in ((synth.random_small(8, p=0.45, seed=3), 8), (synth.chung_lu(200, 1600, gamma=2.1, seed=9), 4)):
        n, rp, col = g
        rng = np.random.default_rng(2)
        depth = rng.integers(0, depth_max + 1, size=n).astype(np.uint8)
        zs = a3.first_meeting_sums(n, rp, col, depth, C)
        for k in range(min(n, 40)):
            want = sum(a3.first_meeting_lemma5(n, rp, col, k, C, int(depth[k]))) if depth[k] else 0.0
            assert abs(zs[k] - want) < 1e-14, (k, zs[k], want)


def test_alg3_query_within_eps_of_power_method(oracle_walks):
    g = synth.erdos_renyi(300, 2400, seed=4)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 2e-3
    for u, seed in ((0, 1), (57, 2)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=2000.0, alg3=True)
        assert q.depth.max() >= 3 and np.count_nonzero(q.depth) > 100
        assert np.max(np.abs(q.s - S[:, u])) <= eps


def test_alg3_given_plan_matches_algorithm2_at_depth_zero(oracle_walks):
    """A plan of depth 0 everywhere (R(k) of Algorithm 2) is Algorithm 2, bit for bit."""
    n, rp, col = synth.erdos_renyi(300, 2400, seed=4)
    q2 = exactsim.query(n, rp, col, 3, C, 1e-2, seed=4, kappa=50.0)
    q3 = exactsim.query(n, rp, col, 3, C, 1e-2, seed=4, kappa=50.0, alg3=True,
                        alg3_plan=(np.zeros(n, dtype=np.uint8), q2.R))
    assert np.array_equal(q2.nonmeet, q3.nonmeet)
    din = np.diff(rp)
    ok = din >= 2
    assert np.array_equal(q2.D[ok], q3.D[ok])


def test_planted_mistake_in_the_counter_is_caught():
    """Counting only the source's own distribution (dropping the l' < l extensions of
    the other walk distributions) fails the listing pin."""
    n, rp, col = synth.random_small(9, p=0.4, seed=2)
    E = a3.explored_edges(n, rp, col, 5)
    din = np.diff(rp).astype(np.float64)
    A = np.zeros((n, n))
    A[np.repeat(np.arange(n), np.diff(rp)), col] = 1.0
    supp = [np.eye(n)]
    for _ in range(5):
        supp.append(((supp[-1] @ A) > 0).astype(np.float64))
    wrong = np.cumsum([supp[ell] @ din for ell in range(6)], axis=0)
    lit = np.array([a3.explored_edges_literal(n, rp, col, k, 5) for k in range(n)]).T
    assert np.array_equal(E, lit)
    assert not np.array_equal(np.rint(wrong).astype(np.int64), lit)


def _lemma5_gap(g, depth=5):
    """Largest |Lemma 5 - rational brute force| over the nodes of a small graph."""
    nn, rp, col = g
    din = np.diff(rp)
    gap = 0.0
    for k in range(nn):
        if din[k] == 0:
            continue
        z = a3.first_meeting_lemma5(nn, rp, col, k, C, depth)
        zb = [float(x) for x in a3.first_meeting_bruteforce(nn, rp, col, k, Fraction(3, 5), depth)]
        gap = max(gap, float(np.max(np.abs(np.array(z) - np.array(zb)))))
    return gap


def test_planted_mistakes_in_lemma5_are_caught(monkeypatch):
    """Plausible mistakes planted in the oracle's Lemma 5 fail the brute-force pin."""
    g = synth.random_small(7, p=0.45, seed=1)
    assert _lemma5_gap(g) < 1e-14
    true_walk = a3.walk_distribution
    # (1) a transposed operand: the walks follow out-edges instead of in-edges
    true_tm = a3.transition_matrix
    monkeypatch.setattr(a3, "transition_matrix", lambda *args: true_tm(*args).T.tocsr())
    assert _lemma5_gap(g) > 1e-3
    monkeypatch.setattr(a3, "transition_matrix", true_tm)
    # (2) the l' >= 2 terms dropped: every walk distribution but the source's loses its
    # steps beyond the first
    calls = {"n": 0}

    def truncated(P, k, steps):
        H = true_walk(P, k, steps)
        calls["n"] += 1
        if calls["n"] > 1:
            H[2:] = 0.0
        return H

    def per_node(*args, **kw):
        calls["n"] = 0
        return lemma5(*args, **kw)

    lemma5 = a3.first_meeting_lemma5
    monkeypatch.setattr(a3, "walk_distribution", truncated)
    monkeypatch.setattr(a3, "first_meeting_lemma5", per_node)
    assert _lemma5_gap(g) > 1e-4
    monkeypatch.setattr(a3, "first_meeting_lemma5", lemma5)
    # (3) one step off: the distributions of the meeting terms taken a step early
    monkeypatch.setattr(a3, "walk_distribution",
                        lambda P, k, steps: np.vstack([true_walk(P, k, steps)[:1], true_walk(P, k, steps)[:-1]]))
    assert _lemma5_gap(g) > 1e-3


def test_planted_sign_in_the_tail_estimator_is_caught(oracle_walks):
    """D^ = 1 - sum Z - c^d tail/R (Algorithm 3); with the tail term's sign flipped the
    z-test against the Power Method's D fails."""
    g = synth.chung_lu(60, 500, gamma=2.1, seed=6)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    din = np.diff(rp)
    ks = [int(k) for k in np.nonzero(din >= 2)[0][:4]]
    R = np.zeros(n, dtype=np.uint64)
    depth = np.zeros(n, dtype=np.uint8)
    zsum = np.zeros(n)
    for k in ks:
        depth[k] = 1
        R[k] = 300_000
        zsum[k] = sum(a3.first_meeting_lemma5(n, rp, col, k, C, 1))
    counts, _ = oracle_walks.walk_pairs_depth(n, rp, col, R, depth, C, seed=3)
    right = a3.dhat_alg3(counts, R, depth, zsum, din, C)
    tail = C * counts.astype(np.float64) / np.maximum(R, 1).astype(np.float64)
    wrong = np.where(depth > 0, 1.0 - zsum + tail, right)
    for k in ks:
        p = (1 - D[k] - zsum[k]) / C
        sd = C * np.sqrt(max(p * (1 - p), 1e-300) / 300_000)
        assert abs(right[k] - D[k]) < 5 * sd + 1e-12
        assert abs(wrong[k] - D[k]) > 5 * sd
