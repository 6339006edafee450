"""Pins of the oracle's Algorithm 3 (local deterministic exploitation).

* Lemma 5's recursion against exact rational first-meeting probabilities of two
  non-stop walks (brute force over pairs of nodes).
* The truncated sum of Z_l(k) stays below 1 - D(k) of the Power Method, and the
  special tail walks estimate the remainder without bias (z-test).
* The exploitation plan's rules, and the whole Algorithm 3 query within eps of
  the Power Method.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import alg3 as a3
from oracle import exactsim, power

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


def test_exploitation_plan_rules():
    n, rp, col = synth.chung_lu(400, 4000, gamma=2.1, seed=7)
    din = np.diff(rp)
    pi = np.random.default_rng(1).random(n) * 0.1
    pi[din == 0] = 0.05
    R_b = 1e12
    depth, R = a3.exploitation_plan(n, rp, col, pi, R_b, C, max_depth=6, min_pairs=1e6, max_nodes=10)
    assert np.all(R[din <= 1] == 0)
    assert 0 < np.count_nonzero(depth) <= 10
    top = np.lexsort((np.arange(n), -pi))[:10]
    for k in np.nonzero(depth)[0]:
        assert k in top and din[k] >= 2
        d = int(depth[k])
        assert 1 <= d <= 6
        assert R[k] == max(1, int(np.ceil(R_b * pi[k] ** 2 * C ** (2 * d))))
    other = (depth == 0) & (din >= 2)
    assert np.array_equal(R[other], np.maximum(1, np.ceil(R_b * pi[other] ** 2)).astype(np.uint64))
    # min_pairs above every count: nothing is exploited
    d0, _ = a3.exploitation_plan(n, rp, col, pi, R_b, C, min_pairs=1e30)
    assert np.count_nonzero(d0) == 0


def test_exploit_cost_limits():
    n, rp, col = synth.chung_lu(400, 4000, gamma=2.1, seed=8)
    m = int(rp[-1])
    P = a3.transition_matrix(n, rp, col)
    k = int(np.argmax(np.diff(rp)))
    supp = a3.supports(P, k, 6)
    assert supp[0] == 1 and supp[1] == np.diff(rp)[k]
    # Algorithm 2 alone costs its pairs times the mean walk length bound 1/(1-c)
    assert a3.exploit_cost(0, 1234.2, C, supp, n, m) == 1235 * (1 / (1 - C))
    # deeper exploitation never costs less deterministic work
    fixed = [a3.exploit_cost(d, 0.0, C, supp, n, m) for d in range(1, 9)]
    assert all(b > a for a, b in zip(fixed, fixed[1:]))
    # with overwhelming walk work the deepest depth wins, with little walk work none
    depth_hi, _ = a3.exploitation_plan(n, rp, col, np.eye(1, n, k)[0], 1e18, C, max_depth=8, min_pairs=1)
    assert depth_hi[k] == 8
    depth_lo, _ = a3.exploitation_plan(n, rp, col, np.eye(1, n, k)[0], 1e3, C, max_depth=8, min_pairs=1)
    assert depth_lo[k] == 0
    # max_depth caps the choice
    depth_1, R1 = a3.exploitation_plan(n, rp, col, np.eye(1, n, k)[0], 1e18, C, max_depth=1, min_pairs=1)
    assert depth_1[k] == 1 and R1[k] == int(np.ceil(1e18 * C ** 2))


def test_alg3_query_within_eps_of_power_method(oracle_walks):
    g = synth.erdos_renyi(300, 2400, seed=4)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 2e-3
    for u, seed in ((0, 1), (57, 2)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=2000.0, alg3=True, alg3_min_pairs=1e3)
        assert np.count_nonzero(q.depth) > 0 and q.depth.max() >= 3
        assert np.max(np.abs(q.s - S[:, u])) <= eps


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
