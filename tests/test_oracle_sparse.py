"""Pins of the oracle's sparse Linearization (Sec. 3.2) and ParSim diagonal (Sec. 2).

* The sparse-linearization lemma: with the exact D, dropping the history entries
  at or below (1 - sqrt c)^2 eps moves every score by at most eps; fewer than
  1 / threshold entries survive (pigeonhole over sum_l sum_k pi^l(k) <= 1).
* The reverse loop over a sparsified history equals the bilinear form evaluated
  with the sparsified source side (an independent formulation).
* The whole sparse query stays within eps of the Power Method.
* ParSim's D = (1 - c) I is exact on a directed cycle (D = (1 - c) I there), and
  differs from SimRank where first meetings matter.
"""
import numpy as np
import pytest

import synth
from oracle import exactsim, power
from oracle import linearization as lin

C = 0.6


@pytest.mark.parametrize("eps", [1e-2, 3e-3, 1e-3])
def test_sparse_lemma_bound_with_exact_D(eps):
    n, rp, col = synth.chung_lu(300, 2400, gamma=2.1, seed=12)
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    L = lin.levels(C, eps)
    theta = lin.sparse_threshold(C, eps)
    assert theta == pytest.approx((1 - np.sqrt(C)) ** 2 * eps, rel=1e-15)
    for u in (0, 17, 123):
        H = lin.hop_vectors(n, rp, col, u, C, L)
        Hs = lin.sparsify(H, theta)
        kept = int(np.count_nonzero(Hs))
        assert 0 < kept < 1.0 / theta
        assert kept < np.count_nonzero(H)  # the threshold bites on these sizes
        dense = lin.reverse(n, rp, col, H, D, C)
        sp = lin.reverse(n, rp, col, Hs, D, C)
        assert np.all(sp <= dense + 1e-15)  # dropping non-negative terms only lowers scores
        assert np.max(dense - sp) <= eps
        # the truncated dense result is within c^(L+1) of S, so sparse is within eps + c^(L+1)
        assert np.max(np.abs(sp - S[:, u])) <= eps + C ** (L + 1) + 1e-12


def test_sparsify_keeps_strictly_above_threshold():
    up = float(np.nextafter(1e-3, 1.0))
    H = np.array([[0.5, 0.0, 1e-3], [2e-3, float(np.nextafter(1e-3, 0.0)), up]])
    Hs = lin.sparsify(H, 1e-3)
    assert Hs.tolist() == [[0.5, 0.0, 0.0], [2e-3, 0.0, up]]
    # threshold 0 keeps every positive entry
    assert np.array_equal(lin.sparsify(H, 0.0), H)


def test_sparse_reverse_matches_bilinear_form():
    n, rp, col = synth.erdos_renyi(200, 1400, seed=3)
    eps = 2e-3
    L = lin.levels(C, eps)
    D = synth.uniform_diagonal(n, C, seed=5)
    theta = lin.sparse_threshold(C, eps)
    Hu = lin.sparsify(lin.hop_vectors(n, rp, col, 4, C, L), theta)
    s = lin.reverse(n, rp, col, Hu, D, C)
    for j in (0, 4, 77, 199):
        Hj = lin.hop_vectors(n, rp, col, j, C, L)
        assert s[j] == pytest.approx(lin.bilinear(Hu, Hj, D, C), abs=1e-13)


def test_sparse_query_within_eps_of_power_method(oracle_walks):
    n, rp, col = synth.erdos_renyi(300, 2400, seed=4)
    S = power.power_method(n, rp, col, C)
    eps = 4e-3
    q = exactsim.query(n, rp, col, 5, C, eps, seed=1, kappa=16.0, sparse=True)
    assert q.L == lin.levels(C, eps / 2)
    assert q.R_b == lin.sample_base(n, C, eps / 2, 16.0)
    assert np.max(np.abs(q.s - S[:, 5])) <= eps
    # with Algorithm 3 as well
    q3 = exactsim.query(n, rp, col, 5, C, eps, seed=2, kappa=400.0, sparse=True, alg3=True)
    assert np.count_nonzero(q3.depth) > 0
    assert np.max(np.abs(q3.s - S[:, 5])) <= eps


def test_parsim_diagonal():
    # directed cycle: D = (1 - c) I exactly, so ParSim's answer is ExactSim's exact-D answer
    n, rp, col = synth.directed_cycle(11)
    q = exactsim.query(n, rp, col, 3, C, 1e-4, diag="parsim")
    expect = np.zeros(n)
    expect[3] = 1.0 - C ** (q.L + 1)
    assert np.max(np.abs(q.s - expect)) <= 1e-14
    assert q.pair_steps == 0 and int(q.R.sum()) == 0
    # on a graph where two walks can first-meet, D differs from (1-c) and so do the scores
    n, rp, col = synth.chung_lu(200, 1600, gamma=2.1, seed=9)
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    assert np.max(np.abs(D - (1 - C))) > 0.05
    q = exactsim.query(n, rp, col, 0, C, 1e-4, diag="parsim")
    assert np.max(np.abs(q.s - S[:, 0])) > 1e-3


def test_planted_threshold_without_the_square_factor_is_caught():
    """A threshold of eps (the (1 - sqrt c)^2 factor dropped) breaks the lemma's bound."""
    n, rp, col = synth.chung_lu(300, 2400, gamma=2.1, seed=12)
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    eps = 3e-3
    L = lin.levels(C, eps)
    worst = 0.0
    for u in (0, 17, 123):
        H = lin.hop_vectors(n, rp, col, u, C, L)
        dense = lin.reverse(n, rp, col, H, D, C)
        worst = max(worst, float(np.max(dense - lin.reverse(n, rp, col, lin.sparsify(H, eps), D, C))))
    assert worst > eps
