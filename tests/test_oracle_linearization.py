"""Pins of O2: the deterministic steps of Algorithm 1 in the oracle.

Checks against hand-worked constants, closed forms (directed cycle), the Power
Method column (truncation bound of the proof of Theorem 1), the bilinear identity
(Eq. formula-ppr), and walk-mass conservation of the l-hop PPR vectors.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import linearization as lin
from oracle import power

C = 0.6
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_pairs(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = v
    return out


def test_levels_golden():
    for eps, L in _read_pairs("levels_c0.6.txt").items():
        assert lin.levels(C, float(eps)) == int(L)


def test_constants_golden():
    g = _read_pairs("constants_c0.6.txt")
    assert math.sqrt(C) == pytest.approx(float(g["sqrt_c"]), abs=1e-10)
    assert 1 - math.sqrt(C) == pytest.approx(float(g["a"]), abs=1e-10)
    assert lin.kappa_paper(C) == pytest.approx(float(g["kappa_paper"]), abs=1e-3)
    assert lin.pair_threshold(C) == int(g["T"])


def test_sample_base_formula():
    # R_b = 6 ln n / (a^4 eps^2) with the paper's constant
    n, eps = 2000, 1e-4
    a = 1 - math.sqrt(C)
    assert lin.sample_base(n, C, eps) == pytest.approx(6 * math.log(n) / (a ** 4 * eps ** 2), rel=1e-14)
    assert lin.sample_base(n, C, eps, kappa=1.0) == pytest.approx(math.log(n) / eps ** 2, rel=1e-14)


def test_allocate_hand_values():
    pi = np.array([0.5, 0.25, 0.0, 1e-3])
    # pi^2 = 0.25, 0.0625, 0, 1e-6 ; times 10 -> 2.5, 0.625, 0, 1e-5
    assert lin.allocate(pi, 10.0, "pi2").tolist() == [3, 1, 0, 1]
    # basic: 5, 2.5, 0, 0.01
    assert lin.allocate(pi, 10.0, "basic").tolist() == [5, 3, 0, 1]
    # exact integers stay
    assert lin.allocate(np.array([0.5]), 4.0, "pi2").tolist() == [1]
    # every reached node gets a pair, even when R_b = 0 (n = 1: ln n = 0) or pi^2 underflows
    assert lin.allocate(np.array([0.3, 0.0]), 0.0, "pi2").tolist() == [1, 0]
    assert lin.allocate(np.array([1e-200]), 1e12, "pi2").tolist() == [1]


def test_dhat_ratio():
    assert lin.dhat(np.array([3, 0, 5]), np.array([4, 0, 5])).tolist() == [0.75, 0.0, 1.0]


def test_cycle_closed_form():
    # on a directed cycle pi^l = a sqrt(c)^l e_{u-l} and, with D = (1-c) I, s = (1 - c^(L+1)) e_u
    n, u, L = 9, 4, 12
    g = synth.directed_cycle(n)
    H = lin.hop_vectors(*g, u, C, L)
    a = 1 - math.sqrt(C)
    for ell in range(L + 1):
        expect = np.zeros(n)
        expect[(u - ell) % n] = a * math.sqrt(C) ** ell
        assert np.allclose(H[ell], expect, atol=1e-16, rtol=1e-14)
    s = lin.reverse(*g, H, np.full(n, 1 - C), C)
    expect = np.zeros(n)
    expect[u] = 1 - C ** (L + 1)
    assert np.allclose(s, expect, atol=1e-15)


def test_mass_conservation_without_dangling_nodes():
    # each node has din >= 1, so no walk mass is lost: sum_k pi^l(k) = a sqrt(c)^l
    g = synth.complete_digraph(6)
    H = lin.hop_vectors(*g, 2, C, 15)
    a = 1 - math.sqrt(C)
    for ell in range(16):
        assert H[ell].sum() == pytest.approx(a * math.sqrt(C) ** ell, rel=1e-13)


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
@pytest.mark.parametrize("gen", ["er", "dangling"])
def test_exact_D_sweeps_match_power_method(eps, gen):
    # with the exact D, s^L differs from S e_u only by the truncated tail <= c^(L+1) / (1-c)
    g = synth.erdos_renyi(200, 1600, seed=2) if gen == "er" else synth.with_dangling(200, 1200, seed=3)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    L = lin.levels(C, eps)
    for u in (0, 17, 123):
        H = lin.hop_vectors(n, rp, col, u, C, L)
        s = lin.reverse(n, rp, col, H, D, C)
        err = np.max(np.abs(s - S[:, u]))
        assert err <= C ** (L + 1) / (1 - C) + 1e-12
        assert err <= eps / 2 + 1e-12


def test_bilinear_identity_matches_horner():
    g = synth.chung_lu(300, 3000, gamma=2.1, seed=5)
    n, rp, col = g
    D = synth.uniform_diagonal(n, C, seed=8)
    L = 14
    u = 7
    Hu = lin.hop_vectors(n, rp, col, u, C, L)
    s = lin.reverse(n, rp, col, Hu, D, C)
    for j in (0, 7, 42, 299):
        Hj = lin.hop_vectors(n, rp, col, j, C, L)
        assert lin.bilinear(Hu, Hj, D, C) == pytest.approx(s[j], abs=1e-14)


def test_planted_mistake_reverse_with_P_instead_of_PT_is_caught():
    g = synth.chung_lu(200, 2000, gamma=2.1, seed=6)
    n, rp, col = g
    D = synth.uniform_diagonal(n, C, seed=9)
    L, u = 10, 3
    Hu = lin.hop_vectors(n, rp, col, u, C, L)
    P = power.transition_matrix(n, rp, col)
    a = 1 - math.sqrt(C)
    s = D * Hu[L] / a
    for ell in range(1, L + 1):
        s = math.sqrt(C) * (P @ s) + D * Hu[L - ell] / a  # wrong operand
    ref = np.array([lin.bilinear(Hu, lin.hop_vectors(n, rp, col, j, C, L), D, C) for j in range(20)])
    assert np.max(np.abs(s[:20] - ref)) > 1e-6


def test_topk_order_ties_and_exclusion():
    s = np.array([0.5, 0.9, 0.5, 0.1, 0.9, 1.0])
    ids, vals = lin.topk(s, 4, exclude=5)
    assert ids.tolist() == [1, 4, 0, 2]
    assert vals.tolist() == [0.9, 0.9, 0.5, 0.5]
    ids, _ = lin.topk(s, 2, exclude=None)
    assert ids.tolist() == [5, 1]
