"""Pins of the Power Method oracle (O1) and of the exact diagonal correction D.

Every check here compares against something other than the oracle itself (and runs
for both the NumPy/SciPy Power Method and its C restatement):
closed forms derived from the SimRank definition (Eq. intro-simrank), an exact
rational solve of the walk-meeting chain (Eq. scwwalk), and the invariants the
paper states for D (Eq. def-lsim2: 1-c <= D <= 1; Algorithm 3: din=0 -> 1,
din=1 -> 1-c).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import pair_chain, power

C = 0.6


_IMPL = {"name": "python"}


@pytest.fixture(autouse=True, params=["python", "c"])
def impl(request):
    """Every pin runs against both implementations of the Power Method (NumPy/SciPy and
    the C one with OpenMP that the larger tests use)."""
    _IMPL["name"] = request.param
    yield request.param


def _S(g, c=C):
    n, rp, col = g
    if _IMPL["name"] == "c":
        return power.power_method_c(n, rp, col, c)
    return power.power_method(n, rp, col, c)


def test_out_star_closed_form():
    # leaves share the single in-neighbour 0: S(leaf, leaf') = c; S(0, leaf) = 0 (din(0) = 0)
    S = _S(synth.out_star(5))
    for i in range(1, 6):
        for j in range(1, 6):
            assert S[i, j] == pytest.approx(1.0 if i == j else C, abs=1e-15)
        assert S[0, i] == 0.0 and S[i, 0] == 0.0


def test_in_star_all_off_diagonal_zero():
    S = _S(synth.in_star(6))
    assert np.allclose(S, np.eye(7), atol=0.0)


def test_directed_cycle_is_identity_and_D_is_1_minus_c():
    g = synth.directed_cycle(7)
    S = _S(g)
    assert np.allclose(S, np.eye(7), atol=0.0)
    D = power.exact_diagonal(*g, C, S)
    assert np.allclose(D, 1.0 - C, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_complete_digraph_closed_form(n):
    # s = c(n-2) / ((1-c)(n-1)^2 + c(n-2)) for i != j
    S = _S(synth.complete_digraph(n))
    s = C * (n - 2) / ((1 - C) * (n - 1) ** 2 + C * (n - 2))
    off = S[~np.eye(n, dtype=bool)]
    assert np.allclose(off, s, atol=1e-13)


def test_two_parents_closed_form():
    S = _S(synth.two_parents())
    assert S[2, 3] == pytest.approx(C / 2, abs=1e-15)
    assert S[0, 1] == 0.0


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_power_method_matches_exact_rational_meeting_probability(seed):
    n = 6 if seed % 2 else 8
    g = synth.random_small(n, p=0.35, seed=seed, loops=(seed == 5))
    S = _S(g)
    exact = pair_chain.to_float(pair_chain.meeting_matrix(*g, Fraction(3, 5)))
    assert np.max(np.abs(S - exact)) < 1e-13


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_exact_D_matches_rational_first_meeting(seed):
    g = synth.random_small(7, p=0.4, seed=seed)
    S = _S(g)
    D = power.exact_diagonal(*g, C, S)
    exact = pair_chain.to_float(pair_chain.exact_diagonal_rational(*g, Fraction(3, 5)))
    assert np.max(np.abs(D - exact)) < 1e-13


def test_structural_invariants_on_er_graph():
    g = synth.erdos_renyi(300, 2400, seed=4)
    n, rp, col = g
    S = _S(g)
    assert np.allclose(np.diag(S), 1.0)
    assert np.max(np.abs(S - S.T)) < 1e-14
    assert S.min() >= 0.0 and S.max() <= 1.0
    D = power.exact_diagonal(n, rp, col, C, S)
    din = np.diff(rp)
    assert np.all(D >= 1 - C - 1e-12) and np.all(D <= 1 + 1e-12)
    assert np.allclose(D[din == 0], 1.0)
    assert np.allclose(D[din == 1], 1.0 - C, atol=1e-13)


def test_D_reconstructs_S_through_linearization():
    # Eq. def-lsim2: S = sum_l c^l (P^l)^T D P^l
    g = synth.with_dangling(40, 200, seed=9)
    n, rp, col = g
    S = _S(g)
    D = power.exact_diagonal(n, rp, col, C, S)
    P = power.transition_matrix(n, rp, col).toarray()
    acc = np.zeros((n, n))
    Pl = np.eye(n)
    for ell in range(80):
        acc += C ** ell * Pl.T @ np.diag(D) @ Pl
        Pl = P @ Pl
    assert np.max(np.abs(acc - S)) < 1e-12


def test_planted_transpose_is_caught():
    # a transposed P (walks along out-edges) changes S on an asymmetric graph
    g = synth.random_small(6, p=0.35, seed=21)
    n, rp, col = g
    S = _S(g)
    exact = pair_chain.to_float(pair_chain.meeting_matrix(*g, Fraction(3, 5)))
    # build the reversed graph and check that it disagrees with the true answer
    src = np.asarray(col)
    dst = np.repeat(np.arange(n), np.diff(rp))
    rev = synth.edges_to_in_csr(n, dst, src)
    S_rev = power.power_method(*rev, C)
    assert np.max(np.abs(S - exact)) < 1e-13
    assert np.max(np.abs(S_rev - exact)) > 1e-3
