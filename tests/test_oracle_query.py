"""The whole CPU ExactSim query against the Power Method (Theorem 1).

With the paper's constant (kappa = 6 / (1 - sqrt c)^4) Theorem 1 says every
|s(v) - S(u, v)| <= eps with probability at least 1 - 1/n.  The checks use fixed
seeds, so they are deterministic.
"""
import numpy as np
import pytest

import synth
from oracle import exactsim, power

C = 0.6


@pytest.mark.parametrize("mode", ["pi2", "basic"])
def test_cpu_exactsim_within_eps_of_power_method(oracle_walks, mode):
    g = synth.erdos_renyi(300, 2400, seed=4)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 2e-2 if mode == "basic" else 5e-3
    for u, seed in ((0, 1), (57, 2)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, mode=mode)
        err = np.max(np.abs(q.s - S[:, u]))
        assert err <= eps, (u, err)
        assert q.R.sum() > 0


def test_cpu_exactsim_power_law_graph(oracle_walks):
    g = synth.chung_lu(400, 4000, gamma=2.1, seed=13)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 5e-3
    u = int(synth.random_sources(rp, 1, seed=3)[0])
    q = exactsim.query(n, rp, col, u, C, eps, seed=7)
    assert np.max(np.abs(q.s - S[:, u])) <= eps


def test_lemma2_variance_bound_holds_empirically(oracle_walks):
    """Lemma 2 with the pi^2 allocation bounds Var s(v) by ||pi_v||^2 / (4 a^4 R_b)
    (a = 1 - sqrt c): the bound the benchmark reports as its sampling sigma.  The
    variance over 200 seeds stays under it, and is not zero (the test has power)."""
    from oracle import linearization as lin
    n, rp, col = synth.chung_lu(300, 2400, gamma=2.1, seed=12)
    u, eps, kappa = 5, 1e-2, 0.5
    a = 1.0 - np.sqrt(C)
    runs = np.array([exactsim.query(n, rp, col, u, C, eps, seed=s, kappa=kappa).s for s in range(200)])
    R_b = lin.sample_base(n, C, eps, kappa)
    L = lin.levels(C, eps)
    var = runs.var(axis=0, ddof=1)
    checked = 0
    for v in [u] + [int(x) for x in np.argsort(-runs.mean(axis=0))[1:6]]:
        norm_v = float(np.sum(lin.ppr(lin.hop_vectors(n, rp, col, v, C, L)) ** 2))
        bound = norm_v / (4 * a ** 4 * R_b)
        assert 0 < var[v] <= 1.3 * bound, (v, var[v], bound)
        checked += 1
    assert checked == 6


def test_topk_convergence_protocol_against_the_power_method(oracle_walks):
    """The top-k check the large-graph tests use (Sec. 4): with both queries within their
    eps, every node of the top-k at the coarse eps scores, in the fine query, at least the
    fine k-th best minus 2 (eps_c + eps_f); against the exact S, every returned node has
    S(u, v) >= S_k - 2 eps_c (Precision@k up to ties within the error)."""
    from oracle import linearization as lin
    n, rp, col = synth.chung_lu(400, 4000, gamma=2.1, seed=13)
    S = power.power_method(n, rp, col, C)
    k, eps_c, eps_f = 20, 1e-2, 1e-3
    for u in [int(x) for x in synth.random_sources(rp, 3, seed=5)]:
        coarse = exactsim.query(n, rp, col, u, C, eps_c, seed=1, kappa=16.0).s
        fine = exactsim.query(n, rp, col, u, C, eps_f, seed=2, kappa=16.0).s
        ids, _ = lin.topk(coarse, k, exclude=u)
        t_fine = np.sort(np.delete(fine, u))[::-1][k - 1]
        assert np.all(fine[ids] >= t_fine - 2 * (eps_c + eps_f))
        s_k = np.sort(np.delete(S[:, u], u))[::-1][k - 1]
        assert np.all(S[ids, u] >= s_k - 2 * eps_c)
