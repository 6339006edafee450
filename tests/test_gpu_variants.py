"""GPU parity of the method's variants through the C ABI: sparse Linearization
(Sec. 3.2), ParSim's D = (1 - c) I (Sec. 2), and the basic allocation (Algorithm 1)
as used by the ablation.

Integers (L, R(k) totals, pair steps, kept history entries) must match the oracle
exactly; scores within 1e-12.  Where a floating-point comparison decides an
integer (ceil(R_b pi^2), pi^l(k) > theta) and the oracle's value lies within
rounding of the boundary, that source is skipped (the two sides sum in different
orders).
"""
import numpy as np
import pytest

import synth
from oracle import exactsim, power
from oracle import linearization as lin

pytestmark = pytest.mark.gpu

C = 0.6
TOL = 1e-12


@pytest.fixture(scope="module")
def esim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    import paper_2004_03493_gb300 as pkg
    pkg.build()
    return pkg


def _clean(q, graph, u, c, eps_q):
    """No integer decision of this query sits within rounding of its boundary."""
    n, rp, col = graph
    v = q.R_b * (q.pi * q.pi)
    frac = np.abs(v - np.round(v))
    if not np.all((frac > 1e-12 * v) | (v == 0)):
        return False
    theta = lin.sparse_threshold(c, eps_q)
    H = lin.hop_vectors(n, rp, col, u, c, q.L)
    return bool(np.all(np.abs(H - theta) > 1e-12 * theta))


@pytest.mark.parametrize("alg3", [False, True])
def test_sparse_query_matches_cpu_exactsim(esim, oracle_walks, alg3):
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, kappa=2.0, sparse_hist=1)
    if alg3:
        g.set_option("alg3", 1)  # the paper's adaptive depth
    eps = 1e-3
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=2.0, sparse=True, alg3=alg3)
        if not _clean(q, (n, rp, col), u, C, eps / 2):
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["L"] == q.L == lin.levels(C, eps / 2)
        assert st["R_b"] == q.R_b
        assert st["hist_entries"] == int(np.count_nonzero(q.H))
        assert st["hist_entries"] < (q.L + 1) * n
        assert st["sum_R"] == int(q.R.sum())
        assert st["pair_steps"] == q.pair_steps
        if alg3:
            assert st["alg3_nodes"] == int(np.count_nonzero(q.depth))
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    g.close()


def test_sparse_within_eps_and_smaller_workspace(esim):
    n, rp, col = synth.erdos_renyi(2000, 20000, seed=1)
    S = power.power_method(n, rp, col, C)
    eps = 1e-3
    g = esim.Graph(n, rp, col, sparse_hist=1)
    s = g.query(0, C, eps, 0)
    assert np.max(np.abs(s - S[:, 0])) <= eps
    g.close()
    # a graph large enough for the pigeonhole capacity to undercut the dense history
    n, rp, col = synth.chung_lu(200_000, 1_000_000, gamma=2.1, seed=4)
    gd = esim.Graph(n, rp, col, kappa=0.01)
    gs = esim.Graph(n, rp, col, kappa=0.01, sparse_hist=1)
    u = int(np.argmax(np.diff(rp)))
    sd = gd.query(u, C, 1e-4, 1)
    ss = gs.query(u, C, 1e-4, 1)
    std, sts = gd.stats(), gs.stats()
    assert sts["workspace_bytes"] < std["workspace_bytes"] / 2
    assert sts["hist_entries"] < 1.0 / lin.sparse_threshold(C, 0.5e-4)
    assert std["hist_entries"] == (std["L"] + 1) * n
    assert np.isfinite(ss).all() and ss[u] > 0.2
    gd.close()
    gs.close()
    # precision FP32c and the sparse history exclude each other
    g = esim.Graph(n, rp, col, precision=1)
    with pytest.raises(esim.EsimError) as e:
        g.set_option("sparse_hist", 1)
    assert e.value.status == -6
    g.close()


def test_parsim_diagonal_matches_oracle(esim):
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, diag=1)
    for u in (5, 2999):
        q = exactsim.query(n, rp, col, u, C, 1e-4, diag="parsim")
        s = g.query(u, C, 1e-4, 0)
        st = g.stats()
        assert st["sum_R"] == 0 and st["pair_steps"] == 0
        assert np.max(np.abs(s - q.s)) <= TOL
    # with the sparse history as well
    g.set_option("sparse_hist", 1)
    q = exactsim.query(n, rp, col, 5, C, 1e-4, diag="parsim", sparse=True)
    theta = lin.sparse_threshold(C, 0.5e-4)
    H = lin.hop_vectors(n, rp, col, 5, C, q.L)
    assert np.all(np.abs(H - theta) > 1e-12 * theta)  # no keep/drop decision within rounding
    s = g.query(5, C, 1e-4, 0)
    assert np.max(np.abs(s - q.s)) <= TOL
    g.close()


def test_basic_allocation_query_matches_cpu_exactsim(esim, oracle_walks):
    n, rp, col = synth.erdos_renyi(2000, 16000, seed=4)
    g = esim.Graph(n, rp, col, alloc=1)
    eps = 3e-2
    checked = 0
    for u, seed in ((0, 1), (999, 2), (1999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, mode="basic")
        v = q.R_b * q.pi
        frac = np.abs(v - np.round(v))
        if not np.all((frac > 1e-12 * v) | (v == 0)):
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["sum_R"] == int(q.R.sum()) and st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    g.close()
