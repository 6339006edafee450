"""The seeded input generators keep the recipes that stand in for the paper's datasets.

* Every generator returns a valid in-edge CSR (rows sorted by source id) with exactly
  the requested m distinct edges and no self-loops, and depends only on its seed.
* Erdos-Renyi in-degrees have the binomial's variance (about their mean).
* Chung-Lu in-degrees have the power-law tail of the Pareto weights: the Hill estimate
  of the tail exponent of P(din > x) is near gamma - 1, and the top 1 % of nodes hold a
  large share of the in-edges (the hubs of the power-law graphs of Table 2).
* R-MAT is skewed likewise; sources have in-edges; D values lie in [1 - c, 1].
"""
import numpy as np
import pytest

import synth


def _check_csr(n, rp, col, m):
    rp = np.asarray(rp)
    col = np.asarray(col)
    assert rp.dtype == np.int64 and col.dtype == np.int32
    assert rp.size == n + 1 and rp[0] == 0 and rp[-1] == m == col.size
    assert np.all(np.diff(rp) >= 0)
    assert col.min() >= 0 and col.max() < n
    dst = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(dst == col)  # no self-loops
    keys = dst.astype(np.int64) * n + col
    assert np.unique(keys).size == m  # no repeated edges
    # within a row the sources ascend
    same_row = dst[1:] == dst[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])


def _hill_tail_exponent(deg, frac=0.01):
    x = np.sort(deg[deg > 0])[::-1].astype(np.float64)
    k = max(10, int(x.size * frac))
    return 1.0 / np.mean(np.log(x[:k] / x[k]))


def _top_share(deg, frac=0.01):
    top = np.sort(deg)[::-1]
    return top[: max(1, int(deg.size * frac))].sum() / deg.sum()


def test_erdos_renyi_recipe():
    n, rp, col = synth.erdos_renyi(2000, 20000, seed=1)
    _check_csr(n, rp, col, 20000)
    din = np.diff(rp)
    assert 0.8 < din.var() / din.mean() < 1.2
    assert _top_share(din) < 0.05
    n2, rp2, col2 = synth.erdos_renyi(2000, 20000, seed=1)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    _, rp3, col3 = synth.erdos_renyi(2000, 20000, seed=2)
    assert not np.array_equal(col, col3)


@pytest.mark.parametrize("gamma", [2.1, 2.2])
def test_chung_lu_recipe(gamma):
    n, rp, col = synth.chung_lu(20000, 200000, gamma=gamma, seed=2)
    _check_csr(n, rp, col, 200000)
    din = np.diff(rp)
    dout = np.bincount(col, minlength=n)
    for deg in (din, dout):
        assert abs(_hill_tail_exponent(deg) - (gamma - 1.0)) < 0.3
        assert _top_share(deg) > 0.25
    _, rp2, col2 = synth.chung_lu(20000, 200000, gamma=gamma, seed=2)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_chung_lu_torch_recipe():
    """The torch generator of the largest Chung-Lu graph keeps the recipe (run on the CPU)."""
    pytest.importorskip("torch")
    gamma = 2.2
    n, rp, col = synth.chung_lu_torch(200_000, 2_000_000, gamma=gamma, seed=2, device="cpu")
    _check_csr(n, rp, col, 2_000_000)
    din = np.diff(rp)
    dout = np.bincount(col, minlength=n)
    for deg in (din, dout):
        assert abs(_hill_tail_exponent(deg) - (gamma - 1.0)) < 0.3
        assert _top_share(deg) > 0.25
    _, rp2, col2 = synth.chung_lu_torch(200_000, 2_000_000, gamma=gamma, seed=2, device="cpu")
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)


def test_rmat_recipe():
    n, rp, col = synth.rmat(14, 200_000, seed=1)
    assert n == 1 << 14
    _check_csr(n, rp, col, 200_000)
    assert _top_share(np.diff(rp)) > 0.2


def test_sources_diagonal_and_dangling_nodes():
    n, rp, col = synth.with_dangling(3001, 15000, seed=5)
    _check_csr(n, rp, col, 15000)
    din = np.diff(rp)
    k = int(3001 * 0.2)
    assert k / n <= np.mean(din == 0) <= k / n + 0.01
    src = synth.random_sources(rp, 500, seed=7)
    assert np.all(din[src] >= 1)
    assert np.array_equal(src, synth.random_sources(rp, 500, seed=7))
    D = synth.uniform_diagonal(1000, 0.6, seed=3)
    assert np.all((D >= 0.4) & (D <= 1.0))
