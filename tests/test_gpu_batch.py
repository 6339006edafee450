"""GPU tests of batched queries (multi-RHS sweeps, per-source eps, one seed).

* Accuracy: every column of a batch lies within its own eps of the Power Method
  (Theorem 1 with the paper's R) on the small ER workload.
* A column does not depend on the rest of the batch: a query alone (B = 1) and in
  mixes of other sources, at other positions and widths (W = 32, 64), gives
  bit-identical scores; so do all tile shapes the autotuner may pick.
* Batched top-k is the top-k of the batched scores.
"""
import numpy as np
import pytest

import synth
from oracle import linearization as lin

pytestmark = pytest.mark.gpu

C = 0.6


@pytest.fixture(scope="module")
def esim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    import paper_2004_03493_gb300 as pkg
    pkg.build()
    return pkg


def test_batch_columns_within_eps_of_power_method(esim):
    from oracle import power
    n, rp, col = synth.erdos_renyi(2000, 20000, seed=1)
    S = power.power_method(n, rp, col, C)
    g = esim.Graph(n, rp, col)
    u = np.array([0, 17, 1999, 512], dtype=np.int64)
    eps = np.array([1e-4, 1e-3, 1e-2, 3e-4])
    s = g.query_batch(u, eps, C, seed=3)
    for q in range(u.size):
        err = np.max(np.abs(s[q] - S[:, u[q]]))
        assert err <= eps[q], (q, err)
    g.close()


def test_column_is_bit_identical_alone_and_in_any_mix(esim):
    n, rp, col = synth.chung_lu(6000, 60000, gamma=2.1, seed=4)
    g = esim.Graph(n, rp, col, kappa=0.5)
    srcs = synth.random_sources(rp, 50, seed=9)
    eps = np.exp(np.random.default_rng(1).uniform(np.log(1e-5), np.log(1e-2), size=50))
    target, t_eps = int(srcs[0]), float(eps[0])
    alone = g.query_batch([target], [t_eps], C, seed=11)[0]
    mix1 = g.query_batch(np.r_[srcs[1:6], target], np.r_[eps[1:6], t_eps], C, seed=11)  # W = 32, last position
    assert np.array_equal(mix1[-1], alone)
    mix2 = g.query_batch(np.r_[srcs[1:20], target, srcs[20:45]], np.r_[eps[1:20], t_eps, eps[20:45]], C,
                         seed=11)  # W = 64, middle
    assert np.array_equal(mix2[19], alone)
    # the other columns of mix1 are also unchanged by the company they keep
    for j in range(5):
        single = g.query_batch([srcs[1 + j]], [eps[1 + j]], C, seed=11)[0]
        assert np.array_equal(mix1[j], single)
    g.close()


def test_every_tile_shape_gives_the_same_bits(esim):
    n, rp, col = synth.chung_lu(8000, 120000, gamma=2.1, seed=5)  # hub rows: long-row segments in both CSRs
    srcs = synth.random_sources(rp, 40, seed=2)
    eps = np.full(40, 1e-3)
    ref = None
    for tile in (0, 1, 2):
        g = esim.Graph(n, rp, col, kappa=0.2, batch_tile=tile)
        s = g.query_batch(srcs, eps, C, seed=5)
        if ref is None:
            ref = s
        else:
            assert np.array_equal(s, ref), tile
        g.close()
    g = esim.Graph(n, rp, col, kappa=0.2)  # autotuned
    assert np.array_equal(g.query_batch(srcs, eps, C, seed=5), ref)
    assert g.get_option("batch_tile_fwd64") in (0, 1, 2)
    g.close()


def test_batch_is_close_to_single_precision_queries(esim):
    # different summation orders: the two differ by FP32 rounding and the sampling
    # noise of slightly different R(k); both are within eps of each other here
    n, rp, col = synth.erdos_renyi(1500, 12000, seed=6)
    g = esim.Graph(n, rp, col, precision=1)
    u = np.array([3, 77], dtype=np.int64)
    eps = np.array([1e-3, 3e-3])
    s = g.query_batch(u, eps, C, seed=8)
    for q in range(2):
        single = g.query(int(u[q]), C, float(eps[q]), 8)
        assert np.max(np.abs(single - s[q])) <= eps[q]
    g.close()


def test_batch_topk_and_limits(esim):
    n, rp, col = synth.chung_lu(5000, 50000, gamma=2.1, seed=7)
    g = esim.Graph(n, rp, col, kappa=0.5)
    u = synth.random_sources(rp, 33, seed=4)
    eps = np.full(33, 1e-3)
    s = g.query_batch(u, eps, C, seed=2)
    ids, vals = g.topk_batch(u, eps, C, 25, seed=2)
    for q in range(u.size):
        ids_ref, vals_ref = lin.topk(s[q], 25, exclude=int(u[q]))
        assert np.array_equal(ids[q], ids_ref) and np.array_equal(vals[q], vals_ref)
    with pytest.raises(esim.EsimError) as e:
        g.query_batch(np.zeros(65, dtype=np.int64), np.full(65, 1e-2), C)
    assert e.value.status == -6
    with pytest.raises(esim.EsimError) as e:
        g.query_batch([n], [1e-2], C)
    assert e.value.status == -1
    g.close()


def test_shared_walks_give_the_same_counts_with_fewer_pairs(esim):
    n, rp, col = synth.chung_lu(6000, 60000, gamma=2.1, seed=5)
    srcs = synth.random_sources(rp, 40, seed=2)
    srcs[5] = srcs[4]  # the same source twice: identical thresholds share every interval
    eps = np.exp(np.random.default_rng(3).uniform(np.log(1e-5), np.log(1e-2), size=40))
    eps[5] = eps[4]
    g1 = esim.Graph(n, rp, col, kappa=0.5)
    g0 = esim.Graph(n, rp, col, kappa=0.5, shared_walks=0)
    assert g1.get_option("shared_walks") == 1.0
    s1 = g1.query_batch(srcs, eps, C, seed=7)
    st1 = g1.stats()
    s0 = g0.query_batch(srcs, eps, C, seed=7)
    st0 = g0.stats()
    assert np.array_equal(s1, s0)
    assert np.array_equal(s1[4], s1[5])
    assert st1["sum_R"] < st0["sum_R"]
    assert st1["pair_steps"] < st0["pair_steps"]
    # top-k through the shared path equals the unshared one
    ids1, v1 = g1.topk_batch(srcs[:8], eps[:8], C, 20, seed=7)
    ids0, v0 = g0.topk_batch(srcs[:8], eps[:8], C, 20, seed=7)
    assert np.array_equal(ids1, ids0) and np.array_equal(v1, v0)
    g1.close()
    g0.close()
