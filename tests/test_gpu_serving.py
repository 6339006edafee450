"""GPU tests of the serving loop (continuous batching).

* Every request answered in a mix of concurrent waves gets bit-identical top-k ids
  and scores to the same request served alone.
* Requests submitted while earlier waves are on the GPU are admitted and served.
* Waits are bounded (ESIM_ETIMEOUT), bad requests are rejected on the host, and a
  server destroyed with queued requests returns without hanging.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

C = 0.6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    import paper_2004_03493_gb300 as esim
    esim.build()
    n, rp, col = synth.chung_lu(20000, 200000, gamma=2.1, seed=3)
    return esim, (n, rp, col)


def _requests(rp, count, seed):
    rng = np.random.default_rng(seed)
    srcs = synth.random_sources(rp, count, seed=seed)
    eps = rng.choice([1e-2, 3e-3, 1e-3], size=count)
    return srcs, eps


def test_results_in_the_mix_equal_results_alone(env):
    esim, (n, rp, col) = env
    srcs, eps = _requests(rp, 40, seed=5)
    g = esim.Graph(n, rp, col)
    with esim.Server(g, C, k=20, seed=7, kappa=0.5, max_batch=16, max_waves=3) as srv:
        ids_mix = [srv.submit(u, e) for u, e in zip(srcs, eps)]
        mixed = [srv.wait(r, 120000) for r in ids_mix]
        st = srv.stats()
    assert st["completed"] == 40 and st["failed"] == 0
    assert st["waves"] >= 3
    with esim.Server(g, C, k=20, seed=7, kappa=0.5, max_batch=1, max_waves=1) as srv:
        for q in (0, 13, 39):
            r = srv.submit(srcs[q], eps[q])
            ids, vals, _ = srv.wait(r, 120000)
            assert np.array_equal(ids, mixed[q][0]) and np.array_equal(vals, mixed[q][1])
    # and equal to the batched call with B = 1
    ids1, vals1 = g.topk_batch([srcs[7]], [eps[7]], C, 20, seed=7)
    assert np.array_equal(ids1[0], mixed[7][0]) and np.array_equal(vals1[0], mixed[7][1])
    g.close()


def test_requests_arriving_while_others_run_are_served(env):
    esim, (n, rp, col) = env
    srcs, eps = _requests(rp, 60, seed=8)
    g = esim.Graph(n, rp, col)
    with esim.Server(g, C, k=10, seed=1, kappa=0.5, max_batch=8, max_waves=2) as srv:
        first = [srv.submit(u, e) for u, e in zip(srcs[:30], eps[:30])]
        time.sleep(0.005)
        second = [srv.submit(u, e) for u, e in zip(srcs[30:], eps[30:])]
        for r in first + second:
            ids, vals, lat = srv.wait(r, 120000)
            assert lat > 0 and ids.shape == (10,)
        st = srv.stats()
    assert st["completed"] == 60
    assert st["max_running"] >= 2
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    g.close()


def test_bounded_waits_and_host_side_failures(env):
    esim, (n, rp, col) = env
    g = esim.Graph(n, rp, col)
    srv = esim.Server(g, C, k=5, seed=2, kappa=50.0, max_batch=4, max_waves=1)
    with pytest.raises(esim.EsimError) as e:
        srv.submit(n, 1e-3)  # node out of range: rejected on the host
    assert e.value.status == -1
    with pytest.raises(esim.EsimError) as e:
        srv.submit(0, 1.5)
    assert e.value.status == -1
    rid = srv.submit(int(np.argmax(np.diff(rp))), 1e-4)  # a slow request (many walk pairs)
    with pytest.raises(esim.EsimError) as e:
        srv.wait(rid, 0)
    assert e.value.status == -4  # ESIM_ETIMEOUT; the request stays known
    assert srv.poll(rid) in (0, 1, 2)
    for u in range(6):  # leave queued work behind
        srv.submit(u, 1e-4)
    t0 = time.time()
    srv.close()  # cancels the queued requests, lets the running wave finish
    assert time.time() - t0 < 120
    g.close()
