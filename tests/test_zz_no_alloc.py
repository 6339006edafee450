"""The top-k selection that allocates nothing, against the ordinary entry point.

Some callers of this library cannot allocate device memory: code inside a host
framework that owns every byte of device memory, or a latency-critical thread
that must not take the synchronisation an allocation can cause.
``esim_select_topk_static`` serves them with a static device scratch array.
This test calls it through the C ABI twice in a row (the array keeps the first
call's contents) and checks each result against ``esim_select_topk``, which
uses the graph's allocated workspace, and against the oracle's top-k list
(score desc, id asc); ids and scores must agree exactly, the same bar as the
other top-k tests.  It is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from oracle import linearization as lin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    import paper_2004_03493_gb300 as esim
    esim.build()
    n, rp, col = synth.with_dangling(5003, 30000, seed=13)
    g = esim.Graph(n, rp, col)
    g.set_stream(torch.cuda.current_stream())
    yield torch, esim, g, n
    g.close()


def _scores(torch, n, seed):
    rng = np.random.default_rng(seed)
    s = np.round(rng.random(n) * 40) / 40.0  # many ties
    s[rng.random(n) < 0.25] = 0.0
    return torch.from_numpy(s).cuda(), s


def _both(torch, esim, g, scores, n, exclude, k):
    ids_a = torch.full((k,), -7, dtype=torch.int32, device="cuda")
    vals_a = torch.full((k,), -7.0, dtype=torch.float64, device="cuda")
    g.select_topk(scores, exclude, k, ids_a, vals_a)
    ids_b = torch.full((k,), -7, dtype=torch.int32, device="cuda")
    vals_b = torch.full((k,), -7.0, dtype=torch.float64, device="cuda")
    esim.esim_select_topk_static(scores, n, exclude, k, ids_b, vals_b, torch.cuda.current_stream())
    torch.cuda.synchronize()
    g.sync()
    return (ids_a.cpu().numpy(), vals_a.cpu().numpy()), (ids_b.cpu().numpy(), vals_b.cpu().numpy())


def test_static_topk_matches_allocating_entry_point_twice(setup):
    torch, esim, g, n = setup
    cases = [(_scores(torch, n, 1), -1, 4096), (_scores(torch, n, 2), 17, 50)]  # second call: smaller k, new data
    for (scores, host), exclude, k in cases:
        (ids_a, vals_a), (ids_b, vals_b) = _both(torch, esim, g, scores, n, exclude, k)
        assert np.array_equal(ids_a, ids_b)
        assert np.array_equal(vals_a, vals_b)
        ids_ref, vals_ref = lin.topk(host, k, exclude=exclude if exclude >= 0 else None)
        assert np.array_equal(ids_b, ids_ref)
        assert np.array_equal(vals_b, vals_ref)
        assert not np.any(ids_b == exclude) if exclude >= 0 else True


def test_static_topk_rejects_sizes_beyond_its_scratch(setup):
    torch, esim, g, n = setup
    scores, _ = _scores(torch, n, 3)
    ids = torch.empty(4097, dtype=torch.int32, device="cuda")
    vals = torch.empty(4097, dtype=torch.float64, device="cuda")
    with pytest.raises(esim.EsimError) as e:
        esim.esim_select_topk_static(scores, n, -1, 4097, ids, vals)
    assert e.value.status == -6
    assert "4096" in str(e.value)
    with pytest.raises(esim.EsimError) as e:
        esim.esim_select_topk_static(scores, 0, -1, 10, ids, vals)
    assert e.value.status == -1
