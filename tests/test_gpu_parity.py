"""GPU parity: every step of the CUDA path, through the C ABI, against the oracle.

Tolerances: integer and index work (R(k), offsets, walk counts, top-k ids) must
match bit for bit.  Floating-point sweeps must agree within 1e-12 absolute
(vectors are bounded by 1; the two sides differ only in summation order, about
L * 2^-52 relative).  Where an FP64 value decides an integer (R(k) = ceil(...)),
both sides take the decision in FP64 from the same inputs.
"""
import math

import numpy as np
import pytest

import synth
from oracle import linearization as lin

pytestmark = pytest.mark.gpu

C = 0.6
TOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    return torch


@pytest.fixture(scope="module")
def esim(torch_cuda):
    import paper_2004_03493_gb300 as pkg
    pkg.build()
    return pkg


GRAPHS = {
    "er_2000": lambda: synth.erdos_renyi(2000, 20000, seed=1),          # the small FP64 workload
    "chung_lu_20k": lambda: synth.chung_lu(20000, 200000, gamma=2.1, seed=2),  # hub rows -> long-row path
    "dangling_3001": lambda: synth.with_dangling(3001, 15000, seed=5),  # din = 0 nodes, ragged tail
    "cycle_97": lambda: synth.directed_cycle(97),
}


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request, esim):
    n, rp, col = GRAPHS[request.param]()
    g = esim.Graph(n, rp, col)
    yield request.param, (n, rp, col), g
    g.close()


def _dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _u64(torch, n):
    return torch.zeros(n, dtype=torch.uint64, device="cuda")


def test_forward_sweeps(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    for u, L in ((0, 20), (n - 1, 7), (n // 2, 0)):
        H = lin.hop_vectors(n, rp, col, u, C, L)
        hist = torch.full(((L + 1) * n,), float("nan"), dtype=torch.float64, device="cuda")
        g.forward(u, C, L, hist)
        g.sync()
        got = hist.view(L + 1, n).cpu().numpy()
        assert np.max(np.abs(got - H)) <= TOL, name


def test_allocate_bit_exact(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 20
    H = lin.hop_vectors(n, rp, col, 3 % n, C, L)
    pi_ref = lin.ppr(H)
    hist = _dev(torch, H.reshape(-1))
    for mode, mname in ((0, "pi2"), (1, "basic")):
        R_b = lin.sample_base(n, C, 1e-3) if mode == 0 else lin.sample_base(n, C, 1e-2)
        pi = torch.empty(n, dtype=torch.float64, device="cuda")
        R = _u64(torch, n)
        off = _u64(torch, n + 1)
        g.allocate(hist, L, R_b, mode, pi, R, off)
        g.sync()
        assert np.array_equal(pi.cpu().numpy(), pi_ref), name
        R_ref = lin.allocate(pi_ref, R_b, mname)
        assert np.array_equal(R.cpu().numpy(), R_ref), name
        off_ref = np.concatenate([[0], np.cumsum(R_ref, dtype=np.uint64)]).astype(np.uint64)
        assert np.array_equal(off.cpu().numpy(), off_ref), name


def test_sampler_counts_bit_exact(torch_cuda, graph, oracle_walks):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    rng = np.random.default_rng(17)
    R = rng.integers(0, 400, size=n).astype(np.uint64)
    R[rng.random(n) < 0.3] = 0
    R[0] = 50_000  # one heavy node spanning many threads
    off = np.concatenate([[0], np.cumsum(R, dtype=np.uint64)]).astype(np.uint64)
    for seed in (0, 12345, 2 ** 63 + 7):
        ref, steps_ref = oracle_walks.walk_pairs(n, rp, col, R, C, seed)
        nonmeet = _u64(torch, n)
        steps = _u64(torch, 1)
        g.sample(_dev(torch, off), C, seed, nonmeet, steps)
        g.sync()
        assert np.array_equal(nonmeet.cpu().numpy(), ref), name
        assert int(steps.cpu().numpy()[0]) == steps_ref


def test_dhat_and_reverse(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 20
    H = lin.hop_vectors(n, rp, col, 1 % n, C, L)
    D = synth.uniform_diagonal(n, C, seed=3)
    s_ref = lin.reverse(n, rp, col, H, D, C)
    s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g.reverse(_dev(torch, H.reshape(-1)), L, C, _dev(torch, D), s)
    g.sync()
    assert np.max(np.abs(s.cpu().numpy() - s_ref)) <= TOL, name
    # L = 0: s = D pi^0 / a
    s0 = torch.empty(n, dtype=torch.float64, device="cuda")
    g.reverse(_dev(torch, H[:1].reshape(-1)), 0, C, _dev(torch, D), s0)
    g.sync()
    assert np.max(np.abs(s0.cpu().numpy() - lin.reverse(n, rp, col, H[:1], D, C))) <= TOL
    # D^ from counts
    rng = np.random.default_rng(4)
    R = rng.integers(0, 1000, size=n).astype(np.uint64)
    nm = (R * rng.random(n)).astype(np.uint64)
    off = np.concatenate([[0], np.cumsum(R, dtype=np.uint64)]).astype(np.uint64)
    dh = torch.empty(n, dtype=torch.float64, device="cuda")
    g.dhat(_dev(torch, nm), _dev(torch, off), dh)
    g.sync()
    assert np.array_equal(dh.cpu().numpy(), lin.dhat(nm, R))


@pytest.mark.parametrize("k", [1, 50, 100, 999, 4096])
def test_select_topk_exact(torch_cuda, graph, k):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    rng = np.random.default_rng(k)
    scores = np.round(rng.random(n) * 50) / 50.0  # many ties
    scores[rng.random(n) < 0.2] = 0.0
    for exclude in (-1, 0, n - 1):
        ids_ref, vals_ref = lin.topk(scores, k, exclude if exclude >= 0 else None)
        ids = torch.empty(k, dtype=torch.int32, device="cuda")
        vals = torch.empty(k, dtype=torch.float64, device="cuda")
        g.select_topk(_dev(torch, scores), exclude, k, ids, vals)
        g.sync()
        m = len(ids_ref)
        got_ids = ids.cpu().numpy()
        assert np.array_equal(got_ids[:m], ids_ref), name
        assert np.array_equal(vals.cpu().numpy()[:m], vals_ref)
        assert np.all(got_ids[m:] == -1)


def _decisions_clean(pi, R_b):
    # the GPU's pi differs from the oracle's by summation order (relative ~1e-15);
    # ceil(R_b pi^2) can only differ where R_b pi^2 lies that close to an integer
    v = R_b * (pi * pi)
    frac = np.abs(v - np.round(v))
    return bool(np.all((frac > 1e-12 * v) | (v == 0)))


def test_full_query_matches_cpu_exactsim(torch_cuda, esim, oracle_walks):
    from oracle import exactsim
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col)
    eps = 3e-3
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed)
        if not _decisions_clean(q.pi, q.R_b):
            continue  # an R(k) sits within rounding of an integer; the two sides may round it apart
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["L"] == q.L and st["sum_R"] == int(q.R.sum())
        assert st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    g.close()


def test_query_within_eps_of_power_method(torch_cuda, esim):
    """The small FP64 workload: ER n=2000, m=20000, c=0.6, eps=1e-4, u=0, paper's R."""
    from oracle import power
    n, rp, col = synth.erdos_renyi(2000, 20000, seed=1)
    S = power.power_method(n, rp, col, C)
    g = esim.Graph(n, rp, col)
    eps = 1e-4
    s = g.query(0, C, eps, seed=0)
    err = np.max(np.abs(s - S[:, 0]))
    assert err <= eps, err
    st = g.stats()
    assert st["L"] == 20
    g.close()


def test_topk_query_matches_full_query(torch_cuda, esim):
    n, rp, col = synth.chung_lu(5000, 50000, gamma=2.1, seed=3)
    g = esim.Graph(n, rp, col, kappa=4.0)
    u, eps, seed = 17, 1e-4, 5
    s = g.query(u, C, eps, seed)
    for k in (1, 50, 500):
        ids, vals = g.topk(u, C, eps, k, seed)
        ids_ref, vals_ref = lin.topk(s, k, exclude=u)
        assert np.array_equal(ids, ids_ref) and np.array_equal(vals, vals_ref)
    g.set_option("exclude_source", 0)
    ids, _ = g.topk(u, C, eps, 1, seed)
    assert ids[0] == u  # s(u, u) is the largest score
    g.close()


def test_query_is_deterministic_and_stream_aware(torch_cuda, esim):
    torch = torch_cuda
    n, rp, col = synth.chung_lu(4000, 40000, gamma=2.1, seed=4)
    g = esim.Graph(n, rp, col, kappa=2.0)
    a = g.query(7, C, 1e-4, 3)
    stream = torch.cuda.Stream()
    g.set_stream(stream)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    g.query_device(7, C, 1e-4, 3, out)
    assert np.array_equal(out.cpu().numpy(), a)
    g.set_stream(None)
    b = g.query(7, C, 1e-4, 3)
    assert np.array_equal(a, b)
    c = g.query(7, C, 1e-4, 4)
    assert not np.array_equal(a, c)
    g.close()


def test_edge_cases(torch_cuda, esim):
    # single node without edges: D^ = 1, s = pi^0 / a = 1
    g = esim.Graph(1, np.array([0, 0]), np.zeros(0, dtype=np.int32))
    s = g.query(0, C, 1e-2, 0)
    assert s.tolist() == [1.0]
    ids, vals = g.topk(0, C, 1e-2, 3, 0)
    assert ids.tolist() == [-1, -1, -1]
    g.set_option("exclude_source", 0)
    ids, vals = g.topk(0, C, 1e-2, 3, 0)
    assert ids.tolist() == [0, -1, -1] and vals[0] == 1.0
    g.close()
    # dangling source: its walks stop at once, so s = e_u exactly
    n, rp, col = synth.with_dangling(500, 3000, seed=2)
    g = esim.Graph(n, rp, col)
    u = int(np.nonzero(np.diff(rp) == 0)[0][0])
    s = g.query(u, C, 1e-3, 0)
    expect = np.zeros(n)
    expect[u] = 1.0
    assert np.array_equal(s, expect)
    # invalid arguments
    with pytest.raises(esim.EsimError) as e:
        g.query(n, C, 1e-3, 0)
    assert e.value.status == -1
    with pytest.raises(esim.EsimError) as e:
        g.query(0, 1.0, 1e-3, 0)
    assert e.value.status == -1
    with pytest.raises(esim.EsimError) as e:
        g.topk(0, C, 1e-3, 4097, 0)
    assert e.value.status == -6
    with pytest.raises(esim.EsimError):
        g.set_option("no_such_option", 1)
    # pair budget: refused before any walk, reported as ESIM_EBUDGET
    g.set_option("pair_budget", 10)
    with pytest.raises(esim.EsimError) as e:
        g.query(int(np.argmax(np.diff(rp))), C, 1e-4, 0)
    assert e.value.status == -5
    g.set_option("pair_budget", 1e15)
    s = g.query(u, C, 1e-3, 0)  # the handle stays usable
    assert s[u] == 1.0
    g.close()


def test_basic_allocation_mode(torch_cuda, esim, oracle_walks):
    from oracle import exactsim
    n, rp, col = synth.erdos_renyi(800, 6000, seed=8)
    g = esim.Graph(n, rp, col, alloc=1)
    q = exactsim.query(n, rp, col, 3, C, 1e-2, seed=2, mode="basic")
    s = g.query(3, C, 1e-2, 2)
    assert g.stats()["sum_R"] == int(q.R.sum())
    assert np.max(np.abs(s - q.s)) <= TOL
    g.close()
