"""GPU parity of Algorithm 3 (local deterministic exploitation) through the C ABI.

* Z_1..Z_d of a node (Lemma 5) against the oracle's term-by-term recursion, within
  1e-12 (FP64 sums in different orders).
* The depth-aware sampler (special tail pairs) bit for bit against the oracle's
  C walks, counts and pair steps.
* D^ of Algorithm 3 against the oracle, and the whole query against the CPU
  ExactSim with Algorithm 3 (integers exact, scores within 1e-12) and against the
  Power Method within eps.
"""
import numpy as np
import pytest

import synth
from oracle import alg3 as a3
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
    "er_2000": lambda: synth.erdos_renyi(2000, 20000, seed=1),
    "chung_lu_20k": lambda: synth.chung_lu(20000, 200000, gamma=2.1, seed=2),  # hubs: long-row sweeps
    "dangling_3001": lambda: synth.with_dangling(3001, 15000, seed=5),
}
# deepest Z checked per graph (the oracle's term-by-term Lemma 5 grows with the supports)
MAX_DEPTH = {"er_2000": 6, "chung_lu_20k": 4, "dangling_3001": 6}


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request, esim):
    n, rp, col = GRAPHS[request.param]()
    g = esim.Graph(n, rp, col)
    yield request.param, (n, rp, col), g
    g.close()


def _dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def test_first_meeting_matches_lemma5(graph):
    name, (n, rp, col), g = graph
    din = np.diff(rp)
    rng = np.random.default_rng(3)
    cand = np.nonzero(din >= 2)[0]
    picks = list(rng.choice(cand, size=3, replace=False)) + [int(np.argmax(din))]
    D = MAX_DEPTH[name]
    for k in picks:
        k = int(k)
        ref = a3.first_meeting_lemma5(n, rp, col, k, C, D)
        for d in range(1, D + 1):
            z = g.alg3_first_meeting(k, d, C)
            assert z.shape == (d,)
            assert np.max(np.abs(z - np.array(ref[:d]))) <= TOL, (name, k, d, z, ref)
    # din = 1 and din = 0 nodes: Z_1 = c (one in-neighbour) and Z = 0
    for k in np.nonzero(din <= 1)[0][:3]:
        z = g.alg3_first_meeting(int(k), 3, C)
        ref = a3.first_meeting_lemma5(n, rp, col, int(k), C, 3)
        assert np.max(np.abs(z - np.array(ref))) <= TOL


def test_depth_sampler_bit_exact(torch_cuda, graph, oracle_walks):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    rng = np.random.default_rng(21)
    R = rng.integers(0, 300, size=n).astype(np.uint64)
    R[rng.random(n) < 0.3] = 0
    depth = rng.integers(0, 9, size=n).astype(np.uint8)
    hub = int(np.argmax(np.diff(rp)))
    R[hub] = 60_000
    depth[hub] = 6
    off = np.concatenate([[0], np.cumsum(R, dtype=np.uint64)]).astype(np.uint64)
    for seed in (0, 99, 2 ** 64 - 5):
        ref, steps_ref = oracle_walks.walk_pairs_depth(n, rp, col, R, depth, C, seed)
        counts = torch.zeros(n, dtype=torch.uint64, device="cuda")
        steps = torch.zeros(1, dtype=torch.uint64, device="cuda")
        g.sample_depth(_dev(torch, off), _dev(torch, depth), C, seed, counts, steps)
        g.sync()
        assert np.array_equal(counts.cpu().numpy(), ref), name
        assert int(steps.cpu().numpy()[0]) == steps_ref
    # depth NULL is the Algorithm 2 sampler
    ref, _ = oracle_walks.walk_pairs(n, rp, col, R, C, 5)
    counts = torch.zeros(n, dtype=torch.uint64, device="cuda")
    g.sample_depth(_dev(torch, off), None, C, 5, counts)
    g.sync()
    assert np.array_equal(counts.cpu().numpy(), ref)


def test_dhat_alg3(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    din = np.diff(rp)
    rng = np.random.default_rng(8)
    R = rng.integers(0, 1000, size=n).astype(np.uint64)
    counts = (R * rng.random(n)).astype(np.uint64)
    depth = rng.integers(0, 4, size=n).astype(np.uint8)
    depth[R == 0] = 0
    zsum = np.where(depth > 0, rng.random(n) * 0.3, 0.0)
    off = np.concatenate([[0], np.cumsum(R, dtype=np.uint64)]).astype(np.uint64)
    ref = a3.dhat_alg3(counts, R, depth, zsum, din, C)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    g.dhat_alg3(_dev(torch, counts), _dev(torch, off), _dev(torch, depth), _dev(torch, zsum), C, out)
    g.sync()
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL, name
    assert np.all(got[din == 0] == 1.0) and np.all(got[din == 1] == 1.0 - C)


def _clean(pi, R_b, plan_depth, K):
    """The integer decisions are stable under the ~1e-15 relative gap between the
    GPU's and the oracle's pi: no ceil() argument within rounding of an integer,
    and no near-tie in pi at the edge of the K heaviest nodes."""
    v = R_b * (pi * pi)
    for vv in (v, v * C ** (2.0 * plan_depth)):
        frac = np.abs(vv - np.round(vv))
        if not np.all((frac > 1e-12 * vv) | (vv == 0)):
            return False
    srt = np.sort(pi)[::-1]
    if K < len(srt) and srt[K] > 0 and (srt[K - 1] - srt[K]) <= 1e-12 * srt[K - 1]:
        return False
    return True


@pytest.mark.parametrize("graph_name,kappa,min_pairs,max_nodes", [
    ("cl3000", None, 1e3, 16),
    ("er2000", 2000.0, 1e2, 8),
    ("dang2000", None, 1e3, 24),
])
def test_alg3_query_matches_cpu_exactsim(esim, oracle_walks, graph_name, kappa, min_pairs, max_nodes):
    from oracle import exactsim
    n, rp, col = {
        "cl3000": lambda: synth.chung_lu(3000, 30000, gamma=2.1, seed=9),
        "er2000": lambda: synth.erdos_renyi(2000, 16000, seed=4),
        "dang2000": lambda: synth.with_dangling(2000, 12000, seed=6),
    }[graph_name]()
    g = esim.Graph(n, rp, col) if kappa is None else esim.Graph(n, rp, col, kappa=kappa)
    g.set_option("alg3", 1)
    g.set_option("alg3_min_pairs", min_pairs)
    g.set_option("alg3_max_nodes", max_nodes)
    g.set_option("alg3_max_depth", 6)
    eps = 3e-3
    checked = 0
    deepest = 0
    for u, seed in ((5, 1), (1234, 2), (n - 1, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=kappa, alg3=True, alg3_max_depth=6,
                           alg3_min_pairs=min_pairs, alg3_max_nodes=max_nodes)
        deepest = max(deepest, int(q.depth.max()))
        if not _clean(q.pi, q.R_b, q.depth.astype(np.float64), max_nodes) or q.plan_gap <= 1e-9:
            continue  # an integer or depth decision sits within rounding of its boundary
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["alg3_nodes"] == int(np.count_nonzero(q.depth))
        assert st["sum_R"] == int(q.R.sum())
        assert st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    assert deepest >= 3  # probes (Lemma 5's l' >= 2 terms) were exercised
    g.close()


def test_alg3_within_eps_and_fewer_pairs(esim):
    from oracle import power
    n, rp, col = synth.chung_lu(2000, 20000, gamma=2.1, seed=11)
    S = power.power_method(n, rp, col, C)
    eps = 1e-3
    g = esim.Graph(n, rp, col)
    u = int(np.argmax(np.diff(rp)))
    s2 = g.query(u, C, eps, 0)
    base = g.stats()
    g.set_option("alg3", 1)
    g.set_option("alg3_min_pairs", 1e4)
    s3 = g.query(u, C, eps, 0)
    st = g.stats()
    assert st["alg3_nodes"] > 0
    assert st["sum_R"] < base["sum_R"]
    assert st["pair_steps"] < base["pair_steps"]
    assert np.max(np.abs(s3 - S[:, u])) <= eps
    assert np.max(np.abs(s2 - S[:, u])) <= eps
    # the top-k path carries the same scores
    ids, vals = g.topk(u, C, eps, 20, 0)
    ids_ref, vals_ref = lin.topk(s3, 20, exclude=u)
    assert np.array_equal(ids, ids_ref) and np.array_equal(vals, vals_ref)
    # FP32c precision with Algorithm 3 stays within eps too
    g.set_option("precision", 1)
    s32 = g.query(u, C, eps, 0)
    assert np.max(np.abs(s32 - S[:, u])) <= eps
    g.close()


def test_alg3_rejects_repeated_in_edges(esim):
    # node 2 has in-neighbour 0 twice
    rp = np.array([0, 1, 2, 5], dtype=np.int64)
    col = np.array([1, 2, 0, 0, 1], dtype=np.int32)
    g = esim.Graph(3, rp, col)
    with pytest.raises(esim.EsimError) as e:
        g.set_option("alg3", 1)
    assert e.value.status == -6
    with pytest.raises(esim.EsimError) as e:
        g.alg3_first_meeting(2, 2, C)
    assert e.value.status == -6
    g.close()


def test_alg3_with_basic_allocation_and_fp32c(esim, oracle_walks):
    from oracle import exactsim
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, alloc=1, alg3=1, alg3_min_pairs=1e3, alg3_max_nodes=16, alg3_max_depth=6)
    eps = 2e-2
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, mode="basic", alg3=True, alg3_max_depth=6,
                           alg3_min_pairs=1e3, alg3_max_nodes=16)
        v = q.R_b * q.pi
        vv = np.concatenate([v, v * C ** (2.0 * q.depth)])
        frac = np.abs(vv - np.round(vv))
        if not np.all((frac > 1e-12 * vv) | (vv == 0)) or q.plan_gap <= 1e-9:
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["alg3_nodes"] == int(np.count_nonzero(q.depth)) > 0
        assert st["sum_R"] == int(q.R.sum()) and st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    # FP32c precision with Algorithm 3: same pairs and D^ decisions as FP64 up to FP32 pi,
    # scores within the precision form's bound of FP64
    g.set_option("alloc", 0)
    s64 = g.query(5, C, 1e-3, 4)
    g.set_option("precision", 1)
    s32 = g.query(5, C, 1e-3, 4)
    assert np.max(np.abs(s32 - s64)) < 1e-4
    g.close()


# (2, 1.5e6) splits the exploited nodes of each source between the early and the main stream
@pytest.mark.parametrize("overlap,early", [(0, 1e30), (4, 1e30), (4, 1.0), (2, 1.5e6)])
def test_alg3_walk_overlap_gives_the_same_counts(esim, oracle_walks, overlap, early):
    """The walks split over the side stream (non-candidates), the early stream (each
    planned candidate) and the main stream give the oracle's counts and scores."""
    from oracle import exactsim
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, alg3=1, alg3_min_pairs=1e3, alg3_max_nodes=16, alg3_max_depth=6,
                   alg3_overlap=overlap, alg3_early_pairs=early)
    eps = 3e-3
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, alg3=True, alg3_max_depth=6, alg3_min_pairs=1e3,
                           alg3_max_nodes=16)
        if not _clean(q.pi, q.R_b, q.depth.astype(np.float64), 16) or q.plan_gap <= 1e-9:
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["sum_R"] == int(q.R.sum()) and st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        if overlap and early <= 1.0:
            assert st["early_launches"] == st["alg3_nodes"] > 0
        if overlap and early == 1.5e6:  # exploited R(k) of these sources lie on both sides of 1.5e6
            n_early = int(np.count_nonzero(q.R[q.depth > 0] >= early))
            assert 0 < st["early_launches"] == n_early < st["alg3_nodes"]
        checked += 1
    assert checked >= 2
    g.close()
