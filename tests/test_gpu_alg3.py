"""GPU parity of Algorithm 3 (local deterministic exploitation) through the C ABI.

* Z_1..Z_d of a node (Lemma 5) against the oracle's term-by-term recursion, within
  1e-12 (FP64 sums in different orders).
* The depth-aware sampler (special tail pairs) bit for bit against the oracle's
  C walks, counts and pair steps.
* The paper's adaptive depth (explored edges reach 2 R(k)/sqrt(c)) node for node
  against the oracle's counter.
* D^ of Algorithm 3 against the oracle, and the whole query against the CPU
  ExactSim with Algorithm 3 under the paper's rule (integers exact, scores within
  1e-12) and against the Power Method within eps.
* The library's cost-model rule (a speed choice, option alg3_rule = 1): the whole
  query against the oracle run on the plan that the tests' restatement of the
  documented cost model picks, with the walks split over streams or not.
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


def test_first_meeting_covers_both_last_level_forms(graph):
    """The last probe level takes g_2 of each support node from a one-warp two-hop table
    when the node's two-hop multiset fits (sum of din over its in-neighbours <= 512), from
    a one-block table when it is at most 8192, else from the dense probes; at the hub of
    the Chung-Lu graph, depth 3, all three forms occur among the support of h_1 = I(k),
    and Z still matches the oracle's Lemma 5."""
    name, (n, rp, col), g = graph
    if name != "chung_lu_20k":
        pytest.skip("the hub graph covers both forms")
    din = np.diff(rp)
    k = int(np.argmax(din))
    sup = col[rp[k]:rp[k + 1]]
    e1 = np.array([int(din[col[rp[q]:rp[q + 1]]].sum()) for q in sup])
    assert np.count_nonzero(e1 <= 512) > 0 and np.count_nonzero((e1 > 512) & (e1 <= 8192)) > 0
    assert np.count_nonzero(e1 > 8192) > 0
    for d in (3, 4):
        ref = a3.first_meeting_lemma5(n, rp, col, k, C, d)
        z = g.alg3_first_meeting(k, d, C)
        assert np.max(np.abs(z - np.array(ref))) <= TOL, (d, z, ref)


def test_first_meeting_hashed_levels_on_a_hub(esim):
    """The last two probe levels run one warp per node where the neighbourhood fits its
    tables (two-hop multiset <= 512; for the level below the last also three-hop
    multiset <= 1024), one block per node where it fits the block's (<= 8192; <= 2048 and
    <= 4096), dense probes for the others.  At the hub of a Chung-Lu graph all three forms
    occur at the level below the last; Z_1..Z_d at depths 3..6 match the oracle's Lemma 5."""
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    din = np.diff(rp).astype(np.int64)
    k = int(np.argmax(din))

    def multisets(q):
        s1 = col[rp[q]:rp[q + 1]]
        s2 = np.unique(np.concatenate([col[rp[a]:rp[a + 1]] for a in s1])) if len(s1) else s1
        return int(din[s1].sum()), int(din[s2].sum())

    sizes = np.array([multisets(int(q)) for q in col[rp[k]:rp[k + 1]]])  # the support of h_1
    warp = (sizes[:, 0] <= 512) & (sizes[:, 1] <= 1024)
    block = ~warp & (sizes[:, 0] <= 2048) & (sizes[:, 1] <= 4096)
    assert np.count_nonzero(warp) > 0 and np.count_nonzero(block) > 0 and np.count_nonzero(~warp & ~block) > 0
    g = esim.Graph(n, rp, col)
    ref = a3.first_meeting_lemma5(n, rp, col, k, C, 6)
    for d in (3, 4, 5, 6):
        z = g.alg3_first_meeting(k, d, C)
        assert np.max(np.abs(z - np.array(ref[:d]))) <= TOL, (d, z, ref)
    g.close()


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


def _clean_R(pi, R_b, mode="pi2", scale=None):
    """No ceil() argument of the allocation lies within rounding of an integer: the GPU's
    pi differs from the oracle's by summation order (~1e-15 relative)."""
    v = R_b * (pi * pi) if mode == "pi2" else R_b * pi
    vs = [v] if scale is None else [v, v * scale]
    for vv in vs:
        frac = np.abs(vv - np.round(vv))
        if not np.all((frac > 1e-12 * vv) | (vv == 0)):
            return False
    return True


PAPER_GRAPHS = {
    "er2000": lambda: synth.erdos_renyi(2000, 16000, seed=4),
    "cl3000": lambda: synth.chung_lu(3000, 30000, gamma=2.1, seed=9),
    "dang2000": lambda: synth.with_dangling(2000, 12000, seed=6),
}


@pytest.mark.parametrize("graph_name", list(PAPER_GRAPHS))
def test_paper_depth_rule_step_bit_exact(torch_cuda, esim, graph_name):
    """esim_alg3_paper_depth against the oracle's counter and rule, node for node, for
    sample counts from 1 to 1e12 and several depth caps."""
    torch = torch_cuda
    n, rp, col = PAPER_GRAPHS[graph_name]()
    din = np.diff(rp)
    g = esim.Graph(n, rp, col)
    E = a3.explored_edges(n, rp, col, 16)
    rng = np.random.default_rng(17)
    for max_depth in (16, 5, 0):
        R = np.floor(10.0 ** rng.uniform(0, 12, size=n)).astype(np.uint64)
        R[rng.random(n) < 0.2] = 0
        R[din <= 1] = 0
        want = np.zeros(n, dtype=np.uint8)
        for k in np.nonzero(R)[0]:
            want[k] = a3.paper_depth(E[:, k], int(R[k]), C, max_depth)
        depth = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        g.alg3_paper_depth(_dev(torch, R), C, max_depth, depth)
        g.sync()
        got = depth.cpu().numpy()
        assert np.array_equal(got, want), (graph_name, max_depth, np.nonzero(got != want)[0][:10])
        if max_depth == 16:
            assert want.max() >= 5 and len(np.unique(want)) >= 5
    g.close()


@pytest.mark.parametrize("graph_name", list(PAPER_GRAPHS))
def test_zsum_step_matches_lemma5_sums(torch_cuda, esim, graph_name):
    """esim_alg3_zsum (depth 1 and 2 in closed form, deeper nodes by the Lemma 5 kernels)
    against the oracle's Lemma 5 sums, node for node, on random depth vectors 0..4 that
    include nodes with din 0 and 1."""
    torch = torch_cuda
    n, rp, col = PAPER_GRAPHS[graph_name]()
    din = np.diff(rp)
    g = esim.Graph(n, rp, col)
    rng = np.random.default_rng(41)
    depth = np.zeros(n, dtype=np.uint8)
    picks = rng.choice(n, size=400, replace=False)
    depth[picks] = rng.integers(1, 5, size=picks.size).astype(np.uint8)
    depth[picks[:40]] = 2  # many depth-2 nodes: the closed form's table
    want = a3.first_meeting_sums(n, rp, col, depth, C)
    zsum = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g.alg3_zsum(_dev(torch, depth), C, zsum)
    got = zsum.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - want)) <= TOL, (graph_name, np.argmax(np.abs(got - want)))
    assert np.all(got[depth == 0] == 0.0)
    assert np.any((depth == 2) & (din >= 2)) and np.any((depth >= 1) & (din <= 1))
    g.close()


def test_zsum_and_query_do_not_depend_on_the_workers(torch_cuda, esim):
    """The deep nodes' Lemma 5 computations run on 1..alg3_workers streams at once; each
    node's result is computed alone, so the zsum step and whole cost-model queries are
    bit-identical for 1, 3 and 6 workers."""
    torch = torch_cuda
    n, rp, col = PAPER_GRAPHS["cl3000"]()
    rng = np.random.default_rng(43)
    depth = np.zeros(n, dtype=np.uint8)
    picks = rng.choice(n, size=60, replace=False)
    depth[picks] = rng.integers(3, 7, size=picks.size).astype(np.uint8)
    # light weights on the exact part: source 5 at eps 1e-3 exploits three nodes at depths 3, 4, 6
    g = esim.Graph(n, rp, col, alg3=1, alg3_rule=1, alg3_min_pairs=1e3, alg3_max_nodes=32, alg3_max_depth=6,
                   alg3_w_sweep=0.1, alg3_w_probe=0.01, alg3_w_launch=0.0)
    zs, qs = [], []
    for workers in (1, 3, 6):
        g.set_option("alg3_workers", workers)
        zsum = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        g.alg3_zsum(_dev(torch, depth), C, zsum)
        zs.append(zsum.cpu().numpy())
        qs.append(g.query(5, C, 1e-3, 7))
        assert g.stats()["alg3_nodes"] >= 3
    for z, q in zip(zs[1:], qs[1:]):
        assert np.array_equal(z, zs[0]) and np.array_equal(q, qs[0])
    g.close()


@pytest.mark.parametrize("graph_name,kappa,eps", [
    ("er2000", 2000.0, 3e-3),
    ("cl3000", None, 3e-3),
    ("dang2000", None, 3e-3),
    ("er2000", 4.0, 1e-4),
])
def test_alg3_paper_rule_query_matches_cpu_exactsim(esim, oracle_walks, graph_name, kappa, eps):
    """The whole query with the paper's adaptive depth (the library's default rule)
    against the oracle's Algorithm 3: depths, pair counts and pair steps exact, scores
    within 1e-12."""
    from oracle import exactsim
    n, rp, col = PAPER_GRAPHS[graph_name]()
    g = esim.Graph(n, rp, col) if kappa is None else esim.Graph(n, rp, col, kappa=kappa)
    g.set_option("alg3", 1)
    assert g.get_option("alg3_rule") == 0 and g.get_option("alg3_max_depth") == 16
    checked = 0
    deepest = 0
    for u, seed in ((5, 1), (1234, 2), (n - 1, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=kappa, alg3=True)
        deepest = max(deepest, int(q.depth.max()))
        if not _clean_R(q.pi, q.R_b):
            continue  # an integer decision sits within rounding of its boundary
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


def test_alg3_paper_rule_with_basic_allocation(esim, oracle_walks):
    from oracle import exactsim
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, alloc=1, alg3=1)
    eps = 2e-2
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, mode="basic", alg3=True)
        if not _clean_R(q.pi, q.R_b, "basic"):
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["alg3_nodes"] == int(np.count_nonzero(q.depth)) > 0
        assert st["sum_R"] == int(q.R.sum()) and st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    g.close()


def test_alg3_paper_rule_refuses_graphs_beyond_its_bit_sets(esim):
    # a 131,073-node cycle: the support bit sets would need 2 n ceil(n/32) words > 4 GiB
    n = 131_073
    rp = np.arange(n + 1, dtype=np.int64)
    col = ((np.arange(n) + 1) % n).astype(np.int32)
    g = esim.Graph(n, rp, col, alg3=1)
    with pytest.raises(esim.EsimError) as e:
        g.query(0, C, 1e-2, 0)
    assert e.value.status == -6 and "alg3_rule" in str(e.value)
    g.set_option("alg3_rule", 1)  # the cost model has no such limit
    s = g.query(0, C, 1e-2, 0)
    assert abs(s[0] - (1 - C) * (1 - C ** (esim.esim_levels(C, 1e-2) + 1)) / (1 - C)) < 1e-12
    # nor has the exact part for given depths: on a cycle (one in-neighbour each) the two
    # walks meet at step 1, so Z_1 = c and the deeper terms are 0
    import torch
    depth = np.zeros(n, dtype=np.uint8)
    depth[:6] = np.arange(1, 7)
    depth[n - 1] = 3
    zsum = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g.alg3_zsum(torch.from_numpy(depth).cuda(), C, zsum)
    z = zsum.cpu().numpy()
    assert np.max(np.abs(z[depth > 0] - C)) <= TOL and np.all(z[depth == 0] == 0.0)
    g.close()


def _cost_plan_query(n, rp, col, u, eps, seed, kappa=None, mode="pi2", **kw):
    """The oracle's query under the cost-model plan that tests/alg3_cost_plan.py restates."""
    import alg3_cost_plan as cp
    from oracle import exactsim
    L = lin.levels(C, eps)
    pi = lin.ppr(lin.hop_vectors(n, rp, col, u, C, L))
    R_b = lin.sample_base(n, C, eps, kappa)
    depth, R, gap = cp.plan(n, rp, col, pi, R_b, C, mode=mode, **kw)
    q = exactsim.query(n, rp, col, u, C, eps, seed=seed, kappa=kappa, mode=mode, alg3=True, alg3_plan=(depth, R))
    return q, gap


@pytest.mark.parametrize("graph_name,kappa,min_pairs,max_nodes", [
    ("cl3000", None, 1e3, 16),
    ("er2000", 2000.0, 1e2, 8),
    ("dang2000", None, 1e3, 24),
])
def test_alg3_cost_model_query_matches_oracle_on_its_plan(esim, oracle_walks, graph_name, kappa, min_pairs,
                                                          max_nodes):
    """Option alg3_rule = 1 (the cost model, a speed choice of the library): the oracle
    runs the plan that the tests' restatement of the documented cost model chooses, and
    the library's whole query matches it (integers exact, scores within 1e-12)."""
    n, rp, col = PAPER_GRAPHS[graph_name]()
    g = esim.Graph(n, rp, col) if kappa is None else esim.Graph(n, rp, col, kappa=kappa)
    for key, val in (("alg3", 1), ("alg3_rule", 1), ("alg3_min_pairs", min_pairs), ("alg3_max_nodes", max_nodes),
                     ("alg3_max_depth", 6)):
        g.set_option(key, val)
    eps = 3e-3
    checked = 0
    deepest = 0
    for u, seed in ((5, 1), (1234, 2), (n - 1, 3)):
        q, gap = _cost_plan_query(n, rp, col, u, eps, seed, kappa, max_depth=6, min_pairs=min_pairs,
                                  max_nodes=max_nodes)
        deepest = max(deepest, int(q.depth.max()))
        srt = np.sort(q.pi)[::-1]
        tie = max_nodes < n and srt[max_nodes] > 0 and srt[max_nodes - 1] - srt[max_nodes] <= 1e-12 * srt[max_nodes - 1]
        if not _clean_R(q.pi, q.R_b, scale=C ** (2.0 * q.depth)) or gap <= 1e-9 or tie:
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["alg3_nodes"] == int(np.count_nonzero(q.depth))
        assert st["sum_R"] == int(q.R.sum())
        assert st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        checked += 1
    assert checked >= 2
    assert deepest >= 3
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
    sp = g.query(u, C, eps, 0)  # the paper's depth rule keeps R(k) pairs
    stp = g.stats()
    assert stp["alg3_nodes"] > 0 and stp["sum_R"] <= base["sum_R"]
    assert np.max(np.abs(sp - S[:, u])) <= eps
    g.set_option("alg3_rule", 1)  # the cost model spends fewer pairs
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


def test_alg3_cost_model_with_basic_allocation_and_fp32c(esim, oracle_walks):
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, alloc=1, alg3=1, alg3_rule=1, alg3_min_pairs=1e3, alg3_max_nodes=16,
                   alg3_max_depth=6)
    eps = 2e-2
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q, gap = _cost_plan_query(n, rp, col, u, eps, seed, mode="basic", max_depth=6, min_pairs=1e3,
                                  max_nodes=16)
        if not _clean_R(q.pi, q.R_b, "basic", scale=C ** (2.0 * q.depth)) or gap <= 1e-9:
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
    """Cost model: the walks split between the side launch (non-candidates and the
    candidates with at least alg3_early_pairs pairs, started before the first-meeting
    terms) and the main stream give the oracle's counts and scores on the same plan."""
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    g = esim.Graph(n, rp, col, alg3=1, alg3_rule=1, alg3_min_pairs=1e3, alg3_max_nodes=16, alg3_max_depth=6,
                   alg3_overlap=overlap, alg3_early_pairs=early)
    eps = 3e-3
    checked = 0
    for u, seed in ((5, 1), (1234, 2), (2999, 3)):
        q, gap = _cost_plan_query(n, rp, col, u, eps, seed, max_depth=6, min_pairs=1e3, max_nodes=16)
        if not _clean_R(q.pi, q.R_b, scale=C ** (2.0 * q.depth)) or gap <= 1e-9:
            continue
        s = g.query(u, C, eps, seed)
        st = g.stats()
        assert st["sum_R"] == int(q.R.sum()) and st["pair_steps"] == q.pair_steps
        assert np.max(np.abs(s - q.s)) <= TOL
        if overlap:
            assert st["pair_steps_side"] > 0
        if overlap and early <= 1.0:  # every candidate, exploited or not
            assert st["side_candidates"] >= st["alg3_nodes"] > 0
        if overlap and early == 1.5e6:  # exploited R(k) of these sources lie on both sides of 1.5e6
            planned = q.R[q.depth > 0]
            assert st["side_candidates"] >= int(np.count_nonzero(planned >= early)) > 0
            assert np.count_nonzero(planned < early) > 0
        if not overlap or early > 1e20:
            assert st["side_candidates"] == 0
        checked += 1
    assert checked >= 2
    g.close()
