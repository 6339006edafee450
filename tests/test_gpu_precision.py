"""GPU parity of the precision form (FP32c): FP32 storage with two-float sums.

Error model (derived from the arithmetic, u = 2^-24):
* forward: every stored pi^l and x^l is one rounding of a two-float quantity, and
  all terms are non-negative, so |pi~^l - pi^l| <= (2l + 2) u pi^l;
* reverse from a given FP32 history: two-float arithmetic (about 2^-44 per
  operation) keeps s^L within 1e-11 of FP64 arithmetic on the same inputs;
* whole sweep pair with the same D: by the bilinear form (Eq. formula-ppr),
  |s~ - s| <= u sum_l (2l + 2) c^l = u (2c/(1-c)^2 + 2/(1-c)), 7.45e-7 at c = 0.6.
"""
import math

import numpy as np
import pytest

import synth
from oracle import linearization as lin

pytestmark = pytest.mark.gpu

C = 0.6
U32 = 2.0 ** -24


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
    "chung_lu_20k": lambda: synth.chung_lu(20000, 200000, gamma=2.1, seed=2),
    "dangling_3001": lambda: synth.with_dangling(3001, 15000, seed=5),
}


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request, esim):
    n, rp, col = GRAPHS[request.param]()
    g = esim.Graph(n, rp, col)
    yield request.param, (n, rp, col), g
    g.close()


def _dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _sweep_bound(c):
    return U32 * (2 * c / (1 - c) ** 2 + 2 / (1 - c))


def test_forward_f32_error_bound(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 24
    for u in (0, n // 3):
        H = lin.hop_vectors(n, rp, col, u, C, L)
        hist = torch.full(((L + 1) * n,), float("nan"), dtype=torch.float32, device="cuda")
        g.forward_f32(u, C, L, hist)
        g.sync()
        got = hist.view(L + 1, n).cpu().numpy().astype(np.float64)
        for ell in range(L + 1):
            bound = (2 * ell + 2) * U32 * H[ell] + 1e-38
            assert np.all(np.abs(got[ell] - H[ell]) <= bound), (name, ell)


def test_allocate_f32_sums_levels(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 20
    H32 = lin.hop_vectors(n, rp, col, 1, C, L).astype(np.float32)
    pi_ref = lin.ppr(H32.astype(np.float64))  # FP64 sum of the same FP32 values
    R_b = lin.sample_base(n, C, 1e-3)
    pi = torch.empty(n, dtype=torch.float64, device="cuda")
    R = torch.zeros(n, dtype=torch.uint64, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.uint64, device="cuda")
    g.allocate_f32(_dev(torch, H32.reshape(-1)), L, R_b, 0, pi, R, off)
    g.sync()
    got = pi.cpu().numpy()
    assert np.all(np.abs(got - pi_ref) <= 1e-13 * pi_ref + 1e-300)
    v = R_b * (pi_ref * pi_ref)
    clean = np.abs(v - np.round(v)) > 1e-11 * v
    R_ref = lin.allocate(pi_ref, R_b, "pi2")
    assert np.array_equal(R.cpu().numpy()[clean], R_ref[clean])


def test_fp32c_pair_counts_stay_within_their_rounding_of_fp64(torch_cuda, graph):
    """The FP32c query draws R(k) from FP32 hop vectors: pi within (2L+2) u relative of the
    FP64 form's pi (the forward bound, summed over levels), so R(k) = ceil(R_b pi(k)^2) moves by
    at most 2 (2L+2) u R(k) + 1 pairs, and only where R_b pi(k)^2 lies that close to an
    integer.  Checked node by node on the same source, with the share of nodes whose count
    differs reported."""
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 24
    R_b = lin.sample_base(n, C, 1e-4, 4.0)
    out = {}
    for prec in ("fp64", "fp32c"):
        pi = torch.empty(n, dtype=torch.float64, device="cuda")
        R = torch.zeros(n, dtype=torch.uint64, device="cuda")
        off = torch.zeros(n + 1, dtype=torch.uint64, device="cuda")
        if prec == "fp64":
            hist = torch.empty((L + 1) * n, dtype=torch.float64, device="cuda")
            g.forward(3, C, L, hist)
            g.allocate(hist, L, R_b, 0, pi, R, off)
        else:
            hist = torch.empty((L + 1) * n, dtype=torch.float32, device="cuda")
            g.forward_f32(3, C, L, hist)
            g.allocate_f32(hist, L, R_b, 0, pi, R, off)
        g.sync()
        out[prec] = (pi.cpu().numpy(), R.cpu().numpy().astype(np.float64))
    (p64, R64), (p32, R32) = out["fp64"], out["fp32c"]
    delta = (2 * L + 2) * U32
    assert np.all(np.abs(p32 - p64) <= delta * p64 + 1e-300)
    assert np.all(np.abs(R32 - R64) <= np.ceil(2 * delta * R64) + 1)
    share = float(np.mean(R32 != R64))
    print(f"{name}: FP32c pair counts differ from FP64 on {share:.2%} of the nodes, "
          f"{abs(R32.sum() - R64.sum()) / R64.sum():.2e} of the pairs")
    assert abs(R32.sum() - R64.sum()) <= 2 * delta * R64.sum() + n


def test_reverse_f32_matches_fp64_on_same_inputs(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = 24
    H32 = lin.hop_vectors(n, rp, col, 2, C, L).astype(np.float32)
    D = synth.uniform_diagonal(n, C, seed=4)
    s_ref = lin.reverse(n, rp, col, H32.astype(np.float64), D, C)
    s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g.reverse_f32(_dev(torch, H32.reshape(-1)), L, C, _dev(torch, D), s)
    g.sync()
    assert np.max(np.abs(s.cpu().numpy() - s_ref)) <= 1e-11, name
    # L = 0 writes the FP64 result directly
    s0 = torch.empty(n, dtype=torch.float64, device="cuda")
    g.reverse_f32(_dev(torch, H32[:1].reshape(-1)), 0, C, _dev(torch, D), s0)
    g.sync()
    assert np.max(np.abs(s0.cpu().numpy() - lin.reverse(n, rp, col, H32[:1].astype(np.float64), D, C))) <= 1e-12


def test_fp32c_sweeps_within_derived_bound_of_fp64(torch_cuda, graph):
    torch = torch_cuda
    name, (n, rp, col), g = graph
    L = lin.levels(C, 1e-7)
    D = synth.uniform_diagonal(n, C, seed=6)
    u = 5 % n
    H = lin.hop_vectors(n, rp, col, u, C, L)
    s_ref = lin.reverse(n, rp, col, H, D, C)
    hist = torch.empty(((L + 1) * n,), dtype=torch.float32, device="cuda")
    g.forward_f32(u, C, L, hist)
    s = torch.empty(n, dtype=torch.float64, device="cuda")
    g.reverse_f32(hist, L, C, _dev(torch, D), s)
    g.sync()
    err = np.max(np.abs(s.cpu().numpy() - s_ref))
    assert err <= _sweep_bound(C) + 1e-12, (name, err)


def test_precision_query_equals_its_steps(torch_cuda, esim):
    torch = torch_cuda
    n, rp, col = synth.chung_lu(5000, 50000, gamma=2.1, seed=3)
    g = esim.Graph(n, rp, col, kappa=2.0, precision=1)
    u, eps, seed = 17, 1e-4, 9
    s_query = g.query(u, C, eps, seed)
    L = lin.levels(C, eps)
    hist = torch.empty(((L + 1) * n,), dtype=torch.float32, device="cuda")
    pi = torch.empty(n, dtype=torch.float64, device="cuda")
    R = torch.zeros(n, dtype=torch.uint64, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.uint64, device="cuda")
    nm = torch.zeros(n, dtype=torch.uint64, device="cuda")
    dh = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty(n, dtype=torch.float64, device="cuda")
    g.forward_f32(u, C, L, hist)
    g.allocate_f32(hist, L, esim.esim_sample_base(n, C, eps, 2.0), 0, pi, R, off)
    g.sample(off, C, seed, nm)
    g.dhat(nm, off, dh)
    g.reverse_f32(hist, L, C, dh, s)
    g.sync()
    assert np.array_equal(s.cpu().numpy(), s_query)
    g.close()


def test_precision_query_within_eps_of_power_method(torch_cuda, esim):
    from oracle import power
    n, rp, col = synth.erdos_renyi(2000, 20000, seed=1)
    S = power.power_method(n, rp, col, C)
    g = esim.Graph(n, rp, col, precision=1)
    s = g.query(0, C, 1e-4, seed=0)
    assert np.max(np.abs(s - S[:, 0])) <= 1e-4
    ids, _ = g.topk(0, C, 1e-4, 10, seed=0)
    assert np.array_equal(ids, lin.topk(s, 10, exclude=0)[0])
    g.close()
