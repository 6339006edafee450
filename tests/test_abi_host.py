"""The C ABI library loads and exports every entry point of include/exactsim.h.

Runs without a GPU: only host-side entry points (parameters, validation) are
called.  Calls that need a device are made in the ``gpu`` tests.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import synth
from oracle import linearization as lin

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2004_03493_gb300 import buildlib as build_mod
    build_mod.build()
    from paper_2004_03493_gb300 import _native
    return _native


def _declared_functions():
    with open(os.path.join(ROOT, "include", "exactsim.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(esim_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(native):
    names = _declared_functions()
    assert len(names) >= 20
    h = ctypes.CDLL(native.LIB_PATH)
    for name in names:
        assert hasattr(h, name), name
        assert name in native.SIGNATURES, name
    assert set(native.SIGNATURES) == set(names)


def test_version(native):
    assert "sm_103a" in native.esim_version()


@pytest.mark.parametrize("c,eps", [(0.6, 1e-4), (0.6, 1e-5), (0.6, 1e-6), (0.6, 1e-7), (0.8, 1e-3), (0.25, 0.5)])
def test_levels_and_sample_base_match_oracle(native, c, eps):
    assert native.esim_levels(c, eps) == lin.levels(c, eps)
    for n in (2, 2000, 33554432):
        assert native.esim_sample_base(n, c, eps, 0.0) == lin.sample_base(n, c, eps)
        assert native.esim_sample_base(n, c, eps, 3.5) == lin.sample_base(n, c, eps, 3.5)


def test_walk_threshold_matches_oracle(native):
    for c in (0.6, 0.8, 0.25, 1e-9, 0.999999):
        assert native.esim_walk_threshold(c) == lin.pair_threshold(c)


def test_parameter_validation(native):
    assert native.esim_levels(0.0, 1e-3) == -1
    assert native.esim_levels(0.6, 1.0) == -1
    assert native.esim_sample_base(0, 0.6, 1e-3, 0.0) == -1.0


@pytest.mark.parametrize("case", ["rowptr0", "decreasing", "col_range", "negative_col", "n_zero"])
def test_load_graph_rejects_bad_csr(native, case):
    n, rp, col = synth.erdos_renyi(50, 200, seed=1)
    rp = rp.copy()
    col = col.copy()
    if case == "rowptr0":
        rp[0] = 1
    elif case == "decreasing":
        rp[10] = rp[11] + 1
    elif case == "col_range":
        col[5] = n
    elif case == "negative_col":
        col[5] = -1
    elif case == "n_zero":
        with pytest.raises(native.EsimError) as e:
            native.esim_load_graph(0, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32))
        assert e.value.status == -1
        return
    with pytest.raises(native.EsimError) as e:
        native.esim_load_graph(n, rp, col)
    assert e.value.status == -1  # ESIM_EINVAL, raised before any device work


def test_null_handle_is_rejected(native):
    out = np.empty(4)
    with pytest.raises(native.EsimError) as e:
        native.esim_query(None, 0, 0.6, 1e-3, 0, out)
    assert e.value.status == -1


def test_alg3_cost_model_depth_is_the_documented_argmin(native):
    """The library's cost-model depth choice (host arithmetic, option alg3_rule = 1) is the
    argmin of the cost its header documents, restated in tests/alg3_cost_plan.py, bit for
    bit over random work estimates and real supports."""
    import alg3_cost_plan as cp
    from oracle import power
    rng = np.random.default_rng(5)
    n, rp, col = synth.chung_lu(3000, 30000, gamma=2.1, seed=9)
    m = int(rp[-1])
    P = power.transition_matrix(n, rp, col)
    supps = [cp.supports(P, int(k), 14) for k in rng.choice(n, 12, replace=False)]
    checked = 0
    for trial in range(400):
        supp = supps[trial % len(supps)]
        v = float(10 ** rng.uniform(2, 15))
        c = float(rng.choice([0.6, 0.8, 0.5]))
        max_depth = int(rng.integers(0, 17))
        weights = (float(rng.choice([4.0, 1.0])), float(rng.choice([0.2, 0.5, 0.05])),
                   float(rng.choice([524288.0, 2.0 ** 16])), float(rng.choice([0.0625, 1.0, 0.0])))
        costs = [cp.cost(d, v, c, supp, n, m, *weights) for d in range(max_depth + 1)]
        want = min(range(max_depth + 1), key=lambda d: (costs[d], d))
        got = native.esim_alg3_depth(v, c, supp[:max(1, max_depth - 1)] + [0] * 2, max_depth, n, m, weights)
        assert got == want, (v, c, max_depth, weights, costs)
        checked += want > 0
    assert checked > 50  # exploitation is chosen often enough to matter
    # invalid arguments
    assert native.esim_alg3_depth(1e9, 1.5, [1, 2, 3], 3, n, m) == -1
    assert native.esim_alg3_depth(1e9, 0.6, [1, 2, 3], 17, n, m) == -1


def test_no_cpu_fallback_without_a_device(native):
    """Without a usable CUDA device the device calls report ESIM_ECUDA: no call computes
    on the CPU instead."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    n, rp, col = synth.erdos_renyi(50, 200, seed=1)
    with pytest.raises(native.EsimError) as e:
        native.esim_load_graph(n, rp, col)
    assert e.value.status == -3


def test_missing_library_raises(native, monkeypatch):
    """The binding refuses to run when the CUDA library was not built."""
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libexactsim.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        native.lib()
