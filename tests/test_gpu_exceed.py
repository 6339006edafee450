"""Theorem 1 at the benchmark's settings: max_v |s(v) - S(u, v)| <= eps, over 100 seeds.

The timed workload (directed Chung-Lu n = 1e5, m = 1e6, gamma 2.1, eps = 1e-6) is out
of the Power Method's reach (S would take 80 GB), so this test takes the same recipe
at n = 2e4, m = 2e5 (S: 3.2 GB, by the oracle's C Power Method to c^45 = 1e-10), and
runs the benchmark's exact options: eps = 1e-6, kappa = 4, FP64, Algorithm 3 with the
library's cost-model rule (alg3_rule 1, depth <= 8, 128 candidates).  100 seeded queries cycle over five
seeded sources.  It asserts that no query's error exceeds eps, and prints the exceed
rate and the error distribution (over all v, and over v != u) as one JSON line.

Lemma 2 bounds the sampling standard deviation of s(v) by
sqrt(||pi_v||^2 / (4 (1 - sqrt c)^4 R_b)); at kappa = 4 this is at most 1.45e-6 for an
arbitrary node and 3.7e-7 for the source, whose own pairs dominate the error, so the
bound alone does not give max-err <= eps at this kappa: the measurement does.
"""
import json

import numpy as np
import pytest

import synth
from oracle import power

pytestmark = pytest.mark.gpu

C = 0.6
EPS = 1e-6
KAPPA = 4.0
SEEDS = 100


def test_exceed_rate_at_the_benchmark_settings():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for gpu tests")
    import paper_2004_03493_gb300 as esim
    esim.build()
    n, rp, col = synth.chung_lu(20_000, 200_000, gamma=2.1, seed=1)
    srcs = [int(x) for x in synth.random_sources(rp, 5, seed=7)]
    S = power.power_method_c(n, rp, col, C, iterations=power.power_iterations(C, 1e-10))
    g = esim.Graph(n, rp, col, kappa=KAPPA, alg3=1, alg3_rule=1, alg3_max_depth=8, alg3_max_nodes=128,
                   alg3_overlap=5)
    errs, errs_off, pairs, nodes = [], [], [], []
    for seed in range(SEEDS):
        u = srcs[seed % len(srcs)]
        s = g.query(u, C, EPS, seed)
        st = g.stats()
        d = np.abs(s - S[u])  # S is symmetric: row u is column u
        errs.append(float(d.max()))
        d[u] = 0.0
        errs_off.append(float(d.max()))
        pairs.append(st["sum_R"])
        nodes.append(st["alg3_nodes"])
    g.close()
    errs = np.array(errs)
    errs_off = np.array(errs_off)
    summary = {"graph": f"chung_lu n={n} m={len(col)} gamma=2.1 seed=1", "sources": srcs, "eps": EPS,
               "kappa": KAPPA, "dhat": "Algorithm 3, cost-model rule, depth <= 8", "seeds": SEEDS,
               "exceed": int(np.sum(errs > EPS)), "max_err": float(errs.max()), "p50_err": float(np.median(errs)),
               "p99_err": float(np.percentile(errs, 99)), "max_err_off_source": float(errs_off.max()),
               "pairs_per_query": float(np.mean(pairs)), "alg3_nodes_per_query": float(np.mean(nodes))}
    print("EXCEED " + json.dumps(summary))
    assert summary["exceed"] == 0, summary
