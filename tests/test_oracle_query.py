"""The whole CPU ExactSim query against the Power Method (Theorem 1).

With the paper's constant (kappa = 6 / (1 - sqrt c)^4) Theorem 1 says every
|s(v) - S(u, v)| <= eps with probability at least 1 - 1/n.  The checks use fixed
seeds, so they are deterministic.
"""
import numpy as np
import pytest

import synth
from oracle import exactsim, power

C = 0.6


@pytest.mark.parametrize("mode", ["pi2", "basic"])
def test_cpu_exactsim_within_eps_of_power_method(oracle_walks, mode):
    g = synth.erdos_renyi(300, 2400, seed=4)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 2e-2 if mode == "basic" else 5e-3
    for u, seed in ((0, 1), (57, 2)):
        q = exactsim.query(n, rp, col, u, C, eps, seed=seed, mode=mode)
        err = np.max(np.abs(q.s - S[:, u]))
        assert err <= eps, (u, err)
        assert q.R.sum() > 0


def test_cpu_exactsim_power_law_graph(oracle_walks):
    g = synth.chung_lu(400, 4000, gamma=2.1, seed=13)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    eps = 5e-3
    u = int(synth.random_sources(rp, 1, seed=3)[0])
    q = exactsim.query(n, rp, col, u, C, eps, seed=7)
    assert np.max(np.abs(q.s - S[:, u])) <= eps
