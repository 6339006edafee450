"""Pins of O3, the CPU walk-pair sampler of Algorithm 2 and its Philox stream.

* Philox-4x32-10 against Triton's CPU interpreter (an independent implementation
  of the generator of Salmon et al., SC'11).
* E[D^(k)] = D(k) (Algorithm 2 is a Bernoulli estimator of D) against the exact D
  of the Power Method and of the rational first-meeting solve: z-tests.
* din = 0 gives D^ = 1 exactly; din = 1 gives D = 1 - c (Algorithm 3's cases).
* Counts do not depend on the number of threads; seeds matter.
"""
import json
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import linearization as lin
from oracle import pair_chain, power

C = 0.6

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0); c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2); c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a); tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c); tl.store(out_ptr + 4 * i + 3, d)
req = json.loads(sys.stdin.read())
ctr = torch.tensor(req["ctr"], dtype=torch.int64).to(torch.uint32)
out = torch.zeros_like(ctr)
k[(1,)](ctr, out, req["seed"], N=ctr.shape[0])
print(json.dumps(out.to(torch.int64).tolist()))
"""


def _triton_philox(ctr, seed):
    pytest.importorskip("triton")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps({"ctr": ctr.tolist(), "seed": seed}),
                       capture_output=True, text=True, timeout=600,
                       env={**os.environ, "TRITON_INTERPRET": "1"})
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    return np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64)


def test_philox_matches_triton_interpreter(oracle_walks):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 2 ** 32 - 1
    for seed in (0, 0x243F6A8885A308D3, 2 ** 64 - 1):
        ref = _triton_philox(ctr, seed)
        got = oracle_walks.philox(ctr.astype(np.uint32), seed).astype(np.uint64)
        assert np.array_equal(got, ref)


def test_threshold_matches_formula(oracle_walks):
    for c in (0.6, 0.8, 0.25, 1e-9, 0.999999):
        assert oracle_walks.threshold(c) == lin.pair_threshold(c)


def _z(dhat, D, R):
    sd = np.sqrt(np.maximum(D * (1 - D), 1e-300) / R)
    return np.abs(dhat - D) / sd


def test_dhat_unbiased_against_power_method(oracle_walks):
    g = synth.chung_lu(60, 400, gamma=2.1, seed=12)
    n, rp, col = g
    S = power.power_method(n, rp, col, C)
    D = power.exact_diagonal(n, rp, col, C, S)
    R = np.full(n, 100_000, dtype=np.uint64)
    nonmeet, steps = oracle_walks.walk_pairs(n, rp, col, R, C, seed=99)
    dh = lin.dhat(nonmeet, R)
    din = np.diff(rp)
    assert np.all(dh[din == 0] == 1.0)
    live = (din > 0) & (D < 1 - 1e-12)
    assert np.max(_z(dh[live], D[live], 100_000)) < 5.0
    # steps per pair: at least 1, at most the mean length of a joint walk 1/(1-c)
    assert n * 100_000 <= steps <= n * 100_000 / (1 - C) * 1.01


def test_dhat_unbiased_against_exact_rational_D(oracle_walks):
    g = synth.random_small(7, p=0.45, seed=31)
    n, rp, col = g
    D = pair_chain.to_float(pair_chain.exact_diagonal_rational(n, rp, col, Fraction(3, 5)))
    R = np.full(n, 400_000, dtype=np.uint64)
    nonmeet, _ = oracle_walks.walk_pairs(n, rp, col, R, C, seed=5)
    dh = lin.dhat(nonmeet, R)
    live = D < 1 - 1e-12
    assert np.max(_z(dh[live], D[live], 400_000)) < 5.0


def test_single_in_neighbour_gives_one_minus_c(oracle_walks):
    g = synth.directed_cycle(10)
    n, rp, col = g
    R = np.full(n, 200_000, dtype=np.uint64)
    nonmeet, steps = oracle_walks.walk_pairs(n, rp, col, R, C, seed=3)
    dh = lin.dhat(nonmeet, R)
    assert np.max(_z(dh, np.full(n, 1 - C), 200_000)) < 5.0
    # every pair ends after exactly one step on a cycle (meet or stop)
    assert steps == n * 200_000


def test_dangling_source_never_meets(oracle_walks):
    g = synth.in_star(5)  # leaves have din = 0
    n, rp, col = g
    R = np.array([0, 7, 7, 7, 7, 7], dtype=np.uint64)
    nonmeet, steps = oracle_walks.walk_pairs(n, rp, col, R, C, seed=1)
    assert nonmeet.tolist() == [0, 7, 7, 7, 7, 7]
    assert steps == 35


def test_thread_count_independence_and_seed_dependence(oracle_walks):
    g = synth.erdos_renyi(500, 5000, seed=8)
    n, rp, col = g
    R = np.random.default_rng(1).integers(0, 3000, size=n).astype(np.uint64)
    a, sa = oracle_walks.walk_pairs(n, rp, col, R, C, seed=42, threads=1)
    b, sb = oracle_walks.walk_pairs(n, rp, col, R, C, seed=42, threads=4)
    assert np.array_equal(a, b) and sa == sb
    d, _ = oracle_walks.walk_pairs(n, rp, col, R, C, seed=43, threads=4)
    assert not np.array_equal(a, d)
    assert np.all(a <= R)


def test_pick_is_exactly_uniform_with_rejection(oracle_walks):
    # d = 3 * 2^30: 2^32 mod d = 2^30, so a quarter of the words are rejected and redrawn
    d = 3 * 2 ** 30
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2 ** 32, size=60000, dtype=np.uint64).astype(np.uint32)
    got = oracle_walks.pick(x, d, seed=9).astype(np.uint64)
    assert got.max() < d
    plain = (x.astype(np.uint64) * d) >> 32
    low = (x.astype(np.uint64) * d) & 0xFFFFFFFF
    accepted = low >= 2 ** 30
    assert np.array_equal(got[accepted], plain[accepted])       # accepted words keep multiply-shift
    assert 0.23 < 1 - accepted.mean() < 0.27                     # rejection rate 1/4
    # multiply-shift alone maps x to floor(3x/4): indices i = 0 mod 3 receive two words of
    # every four, so they would carry probability 1/2 instead of 1/3
    frac_plain = float(np.mean(plain % 3 == 0))
    frac_got = float(np.mean(got % 3 == 0))
    assert abs(frac_plain - 0.5) < 0.01
    assert abs(frac_got - 1.0 / 3.0) < 0.01
    # small d: no word is ever rejected
    assert np.array_equal(oracle_walks.pick(x, 7), ((x.astype(np.uint64) * 7) >> 32).astype(np.uint32))
