"""The library's cost-model plan for Algorithm 3 (option alg3_rule = 1), restated for tests.

This is not the oracle and not the paper's rule: it is the speed choice the library
documents in include/exactsim.h (options "alg3_rule", "alg3_w_*"), written out here so
that tests can hand the oracle the same test-chosen plan -- (depth, R) per node -- and
compare the library's whole query with it.  ``test_abi_host`` pins ``cost`` against the
library's own host function ``esim_alg3_depth`` bit for bit.

cost(d) of node k, in sampler pair-steps: R_d (d + 1/(1-c)) walk work, R_d =
max(1, ceil(v c^(2d))), v = R_b pi(k)^2 (R_b pi(k) for the basic allocation), plus for
d > 0 w_sweep (m+n)(2d-1) + w_probe (m+n) (sum_{i=1}^{d-4} |supp h_i|(d-i) +
w_last sum_{i=max(1,d-3)}^{d-2} (d-i)|supp h_i|) + w_launch (3(2d-1) + sum_{i=1}^{d-4}
ceil(|supp h_i|/32)(3(d-i)+2) + 2 per level i in max(1,d-3)..d-2), h_i = (P^T)^i(k, .).
"""
from __future__ import annotations

import math

import numpy as np

from oracle.alg3 import walk_distribution
from oracle.power import in_degrees, transition_matrix

WEIGHTS = (4.0, 0.2, 524288.0, 0.0625)


def cost(d: int, v: float, c: float, supp, n: int, m: int, w_sweep: float = 4.0, w_probe: float = 0.2,
         w_launch: float = 524288.0, w_last: float = 0.0625) -> float:
    r = math.ceil(v) if d == 0 else math.ceil(v * c ** (2 * d))
    r = max(1.0, float(r))
    total = r * (d + 1.0 / (1.0 - c))
    if d > 0:
        edges = float(m + n)
        probe = 0
        launches = 3 * (2 * d - 1)
        for i in range(1, d - 3):
            probe += int(supp[i]) * (d - i)
            launches += (int(supp[i]) + 31) // 32 * (3 * (d - i) + 2)
        last = 0.0
        for i in range(max(1, d - 3), d - 1):
            last += w_last * (float(d - i) * float(supp[i]))
            launches += 2
        total += w_sweep * edges * float(2 * d - 1)
        total += w_probe * edges * (float(probe) + last)
        total += w_launch * float(launches)
    return total


def supports(P, k: int, levels: int) -> list[int]:
    """|supp h_i| for i = 0..levels."""
    H = walk_distribution(P, k, levels)
    return [int(np.count_nonzero(H[i])) for i in range(levels + 1)]


def plan(n: int, in_rowptr, in_col, pi: np.ndarray, R_b: float, c: float, max_depth: int = 8,
         min_pairs: float = 1e6, max_nodes: int = 64, mode: str = "pi2", weights=WEIGHTS):
    """(depth uint8[n], R uint64[n], min_gap): the cost model's plan and the smallest
    relative gap between a chosen cost and another depth's (the margin of the FP64
    depth decisions; tests skip a source whose gap is within rounding)."""
    min_gap = math.inf
    din = in_degrees(in_rowptr)
    m = int(np.asarray(in_rowptr)[-1])
    P = transition_matrix(n, in_rowptr, in_col)
    pi = np.asarray(pi, dtype=np.float64)
    R = np.ceil(R_b * (pi * pi) if mode == "pi2" else R_b * pi).astype(np.uint64)
    R[(pi > 0) & (R == 0)] = 1
    depth = np.zeros(n, dtype=np.uint8)
    R[din <= 1] = 0
    order = np.lexsort((np.arange(n), -pi))[:max_nodes]
    for kk in order:
        kk = int(kk)
        if not pi[kk] > 0:
            break
        if din[kk] < 2:
            continue
        v = R_b * (pi[kk] * pi[kk]) if mode == "pi2" else R_b * pi[kk]
        if max(1.0, float(math.ceil(v))) < min_pairs:
            continue
        supp = supports(P, kk, max(0, max_depth - 2))
        costs = [cost(dd, v, c, supp, n, m, *weights) for dd in range(max_depth + 1)]
        d, best = 0, costs[0]
        for dd in range(1, max_depth + 1):
            if costs[dd] < best:
                d, best = dd, costs[dd]
        for dd, cc in enumerate(costs):
            if dd != d:
                min_gap = min(min_gap, abs(cc - best) / best)
        if d == 0:
            continue
        depth[kk] = d
        R[kk] = max(1, int(math.ceil(v * c ** (2 * d))))
    return depth, R, min_gap
