"""Algorithm 3 ("Improved method for estimating D(k,k)") in the oracle, FP64.

Test infrastructure only (see ``oracle/__init__.py``).

* ``first_meeting_lemma5`` -- Z_l(k) = sum_q Z_l(k, q) for l = 1..depth by the
  recursion of Lemma 5:
      Z_l(k, q) = c^l (P^T)^l(k, q)^2
                  - sum_{l'=1}^{l-1} sum_{q'} c^{l'} (P^T)^{l'}(q', q)^2 Z_{l-l'}(k, q'),
  where (P^T)^l(k, .) is the distribution of a non-stop walk (uniform in-neighbour
  moves) from k after l steps.  Each (P^T)^j(q', .) is propagated separately, so
  the code follows the lemma term by term.
* ``first_meeting_bruteforce`` -- the same quantity from the definition: the exact
  (rational) distribution of two non-stop walks from k over pairs of nodes, step by
  step, removing the pairs that have met; Z_l = c^l * (mass that first meets at
  step l).  An independent formulation that pins the lemma's recursion.
* ``exploitation_plan`` -- the exploitation the library uses: the heaviest nodes (by
  pi(k), at most ``max_nodes``, with R(k) >= ``min_pairs`` and din(k) >= 2) take the
  depth that minimises ``exploit_cost`` (the paper stops its adaptive exploration
  when the explored edges reach the walk work; the cost here weighs the library's
  dense sweeps against its walks); their sample count becomes
  max(1, ceil(R_b pi(k)^2 c^(2 depth))).  Nodes with din <= 1 take the exact values of
  Algorithm 3 (D = 1 at din = 0, 1 - c at din = 1) and no samples.
* ``dhat_alg3`` -- D^(k) = 1 - sum_{l <= depth} Z_l(k) - c^depth * tailmeet(k) / R(k)
  for exploited nodes (Algorithm 3), nonmeet / R for the others.

Pinned by: the rational brute force (Z to 1e-14), the identity
sum_l Z_l(k) = 1 - D(k) against the Power Method's exact D (the truncated sum stays
below it and the tail estimator closes the gap), and z-tests of the tail walks.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from .power import transition_matrix, in_degrees


def walk_distribution(P, k: int, steps: int) -> np.ndarray:
    """(P^T)^l(k, .) for l = 0..steps: non-stop walk from k along in-edges (rows l)."""
    n = P.shape[0]
    H = np.zeros((steps + 1, n))
    H[0, k] = 1.0
    for ell in range(1, steps + 1):
        H[ell] = P @ H[ell - 1]
    return H


def first_meeting_lemma5(n: int, in_rowptr, in_col, k: int, c: float, depth: int) -> list[float]:
    P = transition_matrix(n, in_rowptr, in_col)
    hk = walk_distribution(P, k, depth)
    cache: dict[int, np.ndarray] = {}

    def h_from(q: int, j: int) -> np.ndarray:
        if q not in cache:
            cache[q] = walk_distribution(P, q, depth)
        return cache[q][j]

    Z = [None]  # Z[l] is the vector Z_l(k, .)
    for ell in range(1, depth + 1):
        z = c ** ell * hk[ell] ** 2
        for lp in range(1, ell):
            # sum_{q'} c^{l'} (P^T)^{l'}(q', .)^2 Z_{l-l'}(k, q')
            zz = Z[ell - lp]
            for qp in np.nonzero(zz)[0]:
                z = z - c ** lp * h_from(int(qp), lp) ** 2 * zz[qp]
        Z.append(z)
    return [float(Z[ell].sum()) for ell in range(1, depth + 1)]


def first_meeting_bruteforce(n: int, in_rowptr, in_col, k: int, c: Fraction, depth: int) -> list[Fraction]:
    """Exact Z_1..Z_depth from the pair distribution of two non-stop walks (tiny graphs)."""
    c = Fraction(c)
    rp = [int(x) for x in in_rowptr]
    col = [int(x) for x in in_col]
    I = [col[rp[j]:rp[j + 1]] for j in range(n)]
    dist = {(k, k): Fraction(1)}  # step 0 is not a meeting
    out = []
    for ell in range(1, depth + 1):
        nxt: dict[tuple[int, int], Fraction] = {}
        for (a, b), w in dist.items():
            if not I[a] or not I[b]:
                continue
            wa = Fraction(1, len(I[a]))
            wb = Fraction(1, len(I[b]))
            for x in I[a]:
                for y in I[b]:
                    nxt[(x, y)] = nxt.get((x, y), Fraction(0)) + w * wa * wb
        met = sum((w for (x, y), w in nxt.items() if x == y), Fraction(0))
        out.append(c ** ell * met)
        dist = {p: w for p, w in nxt.items() if p[0] != p[1]}
    return out


def exploit_cost(d: int, v: float, c: float, supp, n: int, m: int, w_sweep: float = 4.0, w_probe: float = 0.2,
                 w_launch: float = 524288.0) -> float:
    """Estimated GPU work (in sampler pair-steps) of exploiting a node to depth d.

    d = 0 is Algorithm 2 alone.  Walks: R_d (d + 1/(1-c)) with R_d = max(1, ceil(v c^(2d))),
    v = R_b pi(k)^2.  Lemma 5 at depth d: 2d-1 single sweeps of m+n entries (weight
    w_sweep per entry), sum_{i=1}^{d-2} |supp h_i| (d-i) probe column-sweeps (w_probe per
    entry and column), and w_launch per kernel launch (3 per sweep; 3 per probe step and
    2 per block of 32 probes).  The same arithmetic, in the same order, as the library's plan,
    so that both sides pick the same depth.
    """
    r = math.ceil(v) if d == 0 else math.ceil(v * c ** (2 * d))
    r = max(1.0, float(r))
    cost = r * (d + 1.0 / (1.0 - c))
    if d > 0:
        edges = float(m + n)
        probe = 0
        launches = 3 * (2 * d - 1)
        for i in range(1, d - 1):
            probe += int(supp[i]) * (d - i)
            launches += (int(supp[i]) + 31) // 32 * (3 * (d - i) + 2)
        cost += w_sweep * edges * float(2 * d - 1)
        cost += w_probe * edges * float(probe)
        cost += w_launch * float(launches)
    return cost


def supports(P, k: int, levels: int) -> list[int]:
    """|supp h_i| for i = 0..levels, h_i the non-stop walk distribution from k."""
    H = walk_distribution(P, k, levels)
    return [int(np.count_nonzero(H[i])) for i in range(levels + 1)]


def exploitation_plan(n: int, in_rowptr, in_col, pi: np.ndarray, R_b: float, c: float, max_depth: int = 8,
                      min_pairs: float = 1e6, max_nodes: int = 64, stats: dict | None = None,
                      weights: tuple = (4.0, 0.2, 524288.0), mode: str = "pi2"):
    """(depth uint8[n], R uint64[n]) of Algorithm 3 with the cost-minimising depth.

    Candidates: the max_nodes largest pi(k) (ties to the lower id) with pi(k) > 0,
    din(k) >= 2 and an Algorithm 2 count max(1, ceil(v)) >= min_pairs, v = R_b pi(k)^2
    (R_b pi(k) for the basic allocation).  Each takes the depth d in 0..max_depth of
    least ``exploit_cost`` (the first on ties); d > 0 gives R(k) = max(1, ceil(v c^(2d))).  Nodes with din <= 1 take the
    exact D and no samples.  ``stats["min_gap"]`` (if given) receives the smallest
    relative gap between a chosen cost and another depth's cost: the margin of the
    floating-point depth decisions.
    """
    min_gap = math.inf
    din = in_degrees(in_rowptr)
    m = int(np.asarray(in_rowptr)[-1])
    P = transition_matrix(n, in_rowptr, in_col)
    pi = np.asarray(pi, dtype=np.float64)
    R = np.ceil(R_b * (pi * pi) if mode == "pi2" else R_b * pi).astype(np.uint64)
    R[(pi > 0) & (R == 0)] = 1
    depth = np.zeros(n, dtype=np.uint8)
    R[din <= 1] = 0  # exact D for din 0 and 1
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
        costs = [exploit_cost(dd, v, c, supp, n, m, *weights) for dd in range(max_depth + 1)]
        d, best = 0, costs[0]
        for dd in range(1, max_depth + 1):
            if costs[dd] < best:
                d, best = dd, costs[dd]
        for dd, cost in enumerate(costs):
            if dd != d:
                min_gap = min(min_gap, abs(cost - best) / best)
        if d == 0:
            continue
        depth[kk] = d
        R[kk] = max(1, int(math.ceil(v * c ** (2 * d))))
    if stats is not None:
        stats["min_gap"] = min_gap
    return depth, R


def dhat_alg3(counts: np.ndarray, R: np.ndarray, depth: np.ndarray, zsum: np.ndarray, din: np.ndarray,
              c: float) -> np.ndarray:
    """D^ of Algorithm 3 (exploited nodes), Algorithm 2 (others), exact values at din <= 1."""
    counts = np.asarray(counts, dtype=np.uint64)
    R = np.asarray(R, dtype=np.uint64)
    D = np.zeros(R.size)
    nz = R > 0
    D[nz] = counts[nz].astype(np.float64) / R[nz].astype(np.float64)
    ex = depth > 0
    D[ex] = 1.0 - zsum[ex] - (c ** depth[ex].astype(np.float64)) * (
        counts[ex].astype(np.float64) / R[ex].astype(np.float64))
    D[din == 0] = 1.0
    D[din == 1] = 1.0 - c
    return D
