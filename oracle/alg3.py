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
* ``explored_edges`` / ``explored_edges_literal`` -- the counter E_k of Algorithm 3:
  every edge the exploration traverses when it extends a walk distribution
  (P^T)^(l')(q', .) by one step, level by level (a vectorised form over all nodes,
  and the listing's loops written out for small graphs).
* ``paper_depth`` / ``exploitation_plan`` -- Algorithm 3's adaptive depth: node k
  stops at the level during which E_k reaches 2 R(k)/sqrt(c), the expected step
  count of its R(k) walk pairs; nodes with din <= 1 take the exact D and no pairs.
* ``first_meeting_sums`` -- sum_{l <= depth(k)} Z_l(k) for every node at once (Lemma 5
  with the sum over q' as a matrix product).
* ``dhat_alg3`` -- D^(k) = 1 - sum_{l <= depth} Z_l(k) - c^depth * tailmeet(k) / R(k)
  for exploited nodes (Algorithm 3), nonmeet / R for the others.

Pinned by: the rational brute force (Z to 1e-14); the identity
sum_l Z_l(k) = 1 - D(k) against the Power Method's exact D (the truncated sum stays
below it, an exhausted exploration reaches it, and the tail estimator closes the gap
without bias: z-tests); the counter against the listing's loops on small graphs and
against its closed form on the complete digraph.
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


def explored_edges_literal(n: int, in_rowptr, in_col, k: int, levels: int) -> list[int]:
    """E_k at the end of each level l = 0..levels, by the loops of Algorithm 3 as printed.

    At level l, for every l' = 0..l, every q' with (P^T)^(l-l')(k, q') != 0 and every x
    with (P^T)^(l')(q', x) != 0, the step to each q in I(x) adds one explored edge.
    Walk distributions are kept per (q', l') and extended one step at a time.  Pure
    Python, for small graphs: it pins ``explored_edges``.
    """
    rp = [int(x) for x in in_rowptr]
    col = [int(x) for x in in_col]
    inn = [col[rp[j]:rp[j + 1]] for j in range(n)]
    dists: dict[int, list[dict[int, Fraction]]] = {}

    def dist(q: int, ell: int) -> dict[int, Fraction]:
        if q not in dists:
            dists[q] = [{q: Fraction(1)}]
        d = dists[q]
        while len(d) <= ell:
            nxt: dict[int, Fraction] = {}
            for x, w in d[-1].items():
                for y in inn[x]:
                    nxt[y] = nxt.get(y, Fraction(0)) + w / len(inn[x])
            d.append(nxt)
        return d[ell]

    E = 0
    out = []
    for ell in range(levels + 1):
        for lp in range(ell + 1):
            for qp, wq in dist(k, ell - lp).items():
                if wq == 0:
                    continue
                for x, wx in dist(qp, lp).items():
                    if wx != 0:
                        E += len(inn[x])
        out.append(E)
    return out


def explored_edges(n: int, in_rowptr, in_col, levels: int) -> np.ndarray:
    """E[l, k]: explored edges of Algorithm 3 from node k at the end of level l.

    supp (P^T)^j(q, .) is row q of the boolean j-th power of A, A(q, x) = [x in I(q)]
    (a library matrix product per power).  e_j(q) = sum of din(x) over that support
    is the number of edges the listing traverses when it extends (P^T)^j(q', .) by a
    step; level l adds W_l(k) = sum_{l'=0..l} sum_{q' in supp (P^T)^(l-l')(k, .)} e_l'(q').
    Dense n x n matrices: small graphs only.
    """
    # 0/1 matrices and integer sums below 2^53 multiply exactly in FP64 (BLAS)
    din = in_degrees(in_rowptr).astype(np.float64)
    rp = np.asarray(in_rowptr, dtype=np.int64)
    col = np.asarray(in_col, dtype=np.int64)
    A = np.zeros((n, n))
    A[np.repeat(np.arange(n), np.diff(rp)), col] = 1.0
    supp = [np.eye(n)]
    for _ in range(levels):
        supp.append(((supp[-1] @ A) > 0).astype(np.float64))
    e = [S @ din for S in supp]  # e[j][q]
    E = np.zeros((levels + 1, n), dtype=np.int64)
    run = np.zeros(n, dtype=np.int64)
    for ell in range(levels + 1):
        W = np.zeros(n, dtype=np.int64)
        for lp in range(ell + 1):
            W += np.rint(supp[ell - lp] @ e[lp]).astype(np.int64)
        run = run + W
        E[ell] = run
    return E


def paper_depth(E_k, R_k: int, c: float, max_depth: int) -> int:
    """l(k) of Algorithm 3: the level during which E_k reaches 2 R(k)/sqrt(c).

    E_k[l] is the count at the end of level l.  Two readings where the listing gives
    no stop: a level that adds no edge (every node reached at that level has din 0,
    so no walk pair can meet later and the Z up to that level give D exactly) stops
    the exploration at that level, and so does ``max_depth``.
    """
    T = 2.0 * float(R_k) / math.sqrt(c)
    prev = 0
    for ell in range(max_depth + 1):
        cur = int(E_k[ell])
        if float(cur) >= T:
            return ell
        if ell > 0 and cur == prev:
            return ell
        prev = cur
    return max_depth


def exploitation_plan(n: int, in_rowptr, in_col, pi: np.ndarray, R_b: float, c: float, max_depth: int = 16,
                      mode: str = "pi2"):
    """(depth uint8[n], R uint64[n]) of Algorithm 3 with the paper's adaptive depth.

    R(k) is the allocation of Lemma 4 (pi2) or Algorithm 1 (basic).  Nodes with din 0
    or 1 take the exact D (Algorithm 3's first cases) and no pairs.  Every other node
    with R(k) > 0 explores until E_k >= 2 R(k)/sqrt(c) (``paper_depth``) and keeps its
    R(k) pairs, which move without stopping for l(k) steps.
    """
    din = in_degrees(in_rowptr)
    pi = np.asarray(pi, dtype=np.float64)
    R = np.ceil(R_b * (pi * pi) if mode == "pi2" else R_b * pi).astype(np.uint64)
    R[(pi > 0) & (R == 0)] = 1
    R[din <= 1] = 0
    depth = np.zeros(n, dtype=np.uint8)
    cand = np.nonzero(R > 0)[0]
    if cand.size:
        E = explored_edges(n, in_rowptr, in_col, max_depth)
        for k in cand:
            depth[k] = paper_depth(E[:, k], int(R[k]), c, max_depth)
    return depth, R


def first_meeting_sums(n: int, in_rowptr, in_col, depth: np.ndarray, c: float) -> np.ndarray:
    """zsum(k) = sum_{l=1..depth(k)} Z_l(k) for every node, Lemma 5 in matrix form.

    With M_j = (P^T)^j (dense) and Q_j = M_j * M_j (element-wise), row k of
    Z_l = c^l Q_l - sum_{l'=1..l-1} c^l' Z_(l-l') Q_l' is Lemma 5 for node k: the sum
    over q' is a library matrix product.  Rows are kept only while l <= depth(k).
    Small graphs only; ``first_meeting_lemma5`` is the term-by-term form that pins it.
    """
    depth = np.asarray(depth)
    D = int(depth.max()) if depth.size else 0
    zsum = np.zeros(n)
    if D == 0:
        return zsum
    P = transition_matrix(n, in_rowptr, in_col)
    PT = P.T.toarray()
    M = [np.eye(n)]
    for _ in range(D):
        M.append(M[-1] @ PT)  # (P^T)^j: row k is the walk distribution from k after j steps
    Q = [x * x for x in M]
    rows = np.nonzero(depth > 0)[0]
    Z = [None]  # Z[l]: Z_l restricted to `rows`
    for ell in range(1, D + 1):
        z = c ** ell * Q[ell][rows]
        for lp in range(1, ell):
            z = z - c ** lp * (Z[ell - lp] @ Q[lp])
        Z.append(z)
        keep = depth[rows] >= ell
        zsum[rows[keep]] += z[keep].sum(axis=1)
    return zsum


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
