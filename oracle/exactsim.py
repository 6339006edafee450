"""The whole CPU ExactSim query: Algorithm 1 with Algorithm 2 (or 3) as its D estimator.

Test infrastructure only (see ``oracle/__init__.py``).  It runs the steps in the
paper's order -- L, hop vectors, allocation, walk pairs, D^, reverse
accumulation -- from ``linearization`` (NumPy/SciPy FP64) and ``walks`` (C,
OpenMP).  This is also the plain multithreaded CPU ExactSim the benchmark times.

Pinned by: max_v |s(v) - S(u, v)| <= eps against the Power Method on small
graphs, and the pins of its parts.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import alg3 as a3
from . import linearization as lin
from . import walks


@dataclass
class QueryResult:
    s: np.ndarray
    H: np.ndarray
    pi: np.ndarray
    R: np.ndarray
    nonmeet: np.ndarray
    D: np.ndarray
    L: int
    R_b: float
    pair_steps: int
    depth: np.ndarray | None = None
    zsum: np.ndarray | None = None


def query(n: int, in_rowptr, in_col, u: int, c: float, eps: float, seed: int = 0,
          kappa: float | None = None, mode: str = "pi2", threads: int = 0, alg3: bool = False,
          alg3_max_depth: int = 16, alg3_plan=None, sparse: bool = False, diag: str = "estimated") -> QueryResult:
    """One single-source query.  ``sparse``: sparse Linearization (Sec. 3.2) -- the
    query runs at eps/2 and the reverse loop reads the history with entries at or
    below (1 - sqrt(c))^2 eps/2 dropped (pi for the allocation is the full sum).
    ``diag="parsim"``: D = (1 - c) I with no walks, ParSim's approximation (Sec. 2).
    ``alg3``: Algorithm 3 with the paper's adaptive depth (explore until the explored
    edges reach 2 R(k)/sqrt(c), at most ``alg3_max_depth`` levels), or with a given
    ``alg3_plan`` = (depth uint8[n], R uint64[n]) chosen by the caller."""
    if sparse:
        eps = 0.5 * eps
    L = lin.levels(c, eps)
    H = lin.hop_vectors(n, in_rowptr, in_col, u, c, L)
    pi = lin.ppr(H)
    R_b = lin.sample_base(n, c, eps, kappa)
    Hr = lin.sparsify(H, lin.sparse_threshold(c, eps)) if sparse else H
    if diag == "parsim":
        D = np.full(n, 1.0 - c)
        s = lin.reverse(n, in_rowptr, in_col, Hr, D, c)
        z = np.zeros(n, dtype=np.uint64)
        return QueryResult(s=s, H=Hr, pi=pi, R=z, nonmeet=z, D=D, L=L, R_b=R_b, pair_steps=0)
    if not alg3:
        R = lin.allocate(pi, R_b, mode)
        nonmeet, steps = walks.walk_pairs(n, in_rowptr, in_col, R, c, seed, threads)
        D = lin.dhat(nonmeet, R)
        s = lin.reverse(n, in_rowptr, in_col, Hr, D, c)
        return QueryResult(s=s, H=Hr, pi=pi, R=R, nonmeet=nonmeet, D=D, L=L, R_b=R_b, pair_steps=steps)
    if alg3_plan is None:
        depth, R = a3.exploitation_plan(n, in_rowptr, in_col, pi, R_b, c, alg3_max_depth, mode)
    else:
        depth = np.asarray(alg3_plan[0], dtype=np.uint8)
        R = np.asarray(alg3_plan[1], dtype=np.uint64)
    zsum = a3.first_meeting_sums(n, in_rowptr, in_col, depth, c)
    counts, steps = walks.walk_pairs_depth(n, in_rowptr, in_col, R, depth, c, seed, threads)
    din = np.diff(np.asarray(in_rowptr, dtype=np.int64))
    D = a3.dhat_alg3(counts, R, depth, zsum, din, c)
    s = lin.reverse(n, in_rowptr, in_col, Hr, D, c)
    return QueryResult(s=s, H=Hr, pi=pi, R=R, nonmeet=counts, D=D, L=L, R_b=R_b, pair_steps=steps,
                       depth=depth, zsum=zsum)
