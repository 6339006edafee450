"""O1: Power Method ground truth and the exact diagonal correction matrix.

Test infrastructure only (see ``oracle/__init__.py``).

* ``transition_matrix`` -- the reverse transition matrix P of Sec. 2.2
  ("Linearization and ParSim"): P(i, j) = 1/din(j) for each in-neighbour i of j.
  A duplicated in-edge contributes once per copy (multiplicity weights).
* ``power_method``      -- S_{t+1} = (c P^T S_t P) v I, the element-wise maximum
  with the identity (Sec. 2.2, "Other Related Work"), from S_0 = I.  After t
  iterations the error is at most c^(t+1) (entries of S_t count walk pairs that
  meet within t steps).
* ``exact_diagonal``    -- D = S - c P^T S P (Eq. def-lsim2 summed once:
  S = D + c P^T S P), so D(k,k) = 1 - c (P^T S P)(k,k).

Pinned by: closed forms (stars, cycle, complete digraph, two parents),
brute-force rational meeting probabilities (``pair_chain``), symmetry,
unit diagonal, 0 <= S <= 1, and the D invariants of Algorithm 3 (din=0 -> 1,
din=1 -> 1-c) and Eq. def-lsim2 (1-c <= D <= 1).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def in_degrees(in_rowptr) -> np.ndarray:
    return np.diff(np.asarray(in_rowptr, dtype=np.int64))


def transition_matrix(n: int, in_rowptr, in_col) -> sp.csr_matrix:
    """Reverse transition matrix P (n x n, CSR): P[i, j] = mult(i->j) / din(j)."""
    rowptr = np.asarray(in_rowptr, dtype=np.int64)
    col = np.asarray(in_col, dtype=np.int64)
    din = in_degrees(rowptr)
    j = np.repeat(np.arange(n, dtype=np.int64), din)  # column index = target node j
    vals = 1.0 / din[j].astype(np.float64)
    # row index = in-neighbour i; duplicates are summed by the constructor
    return sp.csr_matrix((vals, (col, j)), shape=(n, n))


def power_iterations(c: float, tol: float = 1e-13) -> int:
    """Smallest t with c^(t+1) <= tol."""
    return max(1, int(math.ceil(math.log(tol) / math.log(c))) - 1)


def power_method(n: int, in_rowptr, in_col, c: float, iterations: int | None = None) -> np.ndarray:
    """All-pairs SimRank matrix S (dense FP64) by S <- max(c P^T S P, I)."""
    if n > 30000:
        raise ValueError("power_method holds an n x n matrix; n too large")
    P = transition_matrix(n, in_rowptr, in_col)
    PT = P.T.tocsr()
    t = power_iterations(c) if iterations is None else iterations
    eye = np.eye(n)
    S = eye.copy()
    for _ in range(t):
        # (P^T S) is sparse @ dense; (P^T S) P = ((P^T (P^T S)^T)^T) keeps both products sparse @ dense
        A = PT @ S              # P^T S
        M = (PT @ A.T).T        # (P^T S) P
        S = np.maximum(c * M, eye)
    return S


def exact_diagonal(n: int, in_rowptr, in_col, c: float, S: np.ndarray) -> np.ndarray:
    """D(k,k) = S(k,k) - c (P^T S P)(k,k), the diagonal of D = S - c P^T S P."""
    P = transition_matrix(n, in_rowptr, in_col)
    PT = P.T.tocsr()
    M = (PT @ (PT @ S).T).T
    return np.diag(S) - c * np.diag(M)


def simrank_column(n: int, in_rowptr, in_col, c: float, u: int) -> np.ndarray:
    """Column u of the Power Method S."""
    return power_method(n, in_rowptr, in_col, c)[:, u].copy()
