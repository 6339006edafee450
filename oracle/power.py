"""O1: Power Method ground truth and the exact diagonal correction matrix.

Test infrastructure only (see ``oracle/__init__.py``).

* ``transition_matrix`` -- the reverse transition matrix P of Sec. 2.2
  ("Linearization and ParSim"): P(i, j) = 1/din(j) for each in-neighbour i of j.
  A duplicated in-edge contributes once per copy (multiplicity weights).
* ``power_method``      -- S_{t+1} = (c P^T S_t P) v I, the element-wise maximum
  with the identity (Sec. 2.2, "Other Related Work"), from S_0 = I.  After t
  iterations the error is at most c^(t+1) (entries of S_t count walk pairs that
  meet within t steps).
* ``power_method_c``    -- the same iteration in C with OpenMP (``power.c``), for the
  graphs of a few 10^4 nodes that the exceed-rate test needs.
* ``exact_diagonal``    -- D = S - c P^T S P (Eq. def-lsim2 summed once:
  S = D + c P^T S P), so D(k,k) = 1 - c (P^T S P)(k,k).

Pinned by (both implementations): closed forms (stars, cycle, complete digraph, two parents),
brute-force rational meeting probabilities (``pair_chain``), symmetry,
unit diagonal, 0 <= S <= 1, and the D invariants of Algorithm 3 (din=0 -> 1,
din=1 -> 1-c) and Eq. def-lsim2 (1-c <= D <= 1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

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


_C_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "power.c")
_C_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liboracle_power.so")
_c_lib = None


def build_c(force: bool = False) -> str:
    """Compile power.c (gcc -O2 -fopenmp) if the shared object is missing or stale."""
    os.makedirs(os.path.dirname(_C_LIB), exist_ok=True)
    if force or not os.path.exists(_C_LIB) or os.path.getmtime(_C_LIB) < os.path.getmtime(_C_SRC):
        tmp = _C_LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _C_SRC], check=True)
        os.replace(tmp, _C_LIB)
    return _C_LIB


def power_method_c(n: int, in_rowptr, in_col, c: float, iterations: int | None = None) -> np.ndarray:
    """All-pairs S by the C Power Method (power.c), FP64, OpenMP."""
    global _c_lib
    if _c_lib is None:
        build_c()
        lib = ctypes.CDLL(_C_LIB)
        lib.oracle_power_method.restype = ctypes.c_int
        lib.oracle_power_method.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                            ctypes.c_int32, ctypes.c_void_p]
        _c_lib = lib
    rp = np.ascontiguousarray(in_rowptr, dtype=np.int64)
    col = np.ascontiguousarray(in_col, dtype=np.int32)
    if rp.size != n + 1:
        raise ValueError("shape mismatch")
    t = power_iterations(c) if iterations is None else iterations
    S = np.empty((n, n))
    st = _c_lib.oracle_power_method(n, rp.ctypes.data, col.ctypes.data, float(c), int(t), S.ctypes.data)
    if st != 0:
        raise RuntimeError(f"oracle_power_method failed ({st})")
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
