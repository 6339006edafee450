"""O2: the deterministic steps of Algorithm 1 (Basic ExactSim), written plainly in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Notation follows Sec. 3.1: a = 1 - sqrt(c); P is the reverse transition matrix
(``power.transition_matrix``).

* ``levels``          -- L = ceil(log_{1/c}(2/eps))                (Algorithm 1, depth)
* ``hop_vectors``     -- pi^0 = a e_u, pi^l = sqrt(c) P pi^{l-1}    (Algorithm 1, forward loop;
                         the definition pi^l = (1-sqrt(c)) (sqrt(c) P)^l e_u of Sec. 2.2, PRSim)
* ``ppr``             -- pi = sum_{l=0..L} pi^l                    (Algorithm 1, forward loop)
* ``sample_base``     -- R_b = kappa ln(n) / eps^2, kappa = 6 / a^4 by default
                         (Algorithm 1, sample count; natural log, since the bound comes
                         from the exponential of the Bernstein inequality)
* ``allocate``        -- R(k) = ceil(R_b pi(k)^2) (the pi^2 scheme of Lemma 4 with R
                         scaled by ||pi||^2, as in the proof of Lemma 4), or
                         R(k) = ceil(R_b pi(k)) (Algorithm 1, "basic" allocation);
                         at least 1 wherever pi(k) > 0
* ``dhat``            -- D^(k) = nonmeet(k) / R(k)                  (Algorithm 2)
* ``reverse``         -- s^0 = D^ pi^L / a; s^l = sqrt(c) P^T s^{l-1} + D^ pi^{L-l} / a
                         (Algorithm 1, reverse loop; Eq. sL)
* ``bilinear``        -- s(j) = (1/a^2) sum_l sum_k pi_u^l(k) pi_j^l(k) D(k)
                         (Eq. formula-ppr in the proof of Theorem 1); an independent
                         evaluation of the same sum used to pin ``reverse``
* ``topk``            -- k nodes with the largest scores (Sec. 1), order (score desc,
                         id asc), source excluded unless asked
* ``sparse_threshold``/``sparsify`` -- sparse Linearization (Sec. 3.2): the stored
                         pi^l keep only entries above (1 - sqrt(c))^2 eps; the sparse-
                         linearization lemma bounds the extra error by eps

Floating-point decisions that pick integers (L, R(k)) are made with the exact
operation order the library documents, so both sides take them in FP64.
"""
from __future__ import annotations

import math

import numpy as np

from .power import transition_matrix, in_degrees


def sqrt_c(c: float) -> float:
    return math.sqrt(c)


def levels(c: float, eps: float) -> int:
    """L = ceil(log(2/eps) / log(1/c))."""
    return int(math.ceil(math.log(2.0 / eps) / math.log(1.0 / c)))


def kappa_paper(c: float) -> float:
    """6 / (1 - sqrt(c))^4, the constant of Algorithm 1's sample count R."""
    a = 1.0 - math.sqrt(c)
    return 6.0 / (a * a * a * a)


def sample_base(n: int, c: float, eps: float, kappa: float | None = None) -> float:
    """R_b = kappa * ln(n) / (eps * eps)."""
    if kappa is None or kappa <= 0.0:
        kappa = kappa_paper(c)
    return kappa * math.log(float(n)) / (eps * eps)


def hop_vectors(n: int, in_rowptr, in_col, u: int, c: float, L: int) -> np.ndarray:
    """History H[l] = pi_u^l for l = 0..L (shape (L+1, n))."""
    P = transition_matrix(n, in_rowptr, in_col)
    a = 1.0 - math.sqrt(c)
    H = np.zeros((L + 1, n))
    H[0, u] = a
    for ell in range(1, L + 1):
        H[ell] = math.sqrt(c) * (P @ H[ell - 1])
    return H


def ppr(H: np.ndarray) -> np.ndarray:
    """pi(k) = sum over levels of pi^l(k), summed in level order."""
    pi = np.zeros(H.shape[1])
    for ell in range(H.shape[0]):
        pi = pi + H[ell]
    return pi


def allocate(pi: np.ndarray, R_b: float, mode: str = "pi2") -> np.ndarray:
    """Per-node pair counts R(k) (uint64); every node with pi(k) > 0 gets at least one.

    pi2:   R(k) = max(1, ceil(R_b * (pi(k) * pi(k))))   for pi(k) > 0
    basic: R(k) = max(1, ceil(R_b * pi(k)))             for pi(k) > 0
    R(k) = 0 where pi(k) = 0.  The ceiling of a positive number is already >= 1;
    the floor of one only matters when R_b * pi(k)^2 underflows or R_b = 0 (n = 1).
    """
    pi = np.asarray(pi, dtype=np.float64)
    if mode == "pi2":
        v = R_b * (pi * pi)
    elif mode == "basic":
        v = R_b * pi
    else:
        raise ValueError(mode)
    R = np.ceil(v).astype(np.uint64)
    R[(pi > 0) & (R == 0)] = 1
    return R


def dhat(nonmeet: np.ndarray, R: np.ndarray) -> np.ndarray:
    """D^(k) = nonmeet(k) / R(k); nodes with R(k) = 0 get 0 (their pi is 0)."""
    R = np.asarray(R, dtype=np.uint64)
    out = np.zeros(R.size)
    nz = R > 0
    out[nz] = np.asarray(nonmeet, dtype=np.uint64)[nz].astype(np.float64) / R[nz].astype(np.float64)
    return out


def reverse(n: int, in_rowptr, in_col, H: np.ndarray, D: np.ndarray, c: float) -> np.ndarray:
    """s^L of Algorithm 1's reverse loop (Eq. sL)."""
    P = transition_matrix(n, in_rowptr, in_col)
    PT = P.T.tocsr()
    a = 1.0 - math.sqrt(c)
    L = H.shape[0] - 1
    s = D * H[L] / a
    for ell in range(1, L + 1):
        s = math.sqrt(c) * (PT @ s) + D * H[L - ell] / a
    return s


def bilinear(Hu: np.ndarray, Hj: np.ndarray, D: np.ndarray, c: float) -> float:
    """(1/a^2) sum_l sum_k pi_u^l(k) pi_j^l(k) D(k)."""
    a = 1.0 - math.sqrt(c)
    return float(np.sum(Hu * Hj * D[None, :]) / (a * a))


def topk(scores: np.ndarray, k: int, exclude: int | None = None):
    """Ids and scores of the k largest scores, ordered (score desc, id asc)."""
    scores = np.asarray(scores, dtype=np.float64)
    ids = np.arange(scores.size)
    if exclude is not None and 0 <= exclude < scores.size:
        keep = ids != exclude
        ids = ids[keep]
        vals = scores[keep]
    else:
        vals = scores
    order = np.lexsort((ids, -vals))[:k]
    return ids[order].astype(np.int32), vals[order]


def pair_threshold(c: float) -> int:
    """Walk continuation threshold T = floor(sqrt(c) * 2^32) (uint32)."""
    return min(int(math.floor(math.sqrt(c) * 4294967296.0)), 0xFFFFFFFF)


__all__ = [
    "levels", "kappa_paper", "sample_base", "hop_vectors", "ppr", "allocate", "dhat",
    "reverse", "bilinear", "topk", "pair_threshold", "in_degrees",
]


def sparse_threshold(c: float, eps: float) -> float:
    """theta = (1 - sqrt(c))^2 eps: history entries at or below it are dropped (Sec. 3.2)."""
    a = 1.0 - math.sqrt(c)
    return a * a * eps


def sparsify(H: np.ndarray, theta: float) -> np.ndarray:
    """The stored history of sparse Linearization: pi^l(k) if pi^l(k) > theta, else 0."""
    return np.where(H > theta, H, 0.0)
