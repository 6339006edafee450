"""Brute-force meeting probabilities of two sqrt(c)-walks, in exact rational arithmetic.

Test infrastructure only (see ``oracle/__init__.py``).

Eq. scwwalk: S(i, j) is the probability that a sqrt(c)-walk from i and one from j
visit the same node at the same step, where each step moves to a uniform
in-neighbour with probability sqrt(c) and stops otherwise.  Both walks take a
step together with probability c, so for i != j

    h(i, j) = c / (din(i) din(j)) * sum_{a in I(i), b in I(j)} [a == b ? 1 : h(a, b)]

and h(i, i) = 1.  This is a linear system over the ordered pairs (i, j), i != j.
It is solved here by Gaussian elimination over ``fractions.Fraction``, so the
answer is exact.  This formulation shares nothing with ``power``'s matrix
iteration; agreement of the two pins both.

``exact_diagonal_rational`` gives D(k,k) = 1 - Pr[two walks from k meet at some
step t >= 1] (Sec. 3.2, "Local deterministic exploitation").
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _in_lists(n, in_rowptr, in_col):
    rp = [int(x) for x in in_rowptr]
    col = [int(x) for x in in_col]
    return [col[rp[j]:rp[j + 1]] for j in range(n)]


def _solve(A, b):
    """Gaussian elimination over Fractions (A square, list of lists)."""
    N = len(b)
    A = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(N):
        piv = next(r for r in range(col, N) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        for r in range(N):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return [A[i][N] for i in range(N)]


def meeting_matrix(n: int, in_rowptr, in_col, c: Fraction) -> list[list[Fraction]]:
    """Exact S(i, j) = Pr[walks from i and j meet] for all pairs (n <= 8)."""
    if n > 8:
        raise ValueError("brute force is for n <= 8")
    c = Fraction(c)
    I = _in_lists(n, in_rowptr, in_col)
    pairs = [(i, j) for i in range(n) for j in range(n) if i != j]
    idx = {p: t for t, p in enumerate(pairs)}
    N = len(pairs)
    A = [[Fraction(0)] * N for _ in range(N)]
    b = [Fraction(0)] * N
    for t, (i, j) in enumerate(pairs):
        A[t][t] += 1
        if not I[i] or not I[j]:
            continue
        w = c / (len(I[i]) * len(I[j]))
        for a in I[i]:
            for bb in I[j]:
                if a == bb:
                    b[t] += w
                else:
                    A[t][idx[(a, bb)]] -= w
    h = _solve(A, b) if N else []
    S = [[Fraction(1) if i == j else Fraction(0) for j in range(n)] for i in range(n)]
    for t, (i, j) in enumerate(pairs):
        S[i][j] = h[t]
    return S


def exact_diagonal_rational(n: int, in_rowptr, in_col, c: Fraction) -> list[Fraction]:
    """D(k,k) = 1 - Pr[two independent walks from k meet at a step t >= 1]."""
    c = Fraction(c)
    S = meeting_matrix(n, in_rowptr, in_col, c)
    I = _in_lists(n, in_rowptr, in_col)
    D = []
    for k in range(n):
        if not I[k]:
            D.append(Fraction(1))
            continue
        w = c / (len(I[k]) ** 2)
        meet = Fraction(0)
        for a in I[k]:
            for bb in I[k]:
                meet += w * (1 if a == bb else S[a][bb])
        D.append(1 - meet)
    return D


def to_float(M) -> np.ndarray:
    return np.array([[float(x) for x in row] for row in M]) if M and isinstance(M[0], list) \
        else np.array([float(x) for x in M])
