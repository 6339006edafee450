"""Seeded graph generators that stand in for the paper's datasets (Table 2).

Every generator returns ``(n, in_rowptr, in_col)``: an in-edge CSR where row ``j``
lists the in-neighbours ``I(j)`` of node ``j`` (``in_rowptr`` int64 of length n+1,
``in_col`` int32 of length m), rows sorted by source id.  That is the layout the
library's ``esim_load_graph`` takes.

Generators:

* ``erdos_renyi``  -- m distinct uniform (src, dst) pairs, self-loops dropped.
* ``chung_lu``     -- directed power-law graph: independent Pareto in- and
  out-weights w = (1-U)^(-1/(gamma-1)), endpoints drawn proportionally to the
  weights, self-loops dropped, duplicates removed, redrawn to exactly m edges.
* ``rmat``         -- recursive-matrix graph with quadrant probabilities
  (a, b, c, d), duplicates and loops removed, seeded random vertex permutation;
  ``rmat_torch`` draws the same kind of graph with torch on a GPU for the
  largest sizes.
* ``chung_lu_torch`` -- the Chung-Lu recipe with torch on a GPU (the n = 4e6 graph
  of the precision form, generated in seconds).

Small named graphs (stars, cycle, complete digraph, ...) serve the closed-form
checks.  Nothing here computes any part of SimRank.
"""
from __future__ import annotations

import numpy as np


def edges_to_in_csr(n: int, src: np.ndarray, dst: np.ndarray):
    """Build the in-edge CSR (row = destination, entries = sources) of an edge list.

    Duplicate edges are kept (they count with multiplicity); rows are sorted by
    source id so the layout is deterministic.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.size:
        if src.min() < 0 or src.max() >= n or dst.min() < 0 or dst.max() >= n:
            raise ValueError("edge endpoint out of range")
    order = np.lexsort((src, dst))
    src = src[order]
    dst = dst[order]
    counts = np.bincount(dst, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return n, rowptr, src.astype(np.int32)


def _dedupe_keys(keys: np.ndarray) -> np.ndarray:
    return np.unique(keys)


def _fill_distinct(n: int, m: int, draw, rng, max_rounds: int = 200):
    """Draw candidate (src, dst) batches until exactly m distinct non-loop edges exist.

    ``draw(rng, k)`` returns two int64 arrays of k endpoints.  The first m distinct
    edges in draw order are kept, so the result depends only on the seed.
    """
    if m > n * (n - 1):
        raise ValueError("m exceeds the number of possible directed edges")
    keys = np.empty(0, dtype=np.int64)
    need = m
    for _ in range(max_rounds):
        k = int(need * 1.10) + 64
        s, d = draw(rng, k)
        keep = s != d
        new = s[keep] * n + d[keep]
        # keep first occurrence order: unique over (old + new) preserving the old set
        _, first = np.unique(new, return_index=True)
        new = new[np.sort(first)]
        if keys.size:
            new = new[~np.isin(new, keys, assume_unique=False)]
        take = min(need, new.size)
        keys = np.concatenate([keys, new[:take]])
        need = m - keys.size
        if need == 0:
            break
    if need != 0:
        raise RuntimeError("could not reach the requested number of distinct edges")
    return keys // n, keys % n


def erdos_renyi(n: int, m: int, seed: int = 1):
    """Directed Erdos-Renyi graph: m distinct uniform pairs, self-loops dropped."""
    rng = np.random.default_rng(seed)

    def draw(r, k):
        return r.integers(0, n, size=k, dtype=np.int64), r.integers(0, n, size=k, dtype=np.int64)

    s, d = _fill_distinct(n, m, draw, rng)
    return edges_to_in_csr(n, s, d)


def _pareto_weights(rng, n: int, gamma: float) -> np.ndarray:
    u = rng.random(n)
    return (1.0 - u) ** (-1.0 / (gamma - 1.0))


def chung_lu(n: int, m: int, gamma: float = 2.1, seed: int = 1):
    """Directed Chung-Lu power-law graph with independent in/out Pareto weights."""
    rng = np.random.default_rng(seed)
    w_out = _pareto_weights(rng, n, gamma)
    w_in = _pareto_weights(rng, n, gamma)
    c_out = np.cumsum(w_out)
    c_in = np.cumsum(w_in)
    c_out /= c_out[-1]
    c_in /= c_in[-1]

    def draw(r, k):
        s = np.searchsorted(c_out, r.random(k), side="right")
        d = np.searchsorted(c_in, r.random(k), side="right")
        return np.minimum(s, n - 1).astype(np.int64), np.minimum(d, n - 1).astype(np.int64)

    s, d = _fill_distinct(n, m, draw, rng)
    return edges_to_in_csr(n, s, d)


def rmat(scale: int, m: int, a=0.57, b=0.19, c=0.19, d=0.05, seed: int = 1):
    """R-MAT graph on n = 2**scale nodes with exactly m distinct non-loop edges."""
    n = 1 << scale
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    p = np.array([a, b, c, d], dtype=np.float64)
    p = np.cumsum(p / p.sum())

    def draw(r, k):
        s = np.zeros(k, dtype=np.int64)
        t = np.zeros(k, dtype=np.int64)
        for _ in range(scale):
            q = np.searchsorted(p, r.random(k), side="right")
            s = (s << 1) | (q >> 1)
            t = (t << 1) | (q & 1)
        return perm[s], perm[t]

    s, t = _fill_distinct(n, m, draw, rng)
    return edges_to_in_csr(n, s, t)


def rmat_torch(scale: int, m: int, a=0.57, b=0.19, c=0.19, d=0.05, seed: int = 1, device: str = "cuda"):
    """R-MAT graph generated with torch on `device` (for the largest configurations).

    Same recipe as ``rmat`` (quadrant probabilities, loops and duplicates removed,
    seeded vertex permutation, exactly m distinct edges) with torch's generator:
    it is deterministic for a given seed, device type and torch version, but it
    draws a different graph than the NumPy ``rmat``.  Surplus edges are drawn,
    deduplicated, and m of them are kept by a seeded permutation.
    """
    import torch
    n = 1 << scale
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    perm = torch.randperm(n, generator=gen, device=device)
    t0, t1, t2 = a, a + b, a + b + c
    keys = torch.empty(0, dtype=torch.int64, device=device)
    draw = int(m * 1.3) + 4096
    for _ in range(20):
        chunk = 1 << 26
        parts = []
        left = draw
        while left > 0:
            k = min(chunk, left)
            left -= k
            src = torch.zeros(k, dtype=torch.int64, device=device)
            dst = torch.zeros(k, dtype=torch.int64, device=device)
            for _lvl in range(scale):
                r = torch.rand(k, generator=gen, device=device)
                q = (r >= t0).long() + (r >= t1).long() + (r >= t2).long()
                src = (src << 1) | (q >> 1)
                dst = (dst << 1) | (q & 1)
            keep = src != dst
            parts.append(perm[src[keep]] * n + perm[dst[keep]])
            del src, dst, keep
        keys = torch.unique(torch.cat([keys] + parts))
        del parts
        if keys.numel() >= m:
            break
        draw = int((m - keys.numel()) * 2) + 4096
    if keys.numel() < m:
        raise RuntimeError("could not reach the requested number of distinct edges")
    pick = torch.randperm(keys.numel(), generator=gen, device=device)[:m]
    keys = keys[pick]
    src = keys // n
    dst = keys % n
    del keys, pick
    order = torch.argsort(dst * n + src)
    src = src[order]
    dst = dst[order]
    counts = torch.bincount(dst, minlength=n)
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(counts, 0)
    return n, rowptr.cpu().numpy(), src.to(torch.int32).cpu().numpy()


def chung_lu_torch(n: int, m: int, gamma: float = 2.2, seed: int = 1, device: str = "cuda"):
    """Directed Chung-Lu graph generated with torch on `device` (for the largest sizes).

    Same recipe as ``chung_lu`` (independent Pareto in- and out-weights
    w = (1-U)^(-1/(gamma-1)), endpoints drawn proportionally to the weights, loops and
    duplicates removed, exactly m distinct edges) with torch's generator: deterministic
    for a given seed, device type and torch version, but a different graph than the
    NumPy ``chung_lu``.  Surplus edges are drawn, deduplicated, and m of them are kept by
    a seeded permutation.
    """
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)

    def cdf():
        u = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
        w = (1.0 - u) ** (-1.0 / (gamma - 1.0))
        c = torch.cumsum(w, 0)
        return c / c[-1]

    c_out = cdf()
    c_in = cdf()
    keys = torch.empty(0, dtype=torch.int64, device=device)
    draw = int(m * 1.25) + 4096
    for _ in range(20):
        chunk = 1 << 26
        parts = []
        left = draw
        while left > 0:
            k = min(chunk, left)
            left -= k
            src = torch.searchsorted(c_out, torch.rand(k, generator=gen, device=device, dtype=torch.float64),
                                     right=True).clamp_(max=n - 1)
            dst = torch.searchsorted(c_in, torch.rand(k, generator=gen, device=device, dtype=torch.float64),
                                     right=True).clamp_(max=n - 1)
            keep = src != dst
            parts.append(src[keep] * n + dst[keep])
            del src, dst, keep
        keys = torch.unique(torch.cat([keys] + parts))
        del parts
        if keys.numel() >= m:
            break
        draw = int((m - keys.numel()) * 2) + 4096
    if keys.numel() < m:
        raise RuntimeError("could not reach the requested number of distinct edges")
    pick = torch.randperm(keys.numel(), generator=gen, device=device)[:m]
    keys = keys[pick]
    src = keys // n
    dst = keys % n
    del keys, pick
    order = torch.argsort(dst * n + src)
    src = src[order]
    dst = dst[order]
    counts = torch.bincount(dst, minlength=n)
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(counts, 0)
    return n, rowptr.cpu().numpy(), src.to(torch.int32).cpu().numpy()


def random_sources(in_rowptr: np.ndarray, count: int, seed: int = 7) -> np.ndarray:
    """Uniform source nodes among nodes with in-degree >= 1 (redrawn otherwise)."""
    rng = np.random.default_rng(seed)
    din = np.diff(np.asarray(in_rowptr))
    n = din.size
    if not np.any(din > 0):
        raise ValueError("graph has no node with an in-edge")
    out = []
    while len(out) < count:
        v = int(rng.integers(0, n))
        if din[v] > 0:
            out.append(v)
    return np.array(out, dtype=np.int64)


def uniform_diagonal(n: int, c: float, seed: int = 11) -> np.ndarray:
    """Seeded diagonal values uniform in [1-c, 1] (the range of D(k,k))."""
    rng = np.random.default_rng(seed)
    return (1.0 - c) + c * rng.random(n)


# ---------------------------------------------------------------- small named graphs

def out_star(leaves: int):
    """Centre 0 with edges 0 -> 1..leaves."""
    src = np.zeros(leaves, dtype=np.int64)
    dst = np.arange(1, leaves + 1, dtype=np.int64)
    return edges_to_in_csr(leaves + 1, src, dst)


def in_star(leaves: int):
    """Leaves 1..leaves with edges leaf -> 0."""
    src = np.arange(1, leaves + 1, dtype=np.int64)
    dst = np.zeros(leaves, dtype=np.int64)
    return edges_to_in_csr(leaves + 1, src, dst)


def directed_cycle(n: int):
    """Edges i -> (i+1) mod n."""
    src = np.arange(n, dtype=np.int64)
    return edges_to_in_csr(n, src, (src + 1) % n)


def complete_digraph(n: int):
    """All n(n-1) directed edges."""
    s, d = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = s != d
    return edges_to_in_csr(n, s[keep], d[keep])


def two_parents():
    """Nodes a=0, b=1 each point to x=2 and y=3."""
    src = np.array([0, 0, 1, 1])
    dst = np.array([2, 3, 2, 3])
    return edges_to_in_csr(4, src, dst)


def random_small(n: int, p: float = 0.35, seed: int = 3, loops: bool = False):
    """Small random digraph (Bernoulli(p) per ordered pair)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < p
    if not loops:
        np.fill_diagonal(mask, False)
    s, d = np.nonzero(mask)
    return edges_to_in_csr(n, s, d)


def with_dangling(n: int, m: int, dangling_frac: float = 0.2, seed: int = 5):
    """Erdos-Renyi-like graph in which a fraction of nodes has no in-edges."""
    rng = np.random.default_rng(seed)
    k = max(1, int(n * dangling_frac))
    dangling = rng.choice(n, size=k, replace=False)
    alive = np.setdiff1d(np.arange(n), dangling)

    def draw(r, cnt):
        return r.integers(0, n, size=cnt, dtype=np.int64), alive[r.integers(0, alive.size, size=cnt)]

    s, d = _fill_distinct(n, min(m, alive.size * (n - 1)), draw, rng)
    return edges_to_in_csr(n, s, d)
