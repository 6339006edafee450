"""GB300-native ExactSim single-source SimRank (arXiv:2004.03493).

The computation lives in the CUDA library ``_lib/libexactsim.so`` (C ABI in
``include/exactsim.h``); this package is its Python binding.  ``Graph`` wraps a
graph handle; the ``esim_*`` functions mirror the C entry points one to one.
There is no CPU fallback: without the library or a CUDA device every call
raises.
"""
from __future__ import annotations

import numpy as np

from . import _native
from ._native import (  # noqa: F401
    EsimError,
    esim_allocate,
    esim_alg3_first_meeting,
    esim_alg3_paper_depth,
    esim_alg3_zsum,
    esim_sample_depth,
    esim_dhat_alg3,
    esim_dhat,
    esim_forward,
    esim_forward_f32,
    esim_allocate_f32,
    esim_reverse_f32,
    esim_free_graph,
    esim_get_option,
    esim_last_error,
    esim_last_stats,
    esim_levels,
    esim_load_graph,
    esim_num_edges,
    esim_num_nodes,
    esim_query,
    esim_query_batch,
    esim_query_batch_device,
    esim_topk_batch,
    esim_topk_batch_device,
    esim_query_device,
    esim_reverse,
    esim_sample,
    esim_sample_base,
    esim_select_topk,
    esim_select_topk_static,
    esim_set_option,
    esim_set_stream,
    esim_server_create,
    esim_server_destroy,
    esim_server_get_stats,
    esim_server_poll,
    esim_server_submit,
    esim_server_wait,
    esim_sync,
    esim_topk,
    esim_topk_device,
    esim_version,
    esim_walk_threshold,
)


class Graph:
    """A graph resident on the current CUDA device (in-edge CSR input)."""

    def __init__(self, n: int, in_rowptr, in_col, **options):
        self.n = int(n)
        self.handle = esim_load_graph(self.n, in_rowptr, in_col)
        self.m = esim_num_edges(self.handle)
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if getattr(self, "handle", None):
            esim_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, key: str, value: float):
        esim_set_option(self.handle, key, value)

    def get_option(self, key: str) -> float:
        return esim_get_option(self.handle, key)

    def set_stream(self, stream):
        """Use a torch.cuda.Stream (or a raw cudaStream_t int, or None)."""
        ptr = getattr(stream, "cuda_stream", stream)
        esim_set_stream(self.handle, ptr)

    def query(self, u: int, c: float, eps: float, seed: int = 0) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        esim_query(self.handle, u, c, eps, seed, out)
        return out

    def query_device(self, u: int, c: float, eps: float, seed: int, out):
        esim_query_device(self.handle, u, c, eps, seed, out)
        return out

    def topk(self, u: int, c: float, eps: float, k: int, seed: int = 0):
        ids = np.empty(k, dtype=np.int32)
        vals = np.empty(k, dtype=np.float64)
        esim_topk(self.handle, u, c, eps, seed, k, ids, vals)
        return ids, vals

    def topk_device(self, u: int, c: float, eps: float, k: int, seed: int, ids_out, vals_out):
        esim_topk_device(self.handle, u, c, eps, seed, k, ids_out, vals_out)
        return ids_out, vals_out

    def query_batch(self, u, eps, c: float, seed: int = 0) -> np.ndarray:
        """Scores of a batch of sources, shape (B, n)."""
        u = np.asarray(u, dtype=np.int64)
        out = np.empty((u.size, self.n), dtype=np.float64)
        esim_query_batch(self.handle, u, eps, seed, c, out)
        return out

    def query_batch_device(self, u, eps, c: float, seed: int, out):
        esim_query_batch_device(self.handle, u, eps, seed, c, out)
        return out

    def topk_batch(self, u, eps, c: float, k: int, seed: int = 0):
        u = np.asarray(u, dtype=np.int64)
        ids = np.empty((u.size, k), dtype=np.int32)
        vals = np.empty((u.size, k), dtype=np.float64)
        esim_topk_batch(self.handle, u, eps, seed, c, k, ids, vals)
        return ids, vals

    def topk_batch_device(self, u, eps, c: float, k: int, seed: int, ids_out, vals_out):
        esim_topk_batch_device(self.handle, u, eps, seed, c, k, ids_out, vals_out)
        return ids_out, vals_out

    def stats(self) -> dict:
        return esim_last_stats(self.handle)

    # steps (device tensors)
    def forward(self, u, c, L, hist):
        esim_forward(self.handle, u, c, L, hist)

    def allocate(self, hist, L, R_b, mode, pi_out, R_out, off):
        esim_allocate(self.handle, hist, L, R_b, mode, pi_out, R_out, off)

    def sample(self, off, c, seed, nonmeet, pair_steps=None):
        esim_sample(self.handle, off, c, seed, nonmeet, pair_steps)

    def forward_f32(self, u, c, L, hist):
        esim_forward_f32(self.handle, u, c, L, hist)

    def allocate_f32(self, hist, L, R_b, mode, pi_out, R_out, off):
        esim_allocate_f32(self.handle, hist, L, R_b, mode, pi_out, R_out, off)

    def reverse_f32(self, hist, L, c, dhat, s_out):
        esim_reverse_f32(self.handle, hist, L, c, dhat, s_out)

    def alg3_first_meeting(self, k, depth, c):
        return esim_alg3_first_meeting(self.handle, k, depth, c)

    def alg3_paper_depth(self, R, c, max_depth, depth):
        esim_alg3_paper_depth(self.handle, R, c, max_depth, depth)

    def alg3_zsum(self, depth, c, zsum):
        esim_alg3_zsum(self.handle, depth, c, zsum)

    def sample_depth(self, off, depth, c, seed, counts, pair_steps=None):
        esim_sample_depth(self.handle, off, depth, c, seed, counts, pair_steps)

    def dhat_alg3(self, counts, off, depth, zsum, c, out):
        esim_dhat_alg3(self.handle, counts, off, depth, zsum, c, out)

    def dhat(self, nonmeet, off, out):
        esim_dhat(self.handle, nonmeet, off, out)

    def reverse(self, hist, L, c, dhat, s_out):
        esim_reverse(self.handle, hist, L, c, dhat, s_out)

    def select_topk(self, scores, exclude, k, ids_out, vals_out):
        esim_select_topk(self.handle, scores, exclude, k, ids_out, vals_out)

    def sync(self):
        esim_sync(self.handle)


class Server:
    """Continuous-batching request loop over a loaded Graph (top-k queries)."""

    def __init__(self, graph: Graph, c: float, k: int, seed: int = 0, kappa: float = 0.0, max_batch: int = 64,
                 max_waves: int = 2, mem_budget_bytes: float = 0.0):
        self.graph = graph
        self.k = int(k)
        self.handle = esim_server_create(graph.handle, c, k, seed, kappa, max_batch, max_waves, mem_budget_bytes)

    def submit(self, u: int, eps: float) -> int:
        return esim_server_submit(self.handle, int(u), float(eps))

    def poll(self, rid: int) -> int:
        return esim_server_poll(self.handle, rid)

    def wait(self, rid: int, timeout_ms: int = 60000):
        ids = np.empty(self.k, dtype=np.int32)
        vals = np.empty(self.k, dtype=np.float64)
        lat = esim_server_wait(self.handle, rid, timeout_ms, ids, vals)
        return ids, vals, lat

    def stats(self) -> dict:
        return esim_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            esim_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(force: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force)
