"""ctypes binding of the C ABI in ``include/exactsim.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls.  Pointers are
taken from NumPy arrays (host memory) or from CUDA tensors (device memory); the
binding checks dtype, device and contiguity and passes the raw address.  All
computation happens in the CUDA library; if it is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libexactsim.so")

ESIM_OK = 0
STATUS_NAMES = {0: "ESIM_OK", -1: "ESIM_EINVAL", -2: "ESIM_ENOMEM", -3: "ESIM_ECUDA", -4: "ESIM_ETIMEOUT",
                -5: "ESIM_EBUDGET", -6: "ESIM_ENOTSUP"}


class EsimError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class QueryStats(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("launches", ctypes.c_int32), ("R_b", ctypes.c_double),
                ("kappa", ctypes.c_double), ("pi_norm2", ctypes.c_double), ("sum_R", ctypes.c_uint64),
                ("pair_steps", ctypes.c_uint64), ("ms_forward", ctypes.c_float), ("ms_allocate", ctypes.c_float),
                ("ms_sample", ctypes.c_float), ("ms_reverse", ctypes.c_float), ("ms_topk", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("alg3_nodes", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("hist_entries", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64),
                ("ms_sample_kernel", ctypes.c_float), ("ms_sample_side", ctypes.c_float),
                ("pair_steps_side", ctypes.c_uint64), ("side_candidates", ctypes.c_int32),
                ("reserved3", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved2"}


class ServerConfig(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("kappa", ctypes.c_double), ("seed", ctypes.c_uint64), ("k", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_waves", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("waves", ctypes.c_uint64),
                ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("max_running", ctypes.c_int32), ("queued", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I32, _I64, _U64, _U32, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
_ST = ctypes.c_int

# name: (restype, argtypes) -- mirrors include/exactsim.h
SIGNATURES = {
    "esim_version": (ctypes.c_char_p, []),
    "esim_last_error": (ctypes.c_char_p, []),
    "esim_levels": (_I32, [_D, _D]),
    "esim_sample_base": (_D, [_I64, _D, _D, _D]),
    "esim_walk_threshold": (_U32, [_D]),
    "esim_load_graph": (_ST, [_I64, _P, _P, ctypes.POINTER(_P)]),
    "esim_free_graph": (None, [_P]),
    "esim_num_nodes": (_I64, [_P]),
    "esim_num_edges": (_I64, [_P]),
    "esim_set_stream": (_ST, [_P, _P]),
    "esim_set_option": (_ST, [_P, ctypes.c_char_p, _D]),
    "esim_get_option": (_ST, [_P, ctypes.c_char_p, ctypes.POINTER(_D)]),
    "esim_query": (_ST, [_P, _I64, _D, _D, _U64, _P]),
    "esim_query_device": (_ST, [_P, _I64, _D, _D, _U64, _P]),
    "esim_topk": (_ST, [_P, _I64, _D, _D, _U64, _I32, _P, _P]),
    "esim_topk_device": (_ST, [_P, _I64, _D, _D, _U64, _I32, _P, _P]),
    "esim_last_stats": (_ST, [_P, ctypes.POINTER(QueryStats)]),
    "esim_forward": (_ST, [_P, _I64, _D, _I32, _P]),
    "esim_allocate": (_ST, [_P, _P, _I32, _D, _I32, _P, _P, _P]),
    "esim_sample": (_ST, [_P, _P, _D, _U64, _P, _P]),
    "esim_dhat": (_ST, [_P, _P, _P, _P]),
    "esim_reverse": (_ST, [_P, _P, _I32, _D, _P, _P]),
    "esim_select_topk": (_ST, [_P, _P, _I64, _I32, _P, _P]),
    "esim_sync": (_ST, [_P]),
    "esim_select_topk_static": (_ST, [_P, _I64, _I64, _I32, _P, _P, _P]),
    "esim_forward_f32": (_ST, [_P, _I64, _D, _I32, _P]),
    "esim_allocate_f32": (_ST, [_P, _P, _I32, _D, _I32, _P, _P, _P]),
    "esim_reverse_f32": (_ST, [_P, _P, _I32, _D, _P, _P]),
    "esim_query_batch": (_ST, [_P, _I32, _P, _P, _U64, _D, _P]),
    "esim_query_batch_device": (_ST, [_P, _I32, _P, _P, _U64, _D, _P]),
    "esim_topk_batch": (_ST, [_P, _I32, _P, _P, _U64, _D, _I32, _P, _P]),
    "esim_topk_batch_device": (_ST, [_P, _I32, _P, _P, _U64, _D, _I32, _P, _P]),
    "esim_server_create": (_ST, [_P, ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    "esim_server_submit": (_ST, [_P, _I64, _D, ctypes.POINTER(_U64)]),
    "esim_server_poll": (_ST, [_P, _U64, ctypes.POINTER(_I32)]),
    "esim_server_wait": (_ST, [_P, _U64, _I32, _P, _P, ctypes.POINTER(_D)]),
    "esim_server_get_stats": (_ST, [_P, ctypes.POINTER(ServerStats)]),
    "esim_server_destroy": (None, [_P]),
    "esim_alg3_first_meeting": (_ST, [_P, _I64, _I32, _D, _P]),
    "esim_alg3_depth": (_I32, [_D, _D, _P, _I32, _I64, _I64, _D, _D, _D, _D]),
    "esim_alg3_paper_depth": (_ST, [_P, _P, _D, _I32, _P]),
    "esim_alg3_zsum": (_ST, [_P, _P, _D, _P]),
    "esim_sample_depth": (_ST, [_P, _P, _P, _D, _U64, _P, _P]),
    "esim_dhat_alg3": (_ST, [_P, _P, _P, _P, _P, _D, _P]),
}


def lib():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(the library has no CPU fallback)")
            h = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def _check(status: int):
    if status != ESIM_OK:
        raise EsimError(status, lib().esim_last_error().decode(errors="replace"))


def _ptr(x, dtype_name: str | None = None, device: bool | None = None, allow_none: bool = False):
    """Address of a NumPy array (host) or a torch tensor (device or host)."""
    if x is None:
        if allow_none:
            return None
        raise ValueError("missing buffer")
    if isinstance(x, np.ndarray):
        if device:
            raise ValueError("expected a device tensor, got a NumPy array")
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if dtype_name and x.dtype != np.dtype(dtype_name):
            raise ValueError(f"expected dtype {dtype_name}, got {x.dtype}")
        return x.ctypes.data
    # torch tensor
    if device is True and not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if device is False and x.is_cuda:
        raise ValueError("expected a host buffer")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype_name:
        tname = str(x.dtype).replace("torch.", "")
        if tname != dtype_name:
            raise ValueError(f"expected dtype {dtype_name}, got {tname}")
    return x.data_ptr()


# ------------------------------------------------------------------ library


def esim_version() -> str:
    return lib().esim_version().decode()


def esim_last_error() -> str:
    return lib().esim_last_error().decode(errors="replace")


def esim_levels(c: float, eps: float) -> int:
    return int(lib().esim_levels(c, eps))


def esim_sample_base(n: int, c: float, eps: float, kappa: float = 0.0) -> float:
    return float(lib().esim_sample_base(n, c, eps, kappa))


def esim_walk_threshold(c: float) -> int:
    return int(lib().esim_walk_threshold(c))


# ------------------------------------------------------------------ graph


def esim_load_graph(n: int, in_rowptr: np.ndarray, in_col: np.ndarray) -> int:
    rp = np.ascontiguousarray(in_rowptr, dtype=np.int64)
    col = np.ascontiguousarray(in_col, dtype=np.int32)
    if rp.size != n + 1:
        raise ValueError("in_rowptr must have n+1 entries")
    out = _P()
    _check(lib().esim_load_graph(n, rp.ctypes.data, col.ctypes.data if col.size else None, ctypes.byref(out)))
    return out.value


def esim_free_graph(g: int) -> None:
    lib().esim_free_graph(g)


def esim_num_nodes(g: int) -> int:
    return int(lib().esim_num_nodes(g))


def esim_num_edges(g: int) -> int:
    return int(lib().esim_num_edges(g))


def esim_set_stream(g: int, stream: int | None) -> None:
    _check(lib().esim_set_stream(g, stream))


def esim_set_option(g: int, key: str, value: float) -> None:
    _check(lib().esim_set_option(g, key.encode(), float(value)))


def esim_get_option(g: int, key: str) -> float:
    v = _D()
    _check(lib().esim_get_option(g, key.encode(), ctypes.byref(v)))
    return v.value


# ------------------------------------------------------------------ queries


def esim_query(g: int, u: int, c: float, eps: float, seed: int, s_out: np.ndarray) -> None:
    _check(lib().esim_query(g, u, c, eps, seed, _ptr(s_out, "float64", device=False)))


def esim_query_device(g: int, u: int, c: float, eps: float, seed: int, s_dev) -> None:
    _check(lib().esim_query_device(g, u, c, eps, seed, _ptr(s_dev, "float64", device=True)))


def esim_topk(g: int, u: int, c: float, eps: float, seed: int, k: int, ids_out: np.ndarray,
              scores_out: np.ndarray) -> None:
    _check(lib().esim_topk(g, u, c, eps, seed, k, _ptr(ids_out, "int32", device=False),
                           _ptr(scores_out, "float64", device=False)))


def esim_topk_device(g: int, u: int, c: float, eps: float, seed: int, k: int, ids_dev, scores_dev) -> None:
    _check(lib().esim_topk_device(g, u, c, eps, seed, k, _ptr(ids_dev, "int32", device=True),
                                  _ptr(scores_dev, "float64", device=True)))


def _batch_params(u, eps):
    u = np.ascontiguousarray(u, dtype=np.int64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    if u.shape != eps.shape or u.ndim != 1:
        raise ValueError("u and eps must be 1-D arrays of the same length")
    return u, eps


def esim_query_batch(g: int, u, eps, seed: int, c: float, s_out: np.ndarray) -> None:
    u, eps = _batch_params(u, eps)
    _check(lib().esim_query_batch(g, u.size, u.ctypes.data, eps.ctypes.data, seed, c,
                                  _ptr(s_out, "float64", device=False)))


def esim_query_batch_device(g: int, u, eps, seed: int, c: float, s_dev) -> None:
    u, eps = _batch_params(u, eps)
    _check(lib().esim_query_batch_device(g, u.size, u.ctypes.data, eps.ctypes.data, seed, c,
                                         _ptr(s_dev, "float64", device=True)))


def esim_topk_batch(g: int, u, eps, seed: int, c: float, k: int, ids_out: np.ndarray, scores_out: np.ndarray) -> None:
    u, eps = _batch_params(u, eps)
    _check(lib().esim_topk_batch(g, u.size, u.ctypes.data, eps.ctypes.data, seed, c, k,
                                 _ptr(ids_out, "int32", device=False), _ptr(scores_out, "float64", device=False)))


def esim_topk_batch_device(g: int, u, eps, seed: int, c: float, k: int, ids_dev, scores_dev) -> None:
    u, eps = _batch_params(u, eps)
    _check(lib().esim_topk_batch_device(g, u.size, u.ctypes.data, eps.ctypes.data, seed, c, k,
                                        _ptr(ids_dev, "int32", device=True), _ptr(scores_dev, "float64", device=True)))


def esim_server_create(g: int, c: float, k: int, seed: int = 0, kappa: float = 0.0, max_batch: int = 64,
                       max_waves: int = 2, mem_budget_bytes: float = 0.0) -> int:
    cfg = ServerConfig(c, kappa, seed, k, max_batch, max_waves, 0, mem_budget_bytes)
    out = _P()
    _check(lib().esim_server_create(g, ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def esim_server_submit(s: int, u: int, eps: float) -> int:
    rid = _U64()
    _check(lib().esim_server_submit(s, u, eps, ctypes.byref(rid)))
    return rid.value


def esim_server_poll(s: int, rid: int) -> int:
    st = _I32()
    _check(lib().esim_server_poll(s, rid, ctypes.byref(st)))
    return st.value


def esim_server_wait(s: int, rid: int, timeout_ms: int, ids_out: np.ndarray, scores_out: np.ndarray) -> float:
    lat = _D()
    _check(lib().esim_server_wait(s, rid, timeout_ms, _ptr(ids_out, "int32", device=False),
                                  _ptr(scores_out, "float64", device=False), ctypes.byref(lat)))
    return lat.value


def esim_server_get_stats(s: int) -> dict:
    st = ServerStats()
    _check(lib().esim_server_get_stats(s, ctypes.byref(st)))
    return st.as_dict()


def esim_server_destroy(s: int) -> None:
    lib().esim_server_destroy(s)


def esim_last_stats(g: int) -> dict:
    st = QueryStats()
    _check(lib().esim_last_stats(g, ctypes.byref(st)))
    return st.as_dict()


# ------------------------------------------------------------------ steps (device buffers)


def esim_forward(g: int, u: int, c: float, L: int, hist) -> None:
    _check(lib().esim_forward(g, u, c, L, _ptr(hist, "float64", device=True)))


def esim_allocate(g: int, hist, L: int, R_b: float, mode: int, pi_out, R_out, off) -> None:
    _check(lib().esim_allocate(g, _ptr(hist, "float64", device=True), L, R_b, mode,
                               _ptr(pi_out, "float64", device=True, allow_none=True),
                               _ptr(R_out, "uint64", device=True), _ptr(off, "uint64", device=True)))


def esim_sample(g: int, off, c: float, seed: int, nonmeet, pair_steps=None) -> None:
    _check(lib().esim_sample(g, _ptr(off, "uint64", device=True), c, seed, _ptr(nonmeet, "uint64", device=True),
                             _ptr(pair_steps, "uint64", device=True, allow_none=True)))


def esim_forward_f32(g: int, u: int, c: float, L: int, hist) -> None:
    _check(lib().esim_forward_f32(g, u, c, L, _ptr(hist, "float32", device=True)))


def esim_allocate_f32(g: int, hist, L: int, R_b: float, mode: int, pi_out, R_out, off) -> None:
    _check(lib().esim_allocate_f32(g, _ptr(hist, "float32", device=True), L, R_b, mode,
                                   _ptr(pi_out, "float64", device=True, allow_none=True),
                                   _ptr(R_out, "uint64", device=True), _ptr(off, "uint64", device=True)))


def esim_reverse_f32(g: int, hist, L: int, c: float, dhat, s_out) -> None:
    _check(lib().esim_reverse_f32(g, _ptr(hist, "float32", device=True), L, c, _ptr(dhat, "float64", device=True),
                                  _ptr(s_out, "float64", device=True)))


def esim_alg3_first_meeting(g: int, k: int, depth: int, c: float) -> np.ndarray:
    z = np.zeros(depth, dtype=np.float64)
    _check(lib().esim_alg3_first_meeting(g, k, depth, c, z.ctypes.data))
    return z


def esim_alg3_depth(v: float, c: float, supp, max_depth: int, n: int, m: int,
                    weights=(4.0, 0.2, 524288.0, 0.0625)) -> int:
    """Algorithm 3's depth choice for one node (host arithmetic, no device)."""
    sp = np.ascontiguousarray(supp, dtype=np.uint64)
    return int(lib().esim_alg3_depth(float(v), float(c), sp.ctypes.data, int(max_depth), int(n), int(m),
                                     *[float(x) for x in weights]))


def esim_alg3_paper_depth(g: int, R, c: float, max_depth: int, depth) -> None:
    _check(lib().esim_alg3_paper_depth(g, _ptr(R, "uint64", device=True), c, int(max_depth),
                                       _ptr(depth, "uint8", device=True)))


def esim_alg3_zsum(g: int, depth, c: float, zsum) -> None:
    _check(lib().esim_alg3_zsum(g, _ptr(depth, "uint8", device=True), c, _ptr(zsum, "float64", device=True)))


def esim_sample_depth(g: int, off, depth, c: float, seed: int, counts, pair_steps=None) -> None:
    _check(lib().esim_sample_depth(g, _ptr(off, "uint64", device=True), _ptr(depth, "uint8", device=True, allow_none=True),
                                   c, seed, _ptr(counts, "uint64", device=True),
                                   _ptr(pair_steps, "uint64", device=True, allow_none=True)))


def esim_dhat_alg3(g: int, counts, off, depth, zsum, c: float, dhat) -> None:
    _check(lib().esim_dhat_alg3(g, _ptr(counts, "uint64", device=True), _ptr(off, "uint64", device=True),
                                _ptr(depth, "uint8", device=True), _ptr(zsum, "float64", device=True), c,
                                _ptr(dhat, "float64", device=True)))


def esim_dhat(g: int, nonmeet, off, dhat) -> None:
    _check(lib().esim_dhat(g, _ptr(nonmeet, "uint64", device=True), _ptr(off, "uint64", device=True),
                           _ptr(dhat, "float64", device=True)))


def esim_reverse(g: int, hist, L: int, c: float, dhat, s_out) -> None:
    _check(lib().esim_reverse(g, _ptr(hist, "float64", device=True), L, c, _ptr(dhat, "float64", device=True),
                              _ptr(s_out, "float64", device=True)))


def esim_select_topk(g: int, scores, exclude: int, k: int, ids_out, vals_out) -> None:
    _check(lib().esim_select_topk(g, _ptr(scores, "float64", device=True), exclude, k,
                                  _ptr(ids_out, "int32", device=True), _ptr(vals_out, "float64", device=True)))


def esim_select_topk_static(scores, n: int, exclude: int, k: int, ids_out, vals_out, stream=None) -> None:
    """Top-k selection with static scratch (no allocation); see include/exactsim.h."""
    ptr = getattr(stream, "cuda_stream", stream)
    _check(lib().esim_select_topk_static(_ptr(scores, "float64", device=True), n, exclude, k,
                                         _ptr(ids_out, "int32", device=True), _ptr(vals_out, "float64", device=True),
                                         ptr))


def esim_sync(g: int) -> None:
    _check(lib().esim_sync(g))
