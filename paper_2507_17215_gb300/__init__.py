"""Python binding of ``libfolty.so`` (include/folty.h): thresholded triadic queries
"exists u, exists v, forall_rho w" on temporal graphs, computed by CUDA kernels on one
GB300 (FOLTY, arXiv 2507.17215).

The module-level functions carry the C names and only marshal arguments; every step
of loading, preprocessing and querying runs in the library's kernels. PyTorch supplies
device memory (its caching allocator, through the C allocator callbacks) and streams.
There is no fallback: importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_int32, c_int64, c_size_t,
                    c_uint8, c_uint32, c_uint64, c_void_p)
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfolty.so")

FOLTY_OK, FOLTY_EINVAL, FOLTY_ENOMEM, FOLTY_ECUDA, FOLTY_ESTATE, FOLTY_ETIMEOUT = range(6)
STATUS_NAMES = {0: "FOLTY_OK", 1: "FOLTY_EINVAL", 2: "FOLTY_ENOMEM", 3: "FOLTY_ECUDA",
                4: "FOLTY_ESTATE", 5: "FOLTY_ETIMEOUT"}
Q_EXISTS, Q_FORALL_T = 0, 1
DIR_OUT, DIR_IN, DIR_EITHER = 0, 1, 2
U_HEAD, U_TAIL, U_COMMON = 0, 1, 2

# the exported C symbols (folty.h), checked by the test suite
EXPORTED = ["folty_load_temporal_graph", "folty_preprocess", "folty_query", "folty_query_batch",
            "folty_free", "folty_last_error", "folty_graph_get_info", "folty_graph_traffic_model",
            "folty_kernel_launches", "folty_profile_enable", "folty_profile_read",
            "folty_edge_counts_noalloc", "folty_graph_common_counts", "folty_graph_core_numbers",
            "folty_graph_probe_stats", "folty_graph_tuning", "folty_tuning_force", "folty_tuning_clear_cache",
            "folty_server_create", "folty_server_submit",
            "folty_server_wait", "folty_server_get_stats", "folty_server_destroy"]


class FoltyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


# ------------------------------------------------------------------ C structs

ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class folty_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class folty_query_params(Structure):
    _fields_ = [("delta", c_int64), ("rho_num", c_uint32), ("rho_den", c_uint32),
                ("quant", c_uint8), ("dir", c_uint8), ("universe", c_uint8),
                ("want_edge_counts", c_uint8), ("outer", c_uint8), ("want_certificates", c_uint8),
                ("want_triples", c_uint8), ("reserved", c_uint8), ("outer_rho_num", c_uint32),
                ("outer_rho_den", c_uint32)]


class folty_result(Structure):
    _fields_ = [("tag", c_uint64), ("n_pairs", c_int64), ("u", POINTER(c_int32)),
                ("v", POINTER(c_int32)), ("count", POINTER(c_int32)), ("ncert", POINTER(c_int32)),
                ("n_cert_edges", c_int64), ("m", c_int64), ("edge_count", POINTER(c_int32)),
                ("n_vertices", c_int64), ("vertex", POINTER(c_int32)), ("vertex_count", POINTER(c_int32)),
                ("certificate", POINTER(c_int64)), ("n_triples", c_int64), ("triple_x", POINTER(c_int32)),
                ("triple_y", POINTER(c_int32)), ("triple_w", POINTER(c_int32))]


class folty_graph_info(Structure):
    _fields_ = [("n", c_int32), ("m", c_int64), ("m_kept", c_int64), ("static_edges", c_int64),
                ("max_degree", c_int32), ("degeneracy", c_int32), ("max_out_degree", c_int32),
                ("peel_rounds", c_int32), ("triangles", c_int64), ("probes", c_int64),
                ("sigma_max", c_int32), ("time_sorted", c_int32), ("device_bytes", c_int64)]


class folty_server_config(Structure):
    _fields_ = [("memory_budget_bytes", c_int64), ("max_batch", c_int32)]


class folty_ticket_info(Structure):
    _fields_ = [("queued_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("batch_id", c_int64), ("batch_size", c_int32),
                ("graph_index", c_int32)]


class folty_server_stats(Structure):
    _fields_ = [("batches", c_int64), ("queries", c_int64), ("queued", c_int64),
                ("memory_budget_bytes", c_int64), ("peak_memory_bytes", c_int64),
                ("max_batches_in_flight", c_int64)]


class folty_stage_profile(Structure):
    _fields_ = [("launches", c_int64), ("ms", ctypes.c_double), ("bytes", c_int64)]


STAGES = {"probe": 0, "sort": 1, "peel": 2, "threshold": 3, "select": 4, "triangles": 5, "roles": 6,
          "batch": 7, "store": 8}


class folty_probe_stats(Structure):
    _fields_ = [("triangles", c_int64), ("all_roles", c_int64), ("all_probes", c_int64),
                ("kept_triangles", c_int64), ("kept_roles", c_int64), ("kept_probes", c_int64),
                ("select_bytes", c_int64), ("probe_bytes", c_int64)]


class folty_tuning(Structure):
    _fields_ = [("tri_heavy", c_int32), ("probe_items", c_int32), ("probe_blocks_per_sm", c_int32),
                ("tri_source", c_int32), ("probe_source", c_int32), ("tri_ms", ctypes.c_float * 4),
                ("probe_ms", ctypes.c_float * 4)]


TUNE_SOURCES = {0: "default", 1: "timed trials", 2: "cache", 3: "forced"}


class folty_traffic_model(Structure):
    _fields_ = [("enum_bytes", c_int64), ("probe_bytes", c_int64), ("threshold_bytes", c_int64)]


# ------------------------------------------------------------------ library

def _load_library():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import "
                          "__graft_entry__ as g; g.build()'). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    G = c_void_p
    lib.folty_load_temporal_graph.restype = c_int32
    lib.folty_load_temporal_graph.argtypes = [c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                                              POINTER(folty_allocator), c_void_p, POINTER(c_void_p)]
    lib.folty_preprocess.restype = c_int32
    lib.folty_preprocess.argtypes = [G, c_void_p]
    lib.folty_query.restype = c_int32
    lib.folty_query.argtypes = [G, POINTER(folty_query_params), POINTER(folty_result), c_void_p]
    lib.folty_query_batch.restype = c_int32
    lib.folty_query_batch.argtypes = [G, POINTER(folty_query_params), c_int32, POINTER(folty_result),
                                      c_void_p]
    lib.folty_free.restype = None
    lib.folty_free.argtypes = [c_void_p]
    lib.folty_last_error.restype = c_char_p
    lib.folty_last_error.argtypes = []
    lib.folty_graph_get_info.restype = c_int32
    lib.folty_graph_get_info.argtypes = [G, POINTER(folty_graph_info)]
    lib.folty_graph_traffic_model.restype = c_int32
    lib.folty_graph_traffic_model.argtypes = [G, c_int32, POINTER(folty_traffic_model), c_void_p]
    lib.folty_kernel_launches.restype = c_uint64
    lib.folty_kernel_launches.argtypes = []
    lib.folty_profile_enable.restype = None
    lib.folty_profile_enable.argtypes = [c_int32]
    lib.folty_profile_read.restype = c_int32
    lib.folty_profile_read.argtypes = [c_int32, POINTER(folty_stage_profile)]
    lib.folty_graph_tuning.restype = c_int32
    lib.folty_graph_tuning.argtypes = [G, POINTER(folty_tuning)]
    lib.folty_tuning_force.restype = c_int32
    lib.folty_tuning_force.argtypes = [c_int32, c_int32, c_int32]
    lib.folty_tuning_clear_cache.restype = None
    lib.folty_tuning_clear_cache.argtypes = []
    lib.folty_graph_probe_stats.restype = c_int32
    lib.folty_graph_probe_stats.argtypes = [G, c_int64, c_int32, POINTER(folty_probe_stats), c_void_p]
    lib.folty_graph_common_counts.restype = c_int32
    lib.folty_graph_common_counts.argtypes = [G, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.folty_graph_core_numbers.restype = c_int32
    lib.folty_graph_core_numbers.argtypes = [G, c_void_p, c_void_p]
    lib.folty_server_create.restype = c_int32
    lib.folty_server_create.argtypes = [POINTER(c_void_p), c_int32, POINTER(folty_server_config),
                                        POINTER(c_void_p)]
    lib.folty_server_submit.restype = c_int32
    lib.folty_server_submit.argtypes = [c_void_p, c_int32, POINTER(folty_query_params), POINTER(c_int64)]
    lib.folty_server_wait.restype = c_int32
    lib.folty_server_wait.argtypes = [c_void_p, c_int64, c_int64, POINTER(folty_result),
                                      POINTER(folty_ticket_info)]
    lib.folty_server_get_stats.restype = c_int32
    lib.folty_server_get_stats.argtypes = [c_void_p, POINTER(folty_server_stats)]
    lib.folty_server_destroy.restype = None
    lib.folty_server_destroy.argtypes = [c_void_p]
    lib.folty_edge_counts_noalloc.restype = c_int32
    lib.folty_edge_counts_noalloc.argtypes = [G, c_int64, c_int32, c_void_p, c_void_p]
    return lib


lib = _load_library()


def _check(status: int):
    if status != FOLTY_OK:
        raise FoltyError(status, lib.folty_last_error().decode())


# ------------------------------------------------------------------ torch plumbing

def _torch():
    import torch
    return torch


@ALLOC_FN
def _torch_alloc(nbytes, stream, ctx):
    torch = _torch()
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                  stream=int(stream or 0))
    except Exception:  # out of memory -> NULL -> FOLTY_ENOMEM
        return None


@FREE_FN
def _torch_free(ptr, stream, ctx):
    _torch().cuda.caching_allocator_delete(int(ptr))


TORCH_ALLOCATOR = folty_allocator(_torch_alloc, _torch_free, None)


def current_stream() -> int:
    return int(_torch().cuda.current_stream().cuda_stream)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device), contiguous."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return int(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_ok(a, np_dtype, torch_name):
    if isinstance(a, np.ndarray):
        return a.dtype == np_dtype
    return str(a.dtype) == f"torch.{torch_name}"


# ------------------------------------------------------------------ C-named functions

def folty_load_temporal_graph(n: int, src, dst, t, allocator: Optional[str] = None,
                              stream: Optional[int] = None) -> int:
    """Returns a graph handle. src, dst (int32) and t (int64) may be host numpy arrays or
    host/device torch tensors. allocator: None (the library's own stream-ordered pool) or
    "torch" (PyTorch's caching allocator, through a callback per allocation)."""
    m = int(src.shape[0])
    if int(dst.shape[0]) != m or int(t.shape[0]) != m:
        raise ValueError("src, dst and t must have the same length")
    if not (_dtype_ok(src, np.int32, "int32") and _dtype_ok(dst, np.int32, "int32")
            and _dtype_ok(t, np.int64, "int64")):
        raise TypeError("src/dst must be int32 and t int64")
    out = c_void_p()
    alloc = ctypes.byref(TORCH_ALLOCATOR) if allocator == "torch" else None
    s = current_stream() if stream is None else stream
    _check(lib.folty_load_temporal_graph(int(n), m, _ptr(src) if m else None,
                                         _ptr(dst) if m else None, _ptr(t) if m else None,
                                         alloc, s, ctypes.byref(out)))
    return out.value


def folty_preprocess(g: int, stream: Optional[int] = None) -> None:
    _check(lib.folty_preprocess(g, current_stream() if stream is None else stream))


def _params(q) -> folty_query_params:
    p = folty_query_params()
    p.delta, p.rho_num, p.rho_den = int(q.delta), int(q.rho_num), int(q.rho_den)
    p.quant, p.dir, p.universe = int(q.quant), int(q.dir), int(q.universe)
    p.want_edge_counts = int(bool(getattr(q, "want_edge_counts", 0)))
    p.outer = int(getattr(q, "outer", 0))
    p.want_certificates = int(bool(getattr(q, "want_certificates", 0)))
    p.want_triples = int(bool(getattr(q, "want_triples", 0)))
    p.outer_rho_num = int(getattr(q, "outer_rho_num", 1))
    p.outer_rho_den = int(getattr(q, "outer_rho_den", 2))
    return p


def _take_result(r: folty_result) -> Dict[str, object]:
    k = int(r.n_pairs)
    out: Dict[str, object] = {}
    for name in ("u", "v", "count", "ncert"):
        p = getattr(r, name)
        out[name] = (np.ctypeslib.as_array(p, shape=(k,)).copy() if k > 0
                     else np.zeros(0, dtype=np.int32))
    out["n_cert_edges"] = int(r.n_cert_edges)
    if r.edge_count:
        out["edge_count"] = np.ctypeslib.as_array(r.edge_count, shape=(int(r.m),)).copy()
    else:
        out["edge_count"] = None
    nv = int(r.n_vertices)
    if r.vertex:
        out["vertex"] = (np.ctypeslib.as_array(r.vertex, shape=(nv,)).copy() if nv > 0
                         else np.zeros(0, dtype=np.int32))
        out["vertex_count"] = (np.ctypeslib.as_array(r.vertex_count, shape=(nv,)).copy() if nv > 0
                               else np.zeros(0, dtype=np.int32))
    nc = int(r.n_cert_edges)
    if r.certificate:
        out["certificates"] = (np.ctypeslib.as_array(r.certificate, shape=(nc,)).copy() if nc > 0
                               else np.zeros(0, dtype=np.int64))
    nt = int(r.n_triples)
    if r.triple_x:
        cols = [np.ctypeslib.as_array(getattr(r, f), shape=(nt,)).copy() if nt > 0 else np.zeros(0, np.int32)
                for f in ("triple_x", "triple_y", "triple_w")]
        out["triples"] = np.stack(cols, axis=1)
    lib.folty_free(ctypes.byref(r))
    return out


def folty_query(g: int, q, stream: Optional[int] = None) -> Dict[str, object]:
    p = _params(q)
    r = folty_result()
    _check(lib.folty_query(g, ctypes.byref(p), ctypes.byref(r),
                           current_stream() if stream is None else stream))
    return _take_result(r)


def folty_query_batch(g: int, qs: Sequence, stream: Optional[int] = None) -> List[Dict[str, object]]:
    nq = len(qs)
    ps = (folty_query_params * max(nq, 1))(*[_params(q) for q in qs])
    rs = (folty_result * max(nq, 1))()
    _check(lib.folty_query_batch(g, ps, nq, rs, current_stream() if stream is None else stream))
    return [_take_result(rs[i]) for i in range(nq)]


def folty_free(obj: int) -> None:
    lib.folty_free(obj)


def folty_last_error() -> str:
    return lib.folty_last_error().decode()


def folty_graph_get_info(g: int) -> Dict[str, int]:
    info = folty_graph_info()
    _check(lib.folty_graph_get_info(g, ctypes.byref(info)))
    return {name: int(getattr(info, name)) for name, _ in folty_graph_info._fields_}


def folty_graph_traffic_model(g: int, dir: int = DIR_OUT, stream: Optional[int] = None) -> Dict[str, int]:
    tm = folty_traffic_model()
    _check(lib.folty_graph_traffic_model(g, int(dir), ctypes.byref(tm),
                                         current_stream() if stream is None else stream))
    return {name: int(getattr(tm, name)) for name, _ in folty_traffic_model._fields_}


def folty_graph_common_counts(g: int, stream: Optional[int] = None):
    """(a, b, c_ab) for every static edge a < b, sorted by (a, b)."""
    S = folty_graph_get_info(g)["static_edges"]
    a = np.zeros(max(S, 1), np.int32)
    b = np.zeros(max(S, 1), np.int32)
    c = np.zeros(max(S, 1), np.int32)
    _check(lib.folty_graph_common_counts(g, a.ctypes.data, b.ctypes.data, c.ctypes.data,
                                         current_stream() if stream is None else stream))
    return a[:S], b[:S], c[:S]


def folty_graph_probe_stats(g: int, delta: int, dir: int, stream: Optional[int] = None) -> Dict[str, int]:
    """What one query's probe pass keeps (triangles, roles, probes) and its model bytes."""
    out = folty_probe_stats()
    _check(lib.folty_graph_probe_stats(g, int(delta), int(dir), ctypes.byref(out),
                                       current_stream() if stream is None else stream))
    return {name: int(getattr(out, name)) for name, _ in folty_probe_stats._fields_}


def folty_graph_tuning(g: int) -> Dict[str, object]:
    """The kernel shapes chosen for a graph and how (trials, cache, forced)."""
    t = folty_tuning()
    _check(lib.folty_graph_tuning(g, ctypes.byref(t)))
    return {"tri_heavy": int(t.tri_heavy), "probe_items": int(t.probe_items),
            "probe_tile": 256 * int(t.probe_items), "probe_blocks_per_sm": int(t.probe_blocks_per_sm),
            "tri_source": TUNE_SOURCES.get(int(t.tri_source)), "probe_source": TUNE_SOURCES.get(int(t.probe_source)),
            "tri_trial_ms": [float(x) for x in t.tri_ms], "probe_trial_ms": [float(x) for x in t.probe_ms]}


def folty_tuning_force(tri_heavy: int = 0, probe_items: int = 0, probe_blocks_per_sm: int = 0) -> None:
    """Fixed shapes for graphs preprocessed or first queried afterwards (all 0: tune again)."""
    _check(lib.folty_tuning_force(int(tri_heavy), int(probe_items), int(probe_blocks_per_sm)))


def folty_tuning_clear_cache() -> None:
    lib.folty_tuning_clear_cache()


def folty_graph_core_numbers(g: int, stream: Optional[int] = None) -> np.ndarray:
    """Core number of every vertex of the static graph (int32[n])."""
    n = folty_graph_get_info(g)["n"]
    core = np.zeros(max(n, 1), np.int32)
    _check(lib.folty_graph_core_numbers(g, core.ctypes.data, current_stream() if stream is None else stream))
    return core[:n]


def folty_kernel_launches() -> int:
    return int(lib.folty_kernel_launches())


NOALLOC_MAX_EDGES = 1 << 20  # FOLTY_NOALLOC_MAX_EDGES


def folty_edge_counts_noalloc(g: int, delta: int, dir: int, edge_count, stream: Optional[int] = None) -> None:
    """Per-edge counts of one (delta, dir) into a caller-owned device int32 tensor of
    length m (input order), with no allocation inside the library; see folty.h.

    edge_count must be a contiguous int32 CUDA tensor of at least m elements on the
    current device (the graph's); anything else is refused before the call, since the
    library's kernels write m int32 through the pointer."""
    import torch
    if not isinstance(edge_count, torch.Tensor) or not edge_count.is_cuda:
        raise TypeError("edge_count must be a CUDA torch tensor")
    if edge_count.dtype != torch.int32:
        raise TypeError(f"edge_count must be int32, not {edge_count.dtype}")
    if not edge_count.is_contiguous():
        raise ValueError("edge_count must be contiguous")
    if edge_count.device.index != torch.cuda.current_device():
        raise ValueError("edge_count must live on the current device (the graph's)")
    m = folty_graph_get_info(g)["m"]
    if edge_count.numel() < m:
        raise ValueError(f"edge_count holds {edge_count.numel()} elements, the graph has {m} edges")
    _check(lib.folty_edge_counts_noalloc(g, int(delta), int(dir), _ptr(edge_count),
                                         current_stream() if stream is None else stream))


def folty_profile_enable(on: bool = True) -> None:
    lib.folty_profile_enable(1 if on else 0)


def folty_profile_read() -> Dict[str, Dict[str, float]]:
    """Per stage: timed spans, total device ms, total model bytes."""
    out = {}
    for name, idx in STAGES.items():
        p = folty_stage_profile()
        _check(lib.folty_profile_read(idx, ctypes.byref(p)))
        out[name] = {"launches": int(p.launches), "ms": float(p.ms), "bytes": int(p.bytes)}
    return out


def folty_server_create(graphs: Sequence[int], memory_budget_bytes: int = 0, max_batch: int = 0) -> int:
    arr = (c_void_p * len(graphs))(*graphs)
    cfg = folty_server_config(int(memory_budget_bytes), int(max_batch))
    out = c_void_p()
    _check(lib.folty_server_create(arr, len(graphs), ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def folty_server_submit(sv: int, graph_index: int, q) -> int:
    p = _params(q)
    t = c_int64()
    _check(lib.folty_server_submit(sv, int(graph_index), ctypes.byref(p), ctypes.byref(t)))
    return int(t.value)


def folty_server_wait(sv: int, ticket: int, timeout_ms: int = -1):
    r = folty_result()
    info = folty_ticket_info()
    _check(lib.folty_server_wait(sv, int(ticket), int(timeout_ms), ctypes.byref(r), ctypes.byref(info)))
    res = _take_result(r)
    res["info"] = {name: getattr(info, name) for name, _ in folty_ticket_info._fields_}
    return res


def folty_server_get_stats(sv: int) -> Dict[str, int]:
    st = folty_server_stats()
    _check(lib.folty_server_get_stats(sv, ctypes.byref(st)))
    return {name: int(getattr(st, name)) for name, _ in folty_server_stats._fields_}


def folty_server_destroy(sv: int) -> None:
    lib.folty_server_destroy(sv)


# ------------------------------------------------------------------ convenience

class TemporalGraph:
    """Owns a folty graph handle: load, preprocess, query, free."""

    def __init__(self, n: int, src, dst, t, allocator: Optional[str] = None,
                 stream: Optional[int] = None, preprocess: bool = True):
        self.handle = folty_load_temporal_graph(n, src, dst, t, allocator=allocator, stream=stream)
        if preprocess:
            try:
                folty_preprocess(self.handle, stream)
            except Exception:
                self.close()
                raise

    def query(self, q, stream: Optional[int] = None):
        return folty_query(self.handle, q, stream)

    def query_batch(self, qs, stream: Optional[int] = None):
        return folty_query_batch(self.handle, qs, stream)

    def info(self):
        return folty_graph_get_info(self.handle)

    def traffic_model(self, dir: int = DIR_OUT, stream: Optional[int] = None):
        return folty_graph_traffic_model(self.handle, dir, stream)

    def core_numbers(self, stream: Optional[int] = None):
        return folty_graph_core_numbers(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            folty_free(self.handle)
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
