"""CPU oracle for thresholded triadic queries (FOLTY, arXiv 2507.17215).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` import this package. The CUDA library never does, and this package
never imports the library.

``folty_oracle.c`` is the plain C definition (see its header for the paper passages it
follows); ``folty_paper.c`` is the paper's own source-only procedure (out- and
in-neighbour cases, interval lists, three-phase segment trees), an independent
cross-check of the first. This module compiles both with gcc and wraps them with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "folty_oracle.c"), os.path.join(_HERE, "folty_paper.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", *_SRCS,
                    "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_graph_new.restype = P
    lib.oracle_graph_new.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p]
    lib.oracle_graph_free.argtypes = [P]
    lib.oracle_kept_edges.restype = ctypes.c_int64
    lib.oracle_kept_edges.argtypes = [P]
    lib.oracle_degree.restype = ctypes.c_int32
    lib.oracle_degree.argtypes = [P, ctypes.c_int32]
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_counts.restype = ctypes.c_int
    lib.oracle_counts.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                  i64p, i32p, i32p]
    lib.oracle_query.restype = ctypes.c_int64
    lib.oracle_query.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p,
                                 i32p, i32p, i64p]
    lib.oracle_vertices.restype = ctypes.c_int64
    lib.oracle_vertices.argtypes = [P, ctypes.c_int64, i32p, ctypes.c_int64, ctypes.c_int64, i32p, i32p]
    lib.oracle_triples.restype = ctypes.c_int64
    lib.oracle_triples.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, i32p, i32p, i32p]
    lib.paper_counts.restype = ctypes.c_int
    lib.paper_counts.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i64p, ctypes.c_int64, i32p]
    lib.paper_segtree_counts.restype = ctypes.c_int
    lib.paper_segtree_counts.argtypes = [i64p, ctypes.c_int, i64p, i64p, i32p, ctypes.c_int, i64p, ctypes.c_int,
                                         i64p]
    lib.oracle_certificates.restype = ctypes.c_int64
    lib.oracle_certificates.argtypes = [P, i32p, i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, i64p]
    _lib = lib
    return lib


def threads() -> int:
    return int(_load().oracle_threads())


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def paper_counts(g, delta: int) -> np.ndarray:
    """c_e (input order) of the out motif by the paper's procedure (folty_paper.c)."""
    lib = _load()
    src = np.ascontiguousarray(g.src, dtype=np.int32)
    dst = np.ascontiguousarray(g.dst, dtype=np.int32)
    t = np.ascontiguousarray(g.t, dtype=np.int64)
    out = np.zeros(max(src.shape[0], 1), dtype=np.int32)
    rc = lib.paper_counts(int(g.n), src.shape[0], _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32),
                          _ptr(t, ctypes.c_int64), int(delta), _ptr(out, ctypes.c_int32))
    if rc != 0:
        raise ValueError("paper_counts: bad arguments")
    return out[:src.shape[0]]


def paper_segtree_counts(timestamps, lists, queries) -> np.ndarray:
    """The appendix's segment tree on its own: a tree over the distinct ascending
    `timestamps`, the interval lists of successive sources inserted in order
    (`lists[s]` = [(lo, hi), ...]), then the root-to-leaf counter sums at `queries`."""
    lib = _load()
    ts = np.ascontiguousarray(timestamps, dtype=np.int64)
    lo = np.array([a for L in lists for a, _ in L] or [0], dtype=np.int64)
    hi = np.array([b for L in lists for _, b in L] or [0], dtype=np.int64)
    off = np.zeros(len(lists) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(L) for L in lists])
    q = np.ascontiguousarray(queries, dtype=np.int64)
    out = np.zeros(max(q.shape[0], 1), dtype=np.int64)
    rc = lib.paper_segtree_counts(_ptr(ts, ctypes.c_int64), ts.shape[0], _ptr(lo, ctypes.c_int64),
                                  _ptr(hi, ctypes.c_int64), _ptr(off, ctypes.c_int32), len(lists),
                                  _ptr(q, ctypes.c_int64), q.shape[0], _ptr(out, ctypes.c_int64))
    if rc != 0:
        raise MemoryError("paper_segtree_counts")
    return out[:q.shape[0]]


class OracleGraph:
    """A temporal graph held by the C oracle. Arrays are kept alive by this object."""

    def __init__(self, n: int, src, dst, t):
        self._lib = _load()
        self.n = int(n)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.t = np.ascontiguousarray(t, dtype=np.int64)
        self.m = int(self.src.shape[0])
        h = self._lib.oracle_graph_new(self.n, self.m, _ptr(self.src, ctypes.c_int32),
                                       _ptr(self.dst, ctypes.c_int32),
                                       _ptr(self.t, ctypes.c_int64))
        if not h:
            raise ValueError("oracle: invalid temporal graph (ids outside [0, n) or t < 0)")
        self._h = h

    @classmethod
    def of(cls, g) -> "OracleGraph":
        return cls(g.n, g.src, g.dst, g.t)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def triples(self, delta: int, dir: int = 0) -> np.ndarray:
        """Sorted (x, y, w) rows of the all-existential query (Definition 1.2)."""
        i32 = ctypes.c_int32
        z = np.zeros(1, dtype=np.int32)
        k = self._lib.oracle_triples(self._h, int(delta), int(dir), 0, _ptr(z, i32), _ptr(z, i32), _ptr(z, i32))
        if k < 0:
            raise ValueError("oracle: bad triple query")
        tx = np.zeros(max(k, 1), dtype=np.int32)
        ty = np.zeros(max(k, 1), dtype=np.int32)
        tw = np.zeros(max(k, 1), dtype=np.int32)
        self._lib.oracle_triples(self._h, int(delta), int(dir), k, _ptr(tx, i32), _ptr(ty, i32), _ptr(tw, i32))
        return np.stack([tx[:k], ty[:k], tw[:k]], axis=1)

    def degree(self, u: int) -> int:
        return int(self._lib.oracle_degree(self._h, int(u)))

    def degrees(self) -> np.ndarray:
        return np.array([self.degree(u) for u in range(self.n)], dtype=np.int64)

    def counts(self, delta: int, dir: int = 0, brute: bool = False,
               idx: Optional[Sequence[int]] = None):
        """(c_e, |N(x) cap N(y)|) for the given input edges (all when idx is None)."""
        if idx is None:
            k = self.m
            ip = None
        else:
            idx_a = np.ascontiguousarray(idx, dtype=np.int64)
            k = idx_a.shape[0]
            ip = _ptr(idx_a, ctypes.c_int64)
        out = np.zeros(k, dtype=np.int32)
        com = np.zeros(k, dtype=np.int32)
        rc = self._lib.oracle_counts(self._h, int(delta), int(dir), int(bool(brute)), k, ip,
                                     _ptr(out, ctypes.c_int32), _ptr(com, ctypes.c_int32))
        if rc != 0:
            raise ValueError("oracle: bad arguments")
        return out, com

    def query(self, q, brute: bool = False) -> Dict[str, np.ndarray]:
        """The full query: per-edge counts (input order) and the sorted pair list."""
        m = self.m
        counts = np.zeros(m, dtype=np.int32)
        common = np.zeros(m, dtype=np.int32)
        cap = max(m, 1)
        pu = np.zeros(cap, dtype=np.int32)
        pv = np.zeros(cap, dtype=np.int32)
        pc = np.zeros(cap, dtype=np.int32)
        pn = np.zeros(cap, dtype=np.int32)
        ncert = np.zeros(1, dtype=np.int64)
        i32 = ctypes.c_int32
        k = self._lib.oracle_query(self._h, int(q.delta), int(q.rho_num), int(q.rho_den),
                                   int(q.quant), int(q.dir), int(q.universe), int(bool(brute)),
                                   _ptr(counts, i32), _ptr(common, i32), _ptr(pu, i32),
                                   _ptr(pv, i32), _ptr(pc, i32), _ptr(pn, i32),
                                   _ptr(ncert, ctypes.c_int64))
        if k < 0:
            raise ValueError("oracle: bad query parameters")
        res = {"u": pu[:k].copy(), "v": pv[:k].copy(), "count": pc[:k].copy(),
               "ncert": pn[:k].copy(), "edge_count": counts, "common": common,
               "n_cert_edges": int(ncert[0])}
        certs = np.zeros(max(int(ncert[0]), 1), dtype=np.int64)
        nc = self._lib.oracle_certificates(self._h, _ptr(counts, i32), _ptr(common, i32), int(q.rho_num),
                                           int(q.rho_den), int(q.quant), int(q.universe),
                                           _ptr(certs, ctypes.c_int64))
        res["certificates"] = certs[:nc].copy()
        if getattr(q, "want_triples", False):
            res["triples"] = self.triples(q.delta, q.dir)
        if getattr(q, "outer", 0):
            vout = np.zeros(max(self.n, 1), dtype=np.int32)
            cout = np.zeros(max(self.n, 1), dtype=np.int32)
            heads = np.ascontiguousarray(res["u"], dtype=np.int32)
            nv = self._lib.oracle_vertices(self._h, heads.shape[0], _ptr(heads, i32), int(q.outer_rho_num),
                                           int(q.outer_rho_den), _ptr(vout, i32), _ptr(cout, i32))
            if nv < 0:
                raise ValueError("oracle: bad outer threshold")
            res["vertex"] = vout[:nv].copy()
            res["vertex_count"] = cout[:nv].copy()
        return res
