"""Seeded synthetic temporal graphs and query mixes.

This module only draws random inputs. It holds none of the query's arithmetic
(no neighbourhoods, no window tests, no counting), so both the CPU oracle's tests
and the CUDA library's tests and benchmark can take their inputs from it.

Graph recipe (stands in for the SNAP temporal social / Q&A graphs the paper
evaluates on in its Experiments section, which are not available here):

* static edges: Chung-Lu. Vertex ``i`` (0-based) has weight ``(i + 1 + i0) **
  (-1 / (gamma - 1))``; both endpoints of a candidate edge are drawn i.i.d.
  proportional to the weights (inverse CDF). Self-loops and repeated pairs are
  rejected, in draw order.
* every accepted static edge draws a multiplicity ``sigma`` from a truncated
  distribution (geometric or Zipf) and gets ``sigma`` temporal edges; drawing stops
  when the running total reaches ``m`` exactly, the last ``sigma`` truncated.
* every temporal edge picks its direction uniformly.
* timestamps are either uniform integers on ``[0, t_max]`` or "bursty": per static
  edge a start ``t0 ~ U{0..Y-1}`` followed by ``round(LogNormal(mu, s))`` gaps,
  wrapped modulo ``Y``.
* the edge list is returned in increasing timestamp order (stable), the way the
  paper's Preliminaries assume a temporal graph is presented.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, NamedTuple, Optional

import numpy as np

YEAR_S = 31_536_000

# query-parameter codes shared by every caller (plain data, no arithmetic)
Q_EXISTS, Q_FORALL_T = 0, 1
OUTER_NONE, OUTER_FORALL_T = 0, 1
DIR_OUT, DIR_IN, DIR_EITHER = 0, 1, 2
U_HEAD, U_TAIL, U_COMMON = 0, 1, 2


class TemporalGraph(NamedTuple):
    n: int
    src: np.ndarray  # int32[m]
    dst: np.ndarray  # int32[m]
    t: np.ndarray    # int64[m]

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


@dataclasses.dataclass(frozen=True)
class Query:
    delta: int
    rho_num: int = 1
    rho_den: int = 2
    quant: int = Q_FORALL_T
    dir: int = DIR_OUT
    universe: int = U_HEAD
    want_edge_counts: bool = True
    outer: int = OUTER_NONE      # OUTER_FORALL_T: also the vertex solutions (Section 4)
    outer_rho_num: int = 1
    outer_rho_den: int = 2
    want_certificates: bool = False
    want_triples: bool = False   # also the (x, y, w) solutions of the all-existential query


# --------------------------------------------------------------------------- samplers

def _truncated_sampler(kind: str, param: float, cap: int):
    k = np.arange(1, cap + 1, dtype=np.float64)
    if kind == "geometric":
        pmf = (1.0 - param) ** (k - 1) * param
    elif kind == "zipf":
        pmf = k ** (-param)
    else:
        raise ValueError(kind)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]

    def draw(size: int, rng: np.random.Generator) -> np.ndarray:
        idx = np.searchsorted(cdf, rng.random(size), side="right")
        return (np.minimum(idx, cap - 1) + 1).astype(np.int64)

    return draw


def _chung_lu_cdf(n: int, gamma: float, i0: float) -> np.ndarray:
    w = (np.arange(n, dtype=np.float64) + 1.0 + i0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return cdf


def _draw_endpoints(cdf: np.ndarray, count: int, rng: np.random.Generator):
    n = cdf.shape[0]
    a = np.minimum(np.searchsorted(cdf, rng.random(count), side="right"), n - 1)
    b = np.minimum(np.searchsorted(cdf, rng.random(count), side="right"), n - 1)
    return a.astype(np.int64), b.astype(np.int64)


def _bursty_times(sigma: np.ndarray, rng: np.random.Generator, span: int,
                  mu: float, s: float) -> np.ndarray:
    """Per static edge: t0 ~ U{0..span-1}, then round(LogNormal(mu, s)) gaps, mod span."""
    total = int(sigma.sum())
    n_edges = sigma.shape[0]
    t0 = rng.integers(0, span, size=n_edges, dtype=np.int64)
    gaps = np.rint(rng.lognormal(mu, s, size=total)).astype(np.int64)
    gaps = np.minimum(gaps, span)  # a gap longer than the span wraps anyway
    starts = np.zeros(n_edges, dtype=np.int64)
    starts[1:] = np.cumsum(sigma)[:-1]
    gaps[starts] = 0  # the first edge of each static edge sits at t0
    csum = np.cumsum(gaps)
    seg_base = np.repeat(csum[starts], sigma)
    rel = csum - seg_base
    return (np.repeat(t0, sigma) + rel) % span


# --------------------------------------------------------------------------- graphs

def chung_lu_temporal(n: int, m: int, gamma: float, sigma_draw, times: str,
                      rng: np.random.Generator, i0: float = 0.0, t_max: int = 1_000_000,
                      span: int = YEAR_S, mu: float = 6.0, s: float = 2.0,
                      planted: Optional[np.ndarray] = None,
                      planted_sigma_draw=None, time_sorted: bool = True) -> TemporalGraph:
    """Chung-Lu static edges with multiplicities until exactly ``m`` temporal edges.

    ``planted`` (optional, int64[k, 2] with a < b) are static edges placed first, with
    multiplicities from ``planted_sigma_draw``; Chung-Lu edges then fill up to ``m``.
    """
    keys_parts: List[np.ndarray] = []
    sig_parts: List[np.ndarray] = []
    total = 0
    seen = np.zeros(0, dtype=np.int64)
    if planted is not None and planted.shape[0] > 0:
        pk = planted[:, 0].astype(np.int64) * n + planted[:, 1].astype(np.int64)
        ps = planted_sigma_draw(pk.shape[0], rng)
        csum = np.cumsum(ps)
        if csum[-1] >= m:
            cut = int(np.searchsorted(csum, m, side="left"))
            pk, ps = pk[: cut + 1], ps[: cut + 1].copy()
            ps[-1] -= int(csum[cut] - m)
        keys_parts.append(pk)
        sig_parts.append(ps)
        total = int(ps.sum())
        seen = np.sort(pk)
    cdf = _chung_lu_cdf(n, gamma, i0)
    while total < m:
        remaining = m - total
        # expected multiplicity ~ mean of the draw; oversample candidates
        probe = sigma_draw(4096, rng).mean()
        want = max(1024, int(1.4 * remaining / probe) + 1024)
        a, b = _draw_endpoints(cdf, want, rng)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        ok = lo != hi
        key = lo[ok] * n + hi[ok]
        _, first = np.unique(key, return_index=True)
        key = key[np.sort(first)]
        if seen.shape[0]:
            key = key[~np.isin(key, seen, assume_unique=False)]
        if key.shape[0] == 0:
            continue
        sig = sigma_draw(key.shape[0], rng)
        csum = np.cumsum(sig)
        if total + int(csum[-1]) >= m:
            cut = int(np.searchsorted(csum, remaining, side="left"))
            key, sig = key[: cut + 1], sig[: cut + 1].copy()
            sig[-1] -= int(csum[cut] - remaining)
        keys_parts.append(key)
        sig_parts.append(sig)
        total += int(sig.sum())
        seen = np.union1d(seen, key)
    keys = np.concatenate(keys_parts)
    sigma = np.concatenate(sig_parts)
    assert int(sigma.sum()) == m
    lo = np.repeat(keys // n, sigma)
    hi = np.repeat(keys % n, sigma)
    flip = rng.random(m) < 0.5
    src = np.where(flip, hi, lo).astype(np.int32)
    dst = np.where(flip, lo, hi).astype(np.int32)
    if times == "uniform":
        t = rng.integers(0, t_max + 1, size=m, dtype=np.int64)
    elif times == "bursty":
        t = _bursty_times(sigma, rng, span, mu, s)
    else:
        raise ValueError(times)
    if time_sorted:
        order = np.argsort(t, kind="stable")
        src, dst, t = src[order], dst[order], t[order]
    return TemporalGraph(n, np.ascontiguousarray(src), np.ascontiguousarray(dst),
                         np.ascontiguousarray(t))


def planted_communities(n: int, count: int, size: int, p: float,
                        rng: np.random.Generator) -> np.ndarray:
    """``count`` disjoint groups of ``size`` vertices taken from the highest ids (lowest
    Chung-Lu weight); each intra-group pair is a static edge with probability ``p``."""
    pool = np.arange(n - count * size, n, dtype=np.int64)
    pool = rng.permutation(pool)
    iu, ju = np.triu_indices(size, k=1)
    out = []
    for c in range(count):
        g = np.sort(pool[c * size:(c + 1) * size])
        keep = rng.random(iu.shape[0]) < p
        out.append(np.stack([g[iu[keep]], g[ju[keep]]], axis=1))
    return np.concatenate(out, axis=0)


# --------------------------------------------------------------------------- configurations

CONFIG_SEED_BASE = 1000


def config_graph(k: int, seed: Optional[int] = None, scale: float = 1.0) -> TemporalGraph:
    """The synthetic graph of configuration ``k`` (1: tiny, 2: medium, 3: paper-scale;
    4 and 5 reuse the medium recipe). ``scale`` shrinks n and m together (tests)."""
    rng = np.random.default_rng(CONFIG_SEED_BASE + k if seed is None else seed)
    if k == 1:
        n, m = int(2000 * scale), int(20_000 * scale)
        return chung_lu_temporal(max(n, 8), max(m, 8), 2.3,
                                 _truncated_sampler("geometric", 0.5, 16), "uniform", rng,
                                 t_max=1_000_000)
    if k in (2, 4, 5):
        n, m = int(1_000_000 * scale), int(20_000_000 * scale)
        return chung_lu_temporal(max(n, 8), max(m, 8), 2.1,
                                 _truncated_sampler("zipf", 1.5, 1000), "bursty", rng)
    if k == 3:
        n, m = int(5_000_000 * scale), int(70_000_000 * scale)
        comm = max(2, int(round(50 * math.sqrt(scale)))) if scale < 1 else 50
        size = 300 if scale >= 1 else max(10, int(300 * math.sqrt(scale)))
        planted = planted_communities(n, comm, size, 0.7, rng)
        return chung_lu_temporal(n, m, 2.0, _truncated_sampler("zipf", 1.3, 10_000), "bursty",
                                 rng, planted=planted,
                                 planted_sigma_draw=_truncated_sampler("zipf", 1.3, 16))
    raise ValueError(f"no graph for configuration {k}")


def medium_graph_of_size(m: int, seed: int) -> TemporalGraph:
    """Graph with the medium recipe at ``m`` temporal edges and ``n = m / 20`` vertices
    (the resident graphs of the serving workload)."""
    rng = np.random.default_rng(seed)
    return chung_lu_temporal(max(m // 20, 8), m, 2.1, _truncated_sampler("zipf", 1.5, 1000),
                             "bursty", rng)


def config_queries(k: int) -> List[Query]:
    if k == 1:
        return [Query(delta=3600, rho_num=1, rho_den=2)]
    if k == 2:
        return [Query(delta=d, rho_num=1, rho_den=2) for d in (600, 3600, 86400)]
    if k == 3:
        return [Query(delta=3600, rho_num=3, rho_den=10)]
    raise ValueError(k)


def random_query_mix(count: int, rng: np.random.Generator,
                     want_edge_counts: bool = False) -> List[Query]:
    """Queries of the batched workload: delta log-uniform on [60 s, 7 days], rho = k/10
    with k in 1..9, quantifier and direction uniform, universe = head's neighbourhood."""
    out = []
    for _ in range(count):
        d = int(round(math.exp(rng.uniform(math.log(60.0), math.log(604_800.0)))))
        out.append(Query(delta=d, rho_num=int(rng.integers(1, 10)), rho_den=10,
                         quant=int(rng.integers(0, 2)), dir=int(rng.integers(0, 3)),
                         universe=U_HEAD, want_edge_counts=want_edge_counts))
    return out


def random_small_graph(rng: np.random.Generator, n: int, m: int, t_max: int,
                       self_loops: bool = True, time_sorted: bool = False) -> TemporalGraph:
    """Dense tiny multigraph for brute-force checks: uniform endpoints (self-loops
    allowed when asked), uniform times on a small range so that ties are common."""
    src = rng.integers(0, n, size=m).astype(np.int32)
    dst = rng.integers(0, n, size=m).astype(np.int32)
    if not self_loops:
        same = src == dst
        dst[same] = (dst[same] + 1 + rng.integers(0, n - 1, size=int(same.sum()))) % n
    t = rng.integers(0, t_max + 1, size=m).astype(np.int64)
    if time_sorted:
        o = np.argsort(t, kind="stable")
        src, dst, t = src[o], dst[o], t[o]
    return TemporalGraph(n, src, dst, t)
