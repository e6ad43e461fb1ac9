"""Helpers shared by the tests: golden-fixture parser and an independent brute force.

The brute force below is written straight from the definitions (Section 2 of the
paper, "How to solve FOL queries", and Definition 1.1) and deliberately shares nothing
with the C oracle: it never builds N(u) lists or E_{x,y} lists, it loops over every
vertex triple and every pair of temporal edges. It is only usable on tiny graphs.
"""
from __future__ import annotations

import dataclasses
import glob
import os
from typing import Dict, List, Tuple

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_fixture(path: str):
    n = None
    edges: List[Tuple[int, int, int]] = []
    cases = []
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "n":
            n = int(tok[1])
        elif tok[0] == "edge":
            edges.append((int(tok[1]), int(tok[2]), int(tok[3])))
        elif tok[0] == "query":
            d, num, den, quant, dr, uni = map(int, tok[1:7])
            cases.append({"q": W.Query(delta=d, rho_num=num, rho_den=den, quant=quant, dir=dr,
                                       universe=uni), "counts": None, "pairs": []})
        elif tok[0] == "outer":
            cases[-1]["q"] = dataclasses.replace(cases[-1]["q"], outer=W.OUTER_FORALL_T,
                                                 outer_rho_num=int(tok[1]), outer_rho_den=int(tok[2]))
            cases[-1]["vertices"] = []
        elif tok[0] == "vertex":
            cases[-1]["vertices"].append((int(tok[1]), int(tok[2])))
        elif tok[0] == "triples":
            cases[-1]["q"] = dataclasses.replace(cases[-1]["q"], want_triples=True)
            cases[-1]["triples"] = []
        elif tok[0] == "triple":
            cases[-1]["triples"].append(tuple(int(x) for x in tok[1:4]))
        elif tok[0] == "counts":
            cases[-1]["counts"] = np.array([int(x) for x in tok[1:]], dtype=np.int32)
        elif tok[0] == "pair":
            cases[-1]["pairs"].append(tuple(int(x) for x in tok[1:5]))
        else:
            raise ValueError(f"{path}: bad line {raw!r}")
    e = np.array(edges, dtype=np.int64).reshape(-1, 3)
    g = W.TemporalGraph(n, e[:, 0].astype(np.int32).copy(), e[:, 1].astype(np.int32).copy(),
                        e[:, 2].astype(np.int64).copy())
    return g, cases


def golden_files():
    return sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


def _matches(a: int, b: int, p: int, w: int, dir: int) -> bool:
    if dir == W.DIR_OUT:
        return a == p and b == w
    if dir == W.DIR_IN:
        return a == w and b == p
    return (a == p and b == w) or (a == w and b == p)


def brute_counts(g: W.TemporalGraph, delta: int, dir: int) -> np.ndarray:
    """c_e for every input edge, by trying every witness vertex and every edge pair."""
    E = list(zip(g.src.tolist(), g.dst.tolist(), g.t.tolist()))
    out = np.zeros(len(E), dtype=np.int32)
    for i, (x, y, t) in enumerate(E):
        if x == y:
            continue
        c = 0
        for w in range(g.n):
            if w == x or w == y:
                continue
            A = [t2 for (a, b, t2) in E if _matches(a, b, x, w, dir)]
            B = [t3 for (a, b, t3) in E if _matches(a, b, y, w, dir)]
            if any(t <= t2 <= t3 <= t + delta for t2 in A for t3 in B):
                c += 1
        out[i] = c
    return out


def brute_triples(g: W.TemporalGraph, delta: int, dir: int):
    """Sorted (x, y, w): some temporal edge x -> y forms a triangle with witness w."""
    E = list(zip(g.src.tolist(), g.dst.tolist(), g.t.tolist()))
    out = set()
    for (x, y, t) in E:
        if x == y:
            continue
        for w in range(g.n):
            if w == x or w == y or (x, y, w) in out:
                continue
            A = [t2 for (a, b, t2) in E if _matches(a, b, x, w, dir)]
            B = [t3 for (a, b, t3) in E if _matches(a, b, y, w, dir)]
            if any(t <= t2 <= t3 <= t + delta for t2 in A for t3 in B):
                out.add((x, y, w))
    return sorted(out)


def brute_neighbours(g: W.TemporalGraph):
    nb = [set() for _ in range(g.n)]
    for x, y in zip(g.src.tolist(), g.dst.tolist()):
        if x != y:
            nb[x].add(y)
            nb[y].add(x)
    return nb


def brute_pairs(g: W.TemporalGraph, q: W.Query, counts: np.ndarray):
    """Sorted (x, y, max c, #certificates) from per-edge counts, by the definitions."""
    nb = brute_neighbours(g)
    best: Dict[Tuple[int, int], int] = {}
    ncert: Dict[Tuple[int, int], int] = {}
    for i, (x, y) in enumerate(zip(g.src.tolist(), g.dst.tolist())):
        if x == y:
            continue
        c = int(counts[i])
        if q.universe == W.U_HEAD:
            U = len(nb[x])
        elif q.universe == W.U_TAIL:
            U = len(nb[y])
        else:
            U = len(nb[x] & nb[y])
        if q.quant == W.Q_EXISTS:
            sat = c >= 1
        else:
            sat = c >= 1 and c * q.rho_den >= q.rho_num * U
        key = (x, y)
        best[key] = max(best.get(key, 0), c)
        ncert[key] = ncert.get(key, 0) + int(sat)
    return sorted((k[0], k[1], best[k], ncert[k]) for k in best if ncert[k] > 0)


def brute_vertices(g: W.TemporalGraph, q: W.Query, pairs):
    """Section 4 reduction by its definition: count(u) = #{v : (u, v) a solution pair};
    u is a solution when count >= 1 and count * den1 >= num1 * |N(u)|."""
    nb = brute_neighbours(g)
    cnt: Dict[int, int] = {}
    for u, v, _, _ in pairs:
        cnt[u] = cnt.get(u, 0) + 1
    return sorted((u, c) for u, c in cnt.items()
                  if c >= 1 and c * q.outer_rho_den >= q.outer_rho_num * len(nb[u]))


def brute_certificates(g: W.TemporalGraph, q: W.Query, counts: np.ndarray):
    nb = brute_neighbours(g)
    out = []
    for i, (x, y) in enumerate(zip(g.src.tolist(), g.dst.tolist())):
        if x == y:
            continue
        c = int(counts[i])
        U = len(nb[x]) if q.universe == W.U_HEAD else len(nb[y]) if q.universe == W.U_TAIL \
            else len(nb[x] & nb[y])
        if c >= 1 and (q.quant == W.Q_EXISTS or c * q.rho_den >= q.rho_num * U):
            out.append(i)
    return out


def vertices_of(res):
    return list(zip(np.asarray(res["vertex"]).tolist(), np.asarray(res["vertex_count"]).tolist()))


def pairs_of(res) -> List[Tuple[int, int, int, int]]:
    return list(zip(np.asarray(res["u"]).tolist(), np.asarray(res["v"]).tolist(),
                    np.asarray(res["count"]).tolist(), np.asarray(res["ncert"]).tolist()))


def complete_graph(k: int, t: int = 0) -> W.TemporalGraph:
    """Both directions of every pair of k vertices, all at time t."""
    src, dst = [], []
    for a in range(k):
        for b in range(k):
            if a != b:
                src.append(a)
                dst.append(b)
    m = len(src)
    return W.TemporalGraph(k, np.array(src, np.int32), np.array(dst, np.int32),
                           np.full(m, t, np.int64))


def wide_time_span_graph(seed=13, n=8, m=200):
    """Timestamps spread over [0, 2^40]: 5 clusters 2^38 s apart, each edge placed
    uniformly within 2^34 s of its cluster's start. The span is far above 2^32, so the
    library keeps 64-bit timestamps; windows below and above 2^32 both find triangles
    inside a cluster, and only windows of 2^38 or more join clusters."""
    rng = np.random.default_rng(seed)
    g = W.random_small_graph(rng, n, m, 0, self_loops=True)
    t = rng.integers(0, 5, m).astype(np.int64) * (1 << 38) + rng.integers(0, 1 << 34, m).astype(np.int64)
    return W.TemporalGraph(n, g.src, g.dst, t)


WIDE_DELTAS = (0, 1 << 31, (1 << 32) - 1, (1 << 32) + 5, 1 << 33, 1 << 38, (1 << 62) - 1)
