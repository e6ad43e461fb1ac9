"""The paper's own source-only procedure (out- and in-neighbour cases of Section 3,
interval lists, the appendix's three-phase segment trees) as an independent CPU
cross-check of the oracle (oracle/folty_paper.c).

* the appendix's worked example of the segment tree (App. A.1): two intervals of one
  in-neighbour that overlap count once at t = 9, in either insertion order, and a second
  in-neighbour's interval makes it two;
* the segment tree against a brute-force count of distinct sources on random lists;
* per-edge counts of the whole procedure against the oracle on random graphs and the
  workload recipe, for several windows.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _support import golden_files, parse_fixture

TS = [5, 7, 9, 10, 12, 14]


def test_segment_tree_appendix_example():
    # App. A.1: I_{w,u,v} = {[6,13], [8,10]}; e = (u, v, 9) must see w once, not twice
    w_first = [[(6, 13), (8, 10)]]
    w_swapped = [[(8, 10), (6, 13)]]
    q = [5, 7, 9, 10, 12, 14]
    for lists in (w_first, w_swapped):
        got = oracle.paper_segtree_counts(TS, lists, q)
        # 5 lies outside both intervals; 7..12 inside [6,13]; 14 outside
        assert got.tolist() == [0, 1, 1, 1, 1, 0]
    # a second in-neighbour z with I_{z,u,v} = {[8,14]}: t = 9 now sees two sources
    got = oracle.paper_segtree_counts(TS, w_swapped + [[(8, 14)]], q)
    assert got.tolist() == [0, 1, 2, 2, 2, 1]
    assert oracle.paper_segtree_counts(TS, w_first + [[(8, 14)]], q).tolist() == got.tolist()


def test_segment_tree_against_brute_force():
    rng = np.random.default_rng(21)
    for _ in range(300):
        r = int(rng.integers(1, 40))
        ts = np.unique(rng.integers(0, 100, size=r))
        nsrc = int(rng.integers(1, 6))
        lists = []
        for _s in range(nsrc):
            L = []
            for _k in range(int(rng.integers(0, 6))):
                a = int(rng.integers(-5, 105))
                b = a + int(rng.integers(0, 40))
                L.append((max(a, 0), b))
            lists.append(L)
        queries = np.arange(-2, 110)
        got = oracle.paper_segtree_counts(ts, lists, queries)
        leaf = set(ts.tolist())
        want = [sum(any(a <= t <= b for a, b in L) for L in lists) if t in leaf else 0 for t in queries.tolist()]
        assert got.tolist() == want


def _tiny_graphs():
    rng = np.random.default_rng(17)
    out = []
    for i in range(20):
        n = int(rng.integers(3, 14))
        m = int(rng.integers(4, 80))
        out.append(W.random_small_graph(rng, n, m, int(rng.integers(0, 40)), self_loops=bool(i % 4 == 0)))
    return out


@pytest.mark.parametrize("delta", [0, 1, 4, 11, 60])
def test_paper_procedure_equals_oracle_on_random_graphs(delta):
    for g in _tiny_graphs():
        with oracle.OracleGraph.of(g) as og:
            want, _ = og.counts(delta, W.DIR_OUT)
        np.testing.assert_array_equal(oracle.paper_counts(g, delta), want)


def test_paper_procedure_on_fixtures_and_dense_graphs():
    rng = np.random.default_rng(5)
    graphs = [parse_fixture(p)[0] for p in golden_files()]
    graphs += [W.random_small_graph(rng, 25, 2500, 300), W.random_small_graph(rng, 60, 4000, 2000)]
    for g in graphs:
        with oracle.OracleGraph.of(g) as og:
            for delta in (0, 3, 20, 150, 10_000):
                want, _ = og.counts(delta, W.DIR_OUT)
                np.testing.assert_array_equal(oracle.paper_counts(g, delta), want)


def test_paper_procedure_on_the_small_workload():
    g = W.config_graph(1)
    with oracle.OracleGraph.of(g) as og:
        for delta in (3600, 100_000):
            want, _ = og.counts(delta, W.DIR_OUT)
            np.testing.assert_array_equal(oracle.paper_counts(g, delta), want)
