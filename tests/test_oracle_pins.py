"""Pins for the CPU oracle: it is checked against things other than itself.

* hand-worked fixtures in tests/golden/ (paper Figure 2, the window bounds of Section 2,
  Theorem 3.1's search order, multigraph/self-loop handling);
* an independent brute force over vertex triples and edge pairs (tests/_support.py);
* the oracle's own A x B mode (the definition) against its greedy mode (Theorem 3.1);
* closed forms (complete graph) and invariants (relabelling, time shift, monotonicity in
  delta and rho, rho -> 0 equals the existential query, c <= |N(x) cap N(y)|,
  "either" >= max("out", "in")).
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from _support import (brute_certificates, brute_counts, brute_pairs, brute_triples, brute_vertices,
                      complete_graph, golden_files, pairs_of, parse_fixture, vertices_of)


@pytest.mark.parametrize("path", golden_files(), ids=os.path.basename)
def test_golden_fixture(path):
    g, cases = parse_fixture(path)
    assert cases
    with oracle.OracleGraph.of(g) as og:
        for case in cases:
            for brute in (False, True):
                r = og.query(case["q"], brute=brute)
                np.testing.assert_array_equal(r["edge_count"], case["counts"])
                assert pairs_of(r) == case["pairs"]
                if "vertices" in case:
                    assert vertices_of(r) == case["vertices"]
                if "triples" in case:
                    assert [tuple(x) for x in r["triples"].tolist()] == case["triples"]


def _tiny_graphs():
    rng = np.random.default_rng(7)
    out = []
    for i in range(14):
        n = int(rng.integers(3, 11))
        m = int(rng.integers(4, 45))
        t_max = int(rng.integers(0, 25))
        out.append(W.random_small_graph(rng, n, m, t_max, self_loops=bool(i % 3 == 0)))
    return out


@pytest.mark.parametrize("dir", [W.DIR_OUT, W.DIR_IN, W.DIR_EITHER])
def test_oracle_matches_python_brute_force(dir):
    for g in _tiny_graphs():
        for delta in (0, 1, 3, 7, 30):
            want = brute_counts(g, delta, dir)
            with oracle.OracleGraph.of(g) as og:
                got, _ = og.counts(delta, dir)
                np.testing.assert_array_equal(got, want)
                for q in (W.Query(delta, 1, 2, W.Q_FORALL_T, dir, W.U_HEAD),
                          W.Query(delta, 1, 3, W.Q_FORALL_T, dir, W.U_TAIL),
                          W.Query(delta, 2, 3, W.Q_FORALL_T, dir, W.U_COMMON),
                          W.Query(delta, 1, 2, W.Q_EXISTS, dir, W.U_HEAD)):
                    r = og.query(q)
                    assert pairs_of(r) == brute_pairs(g, q, want)


def test_greedy_equals_definition_on_random_graphs():
    """Theorem 3.1 (and its Case-2 twin) as a property: the first-entry search finds a
    window match exactly when one exists."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        g = W.random_small_graph(rng, int(rng.integers(4, 30)), int(rng.integers(20, 400)),
                                 int(rng.integers(5, 200)))
        with oracle.OracleGraph.of(g) as og:
            for dir in (0, 1, 2):
                for delta in (0, 2, 13, 60):
                    a, _ = og.counts(delta, dir, brute=False)
                    b, _ = og.counts(delta, dir, brute=True)
                    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("k", [3, 4, 7, 12])
def test_complete_graph_closed_form(k):
    """Both directions of every pair at one time: every other vertex is a witness for
    every edge, whatever the window, so c_e = k - 2 and |N(x)| = k - 1."""
    g = complete_graph(k, t=1000)
    with oracle.OracleGraph.of(g) as og:
        for dir in (0, 1, 2):
            c, com = og.counts(0, dir)
            assert (c == k - 2).all() and (com == k - 2).all()
        # rho = (k-2)/(k-1): every edge certifies; rho = 1: none does (N(x) contains y)
        r = og.query(W.Query(0, k - 2, k - 1, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD))
        assert len(r["u"]) == k * (k - 1) and (r["count"] == k - 2).all()
        r = og.query(W.Query(0, 1, 1, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD))
        assert len(r["u"]) == 0


def test_staircase_closed_form():
    """x -> w_i at time i and y -> w_i at time i + s for witnesses w_1..w_k, plus one
    x -> y edge at time 0: witness i matches iff i + s <= delta, so
    c = #{i in 1..k : i + s <= delta} = clamp(delta - s, 0, k)."""
    k, s = 9, 3
    x, y = 0, 1
    src, dst, t = [x], [y], [0]
    for i in range(1, k + 1):
        w = 1 + i
        src += [x, y]
        dst += [w, w]
        t += [i, i + s]
    g = W.TemporalGraph(k + 2, np.array(src, np.int32), np.array(dst, np.int32),
                        np.array(t, np.int64))
    with oracle.OracleGraph.of(g) as og:
        for delta in range(0, k + s + 3):
            c, _ = og.counts(delta, W.DIR_OUT, idx=[0])
            assert c[0] == min(max(delta - s, 0), k)
            c_in, _ = og.counts(delta, W.DIR_IN, idx=[0])
            assert c_in[0] == 0


def _medium_random(seed=5):
    rng = np.random.default_rng(seed)
    return W.random_small_graph(rng, 40, 1500, 400)


def test_relabel_and_time_shift_invariance():
    g = _medium_random()
    rng = np.random.default_rng(3)
    perm = rng.permutation(g.n).astype(np.int32)
    g2 = W.TemporalGraph(g.n, perm[g.src], perm[g.dst], g.t + 123_456_789)
    with oracle.OracleGraph.of(g) as a, oracle.OracleGraph.of(g2) as b:
        for dir in (0, 1, 2):
            for delta in (0, 5, 40):
                ca, na = a.counts(delta, dir)
                cb, nb = b.counts(delta, dir)
                np.testing.assert_array_equal(ca, cb)
                np.testing.assert_array_equal(na, nb)
        q = W.Query(40, 1, 4)
        ra, rb = a.query(q), b.query(q)
        got = sorted((int(perm[u]), int(perm[v]), c, n) for u, v, c, n in pairs_of(ra))
        assert got == pairs_of(rb)


def test_bounds_and_monotonicity():
    g = _medium_random(9)
    with oracle.OracleGraph.of(g) as og:
        deg = og.degrees()
        prev = None
        for delta in (0, 1, 5, 20, 80, 400, 10_000):
            c, com = og.counts(delta, W.DIR_OUT)
            loop = g.src == g.dst
            assert (c <= com).all()
            assert (com[~loop] <= np.minimum(deg[g.src], deg[g.dst])[~loop]).all()
            if prev is not None:
                assert (c >= prev).all(), "c_e must not shrink as delta grows"
            prev = c
            ci, _ = og.counts(delta, W.DIR_IN)
            ce, _ = og.counts(delta, W.DIR_EITHER)
            assert (ce >= np.maximum(c, ci)).all()
        # rho monotone: certificates for a larger rho are certificates for a smaller one
        last = None
        for num in (0, 1, 2, 3, 5, 8, 10):
            r = og.query(W.Query(80, num, 10))
            cur = {(u, v): n for u, v, _, n in pairs_of(r)}
            if last is not None:
                assert all(cur.get(k, 0) <= last.get(k, 0) for k in cur)
                assert set(cur) <= set(last)
            last = cur
        # rho = 0 is the existential query (with the c >= 1 reading)
        r0 = og.query(W.Query(80, 0, 1, W.Q_FORALL_T))
        re = og.query(W.Query(80, 1, 2, W.Q_EXISTS))
        assert pairs_of(r0) == pairs_of(re)


def test_config1_oracle_agrees_with_definition_mode():
    g = W.config_graph(1)
    with oracle.OracleGraph.of(g) as og:
        for delta in (3600, 100_000):
            a, _ = og.counts(delta, W.DIR_OUT)
            b, _ = og.counts(delta, W.DIR_OUT, brute=True)
            np.testing.assert_array_equal(a, b)


def test_invalid_graph_rejected():
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32),
                           np.array([0, 0], np.int64))
    with pytest.raises(ValueError):
        oracle.OracleGraph(3, np.array([0], np.int32), np.array([1], np.int32),
                           np.array([-1], np.int64))


def test_vertex_queries_and_certificates_match_brute_force():
    """Section 4 reductions and the certificate list, against their definitions."""
    import dataclasses
    for g in _tiny_graphs():
        for delta in (0, 3, 30):
            for dr in (W.DIR_OUT, W.DIR_EITHER):
                counts = brute_counts(g, delta, dr)
                with oracle.OracleGraph.of(g) as og:
                    for q in (W.Query(delta, 1, 3, W.Q_FORALL_T, dr, W.U_TAIL),
                              W.Query(delta, 1, 2, W.Q_EXISTS, dr, W.U_HEAD)):
                        for num1, den1 in ((0, 1), (1, 4), (1, 2), (1, 1)):
                            qq = dataclasses.replace(q, outer=W.OUTER_FORALL_T, outer_rho_num=num1,
                                                     outer_rho_den=den1)
                            r = og.query(qq)
                            pairs = brute_pairs(g, qq, counts)
                            assert vertices_of(r) == brute_vertices(g, qq, pairs)
                        assert r["certificates"].tolist() == brute_certificates(g, q, counts)


def test_forall_forall_solutions_are_forall_exists_solutions():
    """Every exists-forall-forall solution is an exists-forall-exists solution (Section 5,
    Insights), and vertex solutions shrink as the outer threshold grows."""
    import dataclasses
    g = _medium_random(13)
    with oracle.OracleGraph.of(g) as og:
        for num1 in (1, 2, 3, 5):
            q_ff = W.Query(60, 1, 4, W.Q_FORALL_T, outer=W.OUTER_FORALL_T, outer_rho_num=num1, outer_rho_den=10)
            q_fe = dataclasses.replace(q_ff, quant=W.Q_EXISTS)
            ff = set(og.query(q_ff)["vertex"].tolist())
            fe = set(og.query(q_fe)["vertex"].tolist())
            assert ff <= fe
        prev = None
        for num1 in (0, 1, 2, 4, 7, 10):
            cur = set(og.query(W.Query(60, 0, 1, W.Q_EXISTS, outer=W.OUTER_FORALL_T, outer_rho_num=num1,
                                       outer_rho_den=10))["vertex"].tolist())
            if prev is not None:
                assert cur <= prev
            prev = cur


def test_triples_match_brute_force():
    """Definition 1.2's all-existential query: triples (x, y, w) against the definition."""
    for g in _tiny_graphs():
        with oracle.OracleGraph.of(g) as og:
            for dr in (W.DIR_OUT, W.DIR_IN, W.DIR_EITHER):
                for delta in (0, 3, 30):
                    got = [tuple(x) for x in og.triples(delta, dr).tolist()]
                    assert got == brute_triples(g, delta, dr)
                    # a pair's triples are the union of its edges' witnesses: at least c_e
                    c, _ = og.counts(delta, dr)
                    per_pair = {}
                    for (x, y, _w) in got:
                        per_pair[(x, y)] = per_pair.get((x, y), 0) + 1
                    for i, (x, y) in enumerate(zip(g.src.tolist(), g.dst.tolist())):
                        if x != y:
                            assert per_pair.get((x, y), 0) >= c[i]
