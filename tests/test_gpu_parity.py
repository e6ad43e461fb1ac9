"""CUDA library vs the CPU oracle, element by element (bit-exact: all arithmetic is
integer). Every call goes through the C ABI (libfolty.so) via the thin binding."""
import numpy as np
import pytest

import oracle
import workloads as W
import dataclasses

from _support import WIDE_DELTAS, golden_files, pairs_of, parse_fixture, vertices_of, wide_time_span_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_17215_gb300 as F
    return F


def _lib_results(F, g, queries, allocator="torch", batch=False):
    with F.TemporalGraph(g.n, g.src, g.dst, g.t, allocator=allocator) as G:
        if batch:
            return G.query_batch(queries), G.info()
        return [G.query(q) for q in queries], G.info()


def _assert_same(lib_res, ora_res, what=""):
    np.testing.assert_array_equal(lib_res["edge_count"], ora_res["edge_count"], err_msg=what)
    assert pairs_of(lib_res) == pairs_of(ora_res), what
    assert lib_res["n_cert_edges"] == ora_res["n_cert_edges"], what


def _full_mix(deltas, want=True):
    qs = []
    for d in deltas:
        for dr in (W.DIR_OUT, W.DIR_IN, W.DIR_EITHER):
            qs.append(W.Query(d, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, want))
        qs.append(W.Query(d, 1, 3, W.Q_FORALL_T, W.DIR_OUT, W.U_TAIL, want))
        qs.append(W.Query(d, 3, 4, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, want))
        qs.append(W.Query(d, 1, 2, W.Q_EXISTS, W.DIR_IN, W.U_HEAD, want))
    return qs


def _check_graph(F, g, queries, allocator="torch"):
    res, info = _lib_results(F, g, queries, allocator=allocator)
    with oracle.OracleGraph.of(g) as og:
        for q, r in zip(queries, res):
            _assert_same(r, og.query(q), what=str(q))
    return info


@pytest.mark.parametrize("path", golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden_fixtures_through_library(F, path):
    g, cases = parse_fixture(path)
    qs = [dataclasses.replace(c["q"], want_edge_counts=True) for c in cases]
    res, _ = _lib_results(F, g, qs)
    for c, r in zip(cases, res):
        np.testing.assert_array_equal(r["edge_count"], c["counts"])
        assert pairs_of(r) == c["pairs"]
        if "vertices" in c:
            assert vertices_of(r) == c["vertices"]
        if "triples" in c:
            assert [tuple(x) for x in r["triples"].tolist()] == c["triples"]


def test_random_tiny_graphs(F):
    rng = np.random.default_rng(2024)
    for i in range(25):
        g = W.random_small_graph(rng, int(rng.integers(2, 14)), int(rng.integers(1, 90)),
                                 int(rng.integers(0, 30)), self_loops=bool(i % 2))
        _check_graph(F, g, _full_mix((0, 3, 11, 1000)))


def test_random_dense_graphs_default_allocator(F):
    """Several probe tiles and ragged tails; the library's own stream-ordered allocator."""
    rng = np.random.default_rng(77)
    for n, m, tmax in ((30, 3000, 200), (60, 12000, 5000), (200, 40000, 100000)):
        g = W.random_small_graph(rng, n, m, tmax)
        _check_graph(F, g, _full_mix((0, 40, 700)), allocator=None)


def test_config1_tiny_workload(F):
    g = W.config_graph(1)
    qs = [W.Query(3600, 1, 2, want_edge_counts=True)]
    qs += _full_mix((100_000, 1_000_000))
    qs += [W.Query(10 ** 6, k, 10, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True) for k in (1, 5, 9)]
    _check_graph(F, g, qs)


@pytest.mark.parametrize("k,scale", [(2, 0.02), (3, 0.004)])
def test_scaled_medium_and_paper_scale_recipes(F, k, scale):
    g = W.config_graph(k, scale=scale)
    qs = [W.Query(d, 1, 2, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True) for d in (600, 3600, 86400)]
    qs += [W.Query(3600, 3, 10, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, True),
           W.Query(604800, 1, 10, W.Q_EXISTS, W.DIR_IN, W.U_TAIL, True)]
    info = _check_graph(F, g, qs)
    assert info["triangles"] > 100 and info["probes"] > 1000


def test_unsorted_input_equals_sorted(F):
    rng = np.random.default_rng(5)
    g = W.config_graph(2, scale=0.01)
    perm = rng.permutation(g.m)
    gs = W.TemporalGraph(g.n, g.src[perm].copy(), g.dst[perm].copy(), g.t[perm].copy())
    qs = [W.Query(3600, 1, 2, want_edge_counts=True), W.Query(86400, 1, 5, W.Q_FORALL_T, W.DIR_EITHER,
                                                             W.U_COMMON, True)]
    a, ia = _lib_results(F, g, qs)
    b, ib = _lib_results(F, gs, qs)
    assert ia["time_sorted"] == 1 and ib["time_sorted"] == 0
    for q, ra, rb in zip(qs, a, b):
        assert pairs_of(ra) == pairs_of(rb)
        # edge i of the shuffled graph is edge perm[i] of the sorted one
        np.testing.assert_array_equal(ra["edge_count"][perm], rb["edge_count"])
    with oracle.OracleGraph.of(gs) as og:
        for q, r in zip(qs, b):
            _assert_same(r, og.query(q))


def _device_load_cases():
    """Input graphs for the fused copy-and-check load of device-resident arrays: a ragged
    length (m mod 4 = 3), shuffled times, a time inversion only across a 4-edge group
    boundary, self-loops, and a bad id inside a group and in the ragged tail."""
    rng = np.random.default_rng(21)
    g = W.config_graph(2, scale=0.01)
    m = g.m - (g.m % 4) - 1
    base = W.TemporalGraph(g.n, g.src[:m].copy(), g.dst[:m].copy(), g.t[:m].copy())
    perm = rng.permutation(m)
    shuffled = W.TemporalGraph(g.n, base.src[perm].copy(), base.dst[perm].copy(), base.t[perm].copy())
    assert np.all(base.t[1:] >= base.t[:-1])
    t = base.t.copy()
    j = 4 * (m // 8)
    t[j - 1] = t[j] + 1
    boundary = W.TemporalGraph(g.n, base.src.copy(), base.dst.copy(), t)
    loops = W.TemporalGraph(g.n, base.src.copy(), base.src.copy(), base.t.copy())
    loops.dst[1::3] = base.dst[1::3]
    return base, shuffled, boundary, loops


def test_device_resident_input_equals_host_input(F):
    import torch
    base, shuffled, boundary, loops = _device_load_cases()
    assert base.m % 4 == 3
    # the boundary case is out of time order at exactly one place, across groups of 4
    inv = np.nonzero(boundary.t[1:] < boundary.t[:-1])[0]
    assert len(inv) == 1 and (inv[0] + 1) % 4 == 0
    qs = [W.Query(3600, 1, 2, want_edge_counts=True),
          W.Query(86400, 1, 5, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, True)]
    for g in (base, shuffled, boundary, loops):
        want, want_info = _lib_results(F, g, qs)
        dev = [torch.from_numpy(a).cuda() for a in (g.src, g.dst, g.t)]
        pinned = [torch.from_numpy(a).pin_memory() for a in (g.src, g.dst, g.t)]
        # offset views: 4-byte and 8-byte aligned but not 16-byte aligned (the copy path)
        pad = [torch.cat([a[:1], a]) for a in dev]
        for arrs in (dev, pinned, [a[1:] for a in pad]):
            with F.TemporalGraph(g.n, *arrs) as G:
                got, info = [G.query(q) for q in qs], G.info()
            assert info == want_info
            assert info["time_sorted"] == (0 if g is shuffled or g is boundary else 1)
            for q, a, b in zip(qs, want, got):
                _assert_same(b, a, what=str(q))
    for pos in (4 * (base.m // 8) + 2, base.m - 1):  # inside a group of 4; the ragged tail
        src = base.src.copy()
        src[pos] = base.n
        for arrs in ([src, base.dst, base.t], [torch.from_numpy(a).cuda() for a in (src, base.dst, base.t)],
                     [torch.from_numpy(a).pin_memory() for a in (src, base.dst, base.t)]):
            with pytest.raises(F.FoltyError) as ei:
                F.folty_load_temporal_graph(base.n, *arrs)
            assert ei.value.status == F.FOLTY_EINVAL and f"edge {pos}:" in str(ei.value)


def _edge_case_graphs():
    out = {}
    e = np.zeros(0, np.int32)
    out["empty"] = W.TemporalGraph(5, e, e.copy(), np.zeros(0, np.int64))
    out["single_vertex_loops"] = W.TemporalGraph(1, np.zeros(3, np.int32), np.zeros(3, np.int32),
                                                 np.array([1, 2, 3], np.int64))
    out["path_no_triangles"] = W.TemporalGraph(4, np.array([0, 1, 2], np.int32),
                                               np.array([1, 2, 3], np.int32), np.array([1, 2, 3], np.int64))
    k = 9
    src, dst = zip(*[(a, b) for a in range(k) for b in range(k) if a != b])
    src = np.array(src, np.int32)
    dst = np.array(dst, np.int32)
    out["complete_all_t_equal"] = W.TemporalGraph(k, src, dst, np.full(src.shape, 77, np.int64))
    rng = np.random.default_rng(3)
    hub_n = 300
    hs = np.concatenate([np.zeros(hub_n - 1, np.int32), rng.integers(1, hub_n, 3000).astype(np.int32)])
    hd = np.concatenate([np.arange(1, hub_n, dtype=np.int32), rng.integers(1, hub_n, 3000).astype(np.int32)])
    out["hub"] = W.TemporalGraph(hub_n, hs, hd, rng.integers(0, 50, hs.shape[0]).astype(np.int64))
    out["sigma_one"] = W.random_small_graph(np.random.default_rng(8), 400, 400, 10 ** 6, self_loops=False)
    dup = W.random_small_graph(np.random.default_rng(9), 10, 40, 5)
    out["duplicates"] = W.TemporalGraph(10, np.tile(dup.src, 3), np.tile(dup.dst, 3), np.tile(dup.t, 3))
    iso = W.random_small_graph(np.random.default_rng(10), 8, 60, 20)
    out["isolated_vertices"] = W.TemporalGraph(1000, iso.src, iso.dst, iso.t)
    big_t = W.random_small_graph(np.random.default_rng(11), 8, 80, 20)
    out["large_timestamps"] = W.TemporalGraph(8, big_t.src, big_t.dst,
                                              big_t.t + np.int64((1 << 62) - 100))
    return out


@pytest.mark.parametrize("name", sorted(_edge_case_graphs().keys()))
def test_edge_cases(F, name):
    g = _edge_case_graphs()[name]
    deltas = (0, 5, (1 << 62) - 1)
    _check_graph(F, g, _full_mix(deltas))




def test_int64_timestamp_store(F):
    """The 64-bit timestamp store (time span at least 2^32 - 1), single queries and the
    batch, against the oracle, with windows below and above 2^32."""
    for seed in (13, 14, 15):
        g = wide_time_span_graph(seed)
        assert int(g.t.max() - g.t.min()) >= (1 << 32)
        qs = _full_mix(WIDE_DELTAS)
        res, _ = _lib_results(F, g, qs)
        bat, _ = _lib_results(F, g, qs, batch=True)
        with oracle.OracleGraph.of(g) as og:
            hits = 0
            for q, r, rb in zip(qs, res, bat):
                want = og.query(q)
                _assert_same(r, want, str(q))
                _assert_same(rb, want, str(q))
                hits += int(want["edge_count"].sum())
        assert hits > 0
        # windows on either side of 2^32 both find triangles, and not the same ones
        with oracle.OracleGraph.of(g) as og:
            below, _ = og.counts(1 << 31, W.DIR_EITHER)
            above, _ = og.counts(1 << 33, W.DIR_EITHER)
        assert below.sum() > 0 and (above > below).any()


def _core_numbers(n, src, dst):
    """Batagelj-Zaversnik bucket algorithm (textbook, sequential)."""
    nb = [set() for _ in range(n)]
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            nb[a].add(b)
            nb[b].add(a)
    deg = [len(x) for x in nb]
    md = max(deg) if deg else 0
    bins = [0] * (md + 1)
    for d in deg:
        bins[d] += 1
    start = 0
    for d in range(md + 1):
        bins[d], start = start, start + bins[d]
    pos = [0] * n
    vert = [0] * n
    for v in range(n):
        pos[v] = bins[deg[v]]
        vert[pos[v]] = v
        bins[deg[v]] += 1
    for d in range(md, 0, -1):
        bins[d] = bins[d - 1]
    if md >= 0:
        bins[0] = 0
    for i in range(n):
        v = vert[i]
        for u in nb[v]:
            if deg[u] > deg[v]:
                du, pu = deg[u], pos[u]
                pw = bins[du]
                w = vert[pw]
                if u != w:
                    pos[u], vert[pu] = pw, w
                    pos[w], vert[pw] = pu, u
                bins[du] += 1
                deg[u] -= 1
    return deg


def test_degeneracy_and_orientation(F):
    rng = np.random.default_rng(12)
    # the first four fit the cluster tail from the start; the last two run grid-wide
    # levels first (more than 163,840 vertices alive) and reach hubs in the tail
    for g in (W.config_graph(1), W.random_small_graph(rng, 120, 5000, 10),
              W.config_graph(3, scale=0.002), W.config_graph(2, scale=0.05), W.config_graph(2, scale=0.2),
              W.config_graph(2, scale=0.5)):
        core = _core_numbers(g.n, g.src, g.dst)
        with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
            info = G.info()
            got = G.core_numbers()
        np.testing.assert_array_equal(got, np.asarray(core, dtype=np.int32))
        assert info["degeneracy"] == max(core)
        assert info["max_out_degree"] <= info["degeneracy"]
        loops = int((g.src == g.dst).sum())
        assert info["m_kept"] == g.m - loops


def test_batch_equals_sequential(F):
    g = W.config_graph(2, scale=0.01)
    rng = np.random.default_rng(4)
    qs = W.random_query_mix(40, rng, want_edge_counts=True)
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        seq = [G.query(q) for q in qs]
        bat = G.query_batch(qs)
    for q, a, b in zip(qs, seq, bat):
        np.testing.assert_array_equal(a["edge_count"], b["edge_count"])
        assert pairs_of(a) == pairs_of(b), str(q)


def test_batch_with_a_hub_of_degree_past_16_bits(F):
    """A vertex with 66,000 neighbours: counts no longer fit 16-bit counters, so single
    queries and the batch keep 32-bit ones; results equal each other and the oracle's."""
    rng = np.random.default_rng(12)
    n, leaves = 70_000, 66_000
    src = [np.zeros(leaves, np.int32)]
    dst = [np.arange(1, leaves + 1, dtype=np.int32)]
    a = rng.integers(1, 3000, 40_000).astype(np.int32)  # edges among low leaves: triangles with the hub
    b = rng.integers(1, 3000, 40_000).astype(np.int32)
    src.append(a)
    dst.append(b)
    src, dst = np.concatenate(src), np.concatenate(dst)
    t = rng.integers(0, 5000, src.shape[0]).astype(np.int64)
    o = np.argsort(t, kind="stable")
    g = W.TemporalGraph(n, src[o], dst[o], t[o])
    qs = [W.Query(d, 1, 10, W.Q_FORALL_T, dr, W.U_COMMON, True) for d in (5, 100, 2000) for dr in (W.DIR_OUT, W.DIR_EITHER)]
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        assert G.info()["max_degree"] >= 65535
        seq = [G.query(q) for q in qs]
        bat = G.query_batch(qs)
    with oracle.OracleGraph.of(g) as og:
        for q, a1, b1 in zip(qs, seq, bat):
            want = og.query(q)
            _assert_same(a1, want, str(q))
            _assert_same(b1, want, str(q))


def _pairs_from_counts(src, dst, counts, common, deg, n, q):
    """Solution pairs of query q among the given temporal edges, from their counts and
    common-neighbour numbers (both the oracle's) and the degrees of G_S, written out from
    Definition 1.1 and the pair reading (max count, number of certificates) with numpy:
    the check of a pair list on a subset of heads."""
    keep = src != dst
    x, y = src[keep].astype(np.int64), dst[keep].astype(np.int64)
    c, cm = counts[keep].astype(np.int64), common[keep].astype(np.int64)
    U = {W.U_HEAD: deg[x], W.U_TAIL: deg[y], W.U_COMMON: cm}[q.universe]
    sat = (c >= 1) & ((q.quant == W.Q_EXISTS) | (c * q.rho_den >= q.rho_num * U))
    key = x * n + y
    order = np.argsort(key, kind="stable")
    key, c, sat = key[order], c[order], sat[order]
    starts = np.concatenate([[0], np.nonzero(np.diff(key))[0] + 1])
    mx = np.maximum.reduceat(c, starts) if len(key) else c
    nc = np.add.reduceat(sat.astype(np.int64), starts) if len(key) else c
    k0 = key[starts] if len(key) else key
    sel = nc > 0
    return [(int(a // n), int(a % n), int(b), int(d)) for a, b, d in zip(k0[sel], mx[sel], nc[sel])]


def _degrees(g):
    """|N(u)| in G_S from the input edge list (distinct unordered pairs, no self-loops)."""
    keep = g.src != g.dst
    lo = np.minimum(g.src, g.dst)[keep].astype(np.int64)
    hi = np.maximum(g.src, g.dst)[keep].astype(np.int64)
    key = np.unique(lo * g.n + hi)
    return np.bincount(np.concatenate([key // g.n, key % g.n]), minlength=g.n).astype(np.int64)


@pytest.fixture(scope="module")
def medium_full():
    return W.config_graph(2)


def test_full_size_medium_workload(F, medium_full):
    """The medium workload at full size (1M vertices, 20M edges), the benchmark's three
    queries: every per-edge count and the whole sorted pair list against the oracle."""
    g = medium_full
    qs = [W.Query(d, 1, 2, want_edge_counts=True) for d in (600, 3600, 86400)]
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        res = [G.query(q) for q in qs]
        bat = G.query_batch(qs)
        info = G.info()
    assert info["m"] == g.m and info["probes"] > 10 ** 7
    hits = 0
    with oracle.OracleGraph.of(g) as og:
        for q, r, rb in zip(qs, res, bat):
            want = og.query(q)
            _assert_same(r, want, str(q))
            _assert_same(rb, want, str(q))
            hits += int((want["edge_count"] > 0).sum())
    # a static edge's times span about a day of a year, so few triangles meet a window
    assert hits > 0


@pytest.fixture(scope="module")
def paper_full():
    return W.config_graph(3)


def test_full_size_paper_scale_workload(F, paper_full):
    """The paper-scale workload at full size (5M vertices, 70M temporal edges, 50 planted
    dense communities, degeneracy about 200, 77M triangles): its query (delta = 3600 s,
    rho = 3/10) compared in full -- all 70M per-edge counts, the whole sorted pair list,
    the certificate total -- plus two more query variants on sampled edges and on the
    complete pair lists of sampled heads, and the batch of all three against the singles."""
    g = paper_full
    q0 = W.config_queries(3)[0]
    q0 = W.Query(q0.delta, q0.rho_num, q0.rho_den, q0.quant, q0.dir, q0.universe, True)
    extra = [W.Query(86400, 1, 10, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, True),
             W.Query(604800, 1, 2, W.Q_EXISTS, W.DIR_IN, W.U_TAIL, True)]
    qs = [q0] + extra
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        info = G.info()
        res = [G.query(q) for q in qs]
        bat = G.query_batch(qs)
        a, b, cab = F.folty_graph_common_counts(G.handle)
        core = G.core_numbers()
    assert info["m"] == 70_000_000 and info["triangles"] > 5 * 10 ** 7 and info["degeneracy"] >= 150
    # core numbers vertex by vertex against the textbook bucket algorithm on G_S's edges
    keep = g.src != g.dst
    pk = np.unique(np.minimum(g.src, g.dst)[keep].astype(np.int64) * g.n + np.maximum(g.src, g.dst)[keep])
    core_want = np.asarray(_core_numbers(g.n, pk // g.n, pk % g.n), dtype=np.int32)
    np.testing.assert_array_equal(core, core_want)
    assert info["degeneracy"] == int(core_want.max())
    for r, rb in zip(res, bat):
        np.testing.assert_array_equal(r["edge_count"], rb["edge_count"])
        assert pairs_of(r) == pairs_of(rb)
    rng = np.random.default_rng(33)
    with oracle.OracleGraph.of(g) as og:
        want = og.query(q0)
        _assert_same(res[0], want, str(q0))
        assert int((want["edge_count"] > 0).sum()) > 1000
        deg = _degrees(g)
        skey = a.astype(np.int64) * g.n + b

        def common_of(idx):
            lo = np.minimum(g.src[idx], g.dst[idx]).astype(np.int64)
            hi = np.maximum(g.src[idx], g.dst[idx]).astype(np.int64)
            return cab[np.searchsorted(skey, lo * g.n + hi)].astype(np.int64)

        by_src = np.argsort(g.src, kind="stable")
        src_sorted = g.src[by_src]
        for q, r in zip(extra, res[1:]):
            ec = r["edge_count"]
            idx = np.unique(np.concatenate([rng.integers(0, g.m, 5000), np.argsort(ec)[-500:]]))
            got, common = og.counts(q.delta, q.dir, idx=idx)
            np.testing.assert_array_equal(ec[idx], got, err_msg=str(q))
            np.testing.assert_array_equal(common_of(idx), common)
            # complete pair lists of sampled heads: solution heads and uniform vertices
            heads = np.unique(np.concatenate([rng.choice(r["u"], size=min(20, len(r["u"])), replace=False),
                                              rng.choice(np.unique(g.src), size=20, replace=False)]))
            for x in heads.tolist():
                lo, hi = np.searchsorted(src_sorted, [x, x + 1])
                e = by_src[lo:hi]
                c, cm = og.counts(q.delta, q.dir, idx=e)
                want_pairs = _pairs_from_counts(g.src[e], g.dst[e], c, cm, deg, g.n, q)
                sel = r["u"] == x
                got_pairs = list(zip(r["u"][sel].tolist(), r["v"][sel].tolist(), r["count"][sel].tolist(),
                                     r["ncert"][sel].tolist()))
                assert got_pairs == want_pairs, (str(q), x)


def test_errors(F):
    bad = W.TemporalGraph(3, np.array([0, 5], np.int32), np.array([1, 1], np.int32),
                          np.array([0, 0], np.int64))
    with pytest.raises(F.FoltyError) as ei:
        F.folty_load_temporal_graph(bad.n, bad.src, bad.dst, bad.t)
    assert ei.value.status == F.FOLTY_EINVAL
    neg = W.TemporalGraph(3, np.array([0], np.int32), np.array([1], np.int32), np.array([-4], np.int64))
    with pytest.raises(F.FoltyError) as ei:
        F.folty_load_temporal_graph(neg.n, neg.src, neg.dst, neg.t)
    assert ei.value.status == F.FOLTY_EINVAL
    g = W.config_graph(1)
    h = F.folty_load_temporal_graph(g.n, g.src, g.dst, g.t)
    try:
        with pytest.raises(F.FoltyError) as ei:
            F.folty_query(h, W.Query(10))
        assert ei.value.status == F.FOLTY_ESTATE
        F.folty_preprocess(h)
        with pytest.raises(F.FoltyError) as ei:
            F.folty_preprocess(h)
        assert ei.value.status == F.FOLTY_ESTATE
        for q in (W.Query(-1), W.Query(10, 3, 2), W.Query(10, 1, 0), W.Query(1 << 62)):
            with pytest.raises(F.FoltyError) as ei:
                F.folty_query(h, q)
            assert ei.value.status == F.FOLTY_EINVAL
        with pytest.raises(F.FoltyError) as ei:
            F.folty_query_batch(h, [W.Query(10), W.Query(10, 1, 0)])
        assert ei.value.status == F.FOLTY_EINVAL
    finally:
        F.folty_free(h)


def test_allocator_failure_reports_enomem_without_leak(F):
    import ctypes

    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    live = {}
    budget = {"calls": 0}

    @F.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        budget["calls"] += 1
        if budget["calls"] > 6:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        live[p] = nbytes
        return p

    @F.FREE_FN
    def free(ptr, stream, ctx):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    a = F.folty_allocator(alloc, free, None)
    g = W.config_graph(1)
    h = ctypes.c_void_p()
    st = F.lib.folty_load_temporal_graph(g.n, g.m, g.src.ctypes.data, g.dst.ctypes.data,
                                         g.t.ctypes.data, ctypes.byref(a), F.current_stream(),
                                         ctypes.byref(h))
    if st == F.FOLTY_OK:
        st = F.lib.folty_preprocess(h, F.current_stream())
        assert st == F.FOLTY_ENOMEM, F.folty_last_error()
        F.folty_free(h)
    else:
        assert st == F.FOLTY_ENOMEM
    torch.cuda.synchronize()
    assert not live, "every allocation must be returned"
    assert torch.cuda.memory_allocated() == base


def test_kernel_launch_counter_moves(F):
    g = W.config_graph(1)
    before = F.folty_kernel_launches()
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        G.query(W.Query(3600))
    assert F.folty_kernel_launches() > before + 10


def _outer_mix(deltas):
    qs = []
    for d in deltas:
        for quant in (W.Q_FORALL_T, W.Q_EXISTS):
            for num1, den1 in ((0, 1), (1, 10), (1, 3), (1, 1)):
                qs.append(W.Query(d, 1, 3, quant, W.DIR_OUT if num1 % 2 else W.DIR_EITHER, W.U_TAIL, False,
                                  outer=W.OUTER_FORALL_T, outer_rho_num=num1, outer_rho_den=den1,
                                  want_certificates=True))
    return qs


@pytest.mark.parametrize("which", ["tiny", "config1", "medium_small"])
def test_vertex_queries_and_certificates(F, which):
    rng = np.random.default_rng(31)
    if which == "tiny":
        graphs = [W.random_small_graph(rng, 12, 80, 20) for _ in range(5)]
        deltas = (0, 4, 30)
    elif which == "config1":
        graphs = [W.config_graph(1)]
        deltas = (100_000, 1_000_000)
    else:
        graphs = [W.config_graph(2, scale=0.01)]
        deltas = (3600, 604_800)
    for g in graphs:
        qs = _outer_mix(deltas)
        res, _ = _lib_results(F, g, qs)
        bat, _ = _lib_results(F, g, qs, batch=True)
        with oracle.OracleGraph.of(g) as og:
            for q, r, rb in zip(qs, res, bat):
                want = og.query(q)
                for got in (r, rb):
                    assert pairs_of(got) == pairs_of(want), str(q)
                    assert vertices_of(got) == vertices_of(want), str(q)
                    np.testing.assert_array_equal(got["certificates"], want["certificates"])
                    assert got["n_cert_edges"] == len(want["certificates"])


def test_common_neighbour_counts(F):
    for g in (W.config_graph(1), W.config_graph(3, scale=0.002)):
        with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
            a, b, c = F.folty_graph_common_counts(G.handle)
        keep = g.src != g.dst
        lo = np.minimum(g.src, g.dst)[keep].astype(np.int64)
        hi = np.maximum(g.src, g.dst)[keep].astype(np.int64)
        key = np.unique(lo * g.n + hi)
        np.testing.assert_array_equal(a.astype(np.int64) * g.n + b, key)
        # one input edge per static edge: the oracle's |N(x) cap N(y)|
        first = {}
        for i in np.nonzero(keep)[0]:
            k = int(min(g.src[i], g.dst[i])) * g.n + int(max(g.src[i], g.dst[i]))
            first.setdefault(k, int(i))
        idx = np.array([first[int(k)] for k in key], dtype=np.int64)
        with oracle.OracleGraph.of(g) as og:
            _, common = og.counts(0, W.DIR_OUT, idx=idx)
        np.testing.assert_array_equal(c, common)


@pytest.mark.parametrize("which", ["tiny", "config1", "medium_small"])
def test_all_existential_triples(F, which):
    """Definition 1.2 with three existential quantifiers: the (x, y, w) solutions, sorted,
    against the oracle, for every direction variant, alone and inside a batch."""
    rng = np.random.default_rng(41)
    if which == "tiny":
        graphs = [W.random_small_graph(rng, 14, 120, 25) for _ in range(6)]
        deltas = (0, 3, 40)
    elif which == "config1":
        graphs = [W.config_graph(1)]
        deltas = (100_000, 1_000_000)
    else:
        graphs = [W.config_graph(2, scale=0.01)]
        deltas = (600, 86_400)
    for g in graphs:
        qs = [W.Query(d, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, False, want_triples=True)
              for d in deltas for dr in (W.DIR_OUT, W.DIR_IN, W.DIR_EITHER)]
        mixed = qs + [W.Query(deltas[-1], 1, 2, W.Q_EXISTS, W.DIR_OUT, W.U_HEAD, True)]
        res, _ = _lib_results(F, g, qs)
        bat, _ = _lib_results(F, g, mixed, batch=True)
        with oracle.OracleGraph.of(g) as og:
            for q, r, rb in zip(qs, res, bat):
                want = og.triples(q.delta, q.dir)
                for got in (r, rb):
                    np.testing.assert_array_equal(got["triples"], want, err_msg=str(q))
                    assert pairs_of(got) == pairs_of(og.query(q)), str(q)
            want_last = og.query(mixed[-1])
            assert pairs_of(bat[-1]) == pairs_of(want_last)
            assert "triples" not in bat[-1]


def test_full_key_sort_path(F, monkeypatch):
    """The pair sort without dense pair ids (the 64-bit pair key with the input index as
    the value), which the library takes when its pair table cannot serve; forced here."""
    monkeypatch.setenv("FOLTY_PAIR_SORT", "keys")
    rng = np.random.default_rng(91)
    for n, m, tmax in ((12, 60, 25), (60, 6000, 3000), (300, 30000, 100000)):
        g = W.random_small_graph(rng, n, m, tmax, self_loops=True)
        _check_graph(F, g, _full_mix((0, 40, 700)))
        perm = rng.permutation(g.m)  # an edge list not in time order
        g2 = W.TemporalGraph(g.n, g.src[perm], g.dst[perm], g.t[perm])
        _check_graph(F, g2, _full_mix((40,)))
    monkeypatch.delenv("FOLTY_PAIR_SORT")
    g = W.config_graph(2, scale=0.01)
    perm = rng.permutation(g.m)
    _check_graph(F, W.TemporalGraph(g.n, g.src[perm], g.dst[perm], g.t[perm]),
                 [W.Query(3600, 1, 2, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True)])


def _many_pairs_graph(seed=5):
    """Over 2^20 distinct pairs (random pairs of 200K vertices) plus a dense block of 200
    vertices with many triangles, in time order."""
    rng = np.random.default_rng(seed)
    n, m1, m2 = 200_000, 1_150_000, 60_000
    src = rng.integers(0, n, m1 + m2).astype(np.int32)
    dst = rng.integers(0, n, m1 + m2).astype(np.int32)
    block = rng.choice(n, 200, replace=False).astype(np.int32)
    src[m1:] = block[rng.integers(0, 200, m2)]
    dst[m1:] = block[rng.integers(0, 200, m2)]
    t = rng.integers(0, 10 ** 6, m1 + m2).astype(np.int64)
    t[m1:] = rng.integers(0, 20_000, m2)
    o = np.argsort(t, kind="stable")
    return W.TemporalGraph(n, src[o], dst[o], t[o])


def test_pair_table_past_its_first_size(F):
    """More distinct pairs than the pair table's first size holds: the library retries
    with a larger table (or sorts full keys); results are the oracle's either way."""
    import torch
    g = _many_pairs_graph()
    qs = [W.Query(d, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, True) for d in (50, 2000) for dr in (W.DIR_OUT, W.DIR_EITHER)]
    qs.append(W.Query(500, 1, 10, W.Q_FORALL_T, W.DIR_IN, W.U_COMMON, True))
    info = _check_graph(F, g, qs)
    assert info["static_edges"] > (1 << 20)
    # device-resident input: the load fills the table's first try, which overflows too
    want, _ = _lib_results(F, g, qs)
    with F.TemporalGraph(g.n, *[torch.from_numpy(a).cuda() for a in (g.src, g.dst, g.t)]) as G:
        got, dinfo = [G.query(q) for q in qs], G.info()
    assert dinfo == info
    for q, a, b in zip(qs, want, got):
        _assert_same(b, a, what=str(q))



def test_triangle_layouts_agree(F, monkeypatch):
    """Past the allocation-free entry point's size limit the listing runs once, into a
    layout bounded per oriented edge by min(|N+(u)|, |N+(v)|), and a copy makes it dense;
    FOLTY_TRI_LAYOUT=counted forces the counting pass before it. Both layouts give the
    same triangle statistics and query results (the first matches the oracle in
    test_pair_table_past_its_first_size), the all-existential triples included."""
    g = _many_pairs_graph()
    qs = [W.Query(d, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, True) for d in (50, 2000) for dr in (W.DIR_OUT, W.DIR_EITHER)]
    qs.append(W.Query(500, 1, 2, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, False, want_triples=True))
    want, info = _lib_results(F, g, qs)
    assert info["static_edges"] > (1 << 20) and info["triangles"] > 10 ** 5
    monkeypatch.setenv("FOLTY_TRI_LAYOUT", "counted")
    got, cinfo = _lib_results(F, g, qs)
    # the bounded layout's array holds the bound's entries: more device memory
    assert cinfo.pop("device_bytes") < info.pop("device_bytes")
    assert cinfo == info
    for q, a, b in zip(qs, want, got):
        _assert_same(b, a, what=str(q))
    np.testing.assert_array_equal(got[-1]["triples"], want[-1]["triples"])
    assert len(want[-1]["triples"]) > 0

def _clique_graph(k=20000, size=4, seed=6):
    """k disjoint cliques of `size` vertices, one temporal edge per ordered pair, times
    within 20 s: every ordered pair of a clique has witnesses, so a query has up to
    k * size * (size - 1) solution pairs."""
    rng = np.random.default_rng(seed)
    a, b = zip(*[(i, j) for i in range(size) for j in range(size) if i != j])
    base = (np.arange(k, dtype=np.int32) * size)[:, None]
    src = (base + np.array(a, np.int32)[None, :]).ravel()
    dst = (base + np.array(b, np.int32)[None, :]).ravel()
    t = rng.integers(0, 20, src.shape[0]).astype(np.int64)
    o = np.argsort(t, kind="stable")
    return W.TemporalGraph(k * size, src[o], dst[o], t[o])


def test_pair_lists_past_the_pinned_stage(F):
    """Pair lists longer than the pinned stage that small results come back through
    (2^16 pairs per read-back, shared by a batch's queries) take the copy-out path;
    short and long lists in one batch, single and batched, equal the oracle's."""
    g = _clique_graph()
    qs = [W.Query(100, 1, 2, W.Q_EXISTS, W.DIR_OUT, W.U_HEAD, True),
          W.Query(100, 1, 3, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, True),
          W.Query(3, 1, 1, W.Q_FORALL_T, W.DIR_IN, W.U_TAIL, True),
          W.Query(1, 1, 2, W.Q_EXISTS, W.DIR_OUT, W.U_HEAD, True),
          W.Query(0, 1, 1, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True)]
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        seq = [G.query(q) for q in qs]
        bat = G.query_batch(qs)
    with oracle.OracleGraph.of(g) as og:
        want = [og.query(q) for q in qs]
    sizes = [len(w["u"]) for w in want]
    assert max(sizes) > (1 << 16) and 0 < sorted(sizes)[2] < (1 << 16) // len(qs)
    for q, a1, b1, w in zip(qs, seq, bat, want):
        _assert_same(a1, w, str(q))
        _assert_same(b1, w, str(q))


def _plain(qs):
    return [dataclasses.replace(q, want_edge_counts=False, want_certificates=False, outer=W.OUTER_NONE) for q in qs]


def _assert_pairs(lib_res, ora_res, what=""):
    assert pairs_of(lib_res) == pairs_of(ora_res), what
    assert lib_res["n_cert_edges"] == ora_res["n_cert_edges"], what


def _long_run_graph(seed=17):
    """Ordered pairs with 31, 32, 33, 40, 64, 65 and 100 temporal edges each among 16
    vertices (runs shorter and longer than a warp's 32 lanes), times on a small range."""
    rng = np.random.default_rng(seed)
    src, dst = [], []
    sizes = (1, 31, 32, 33, 40, 64, 65, 100)
    for a in range(16):
        for b in range(16):
            if a != b and rng.random() < 0.6:
                k = int(rng.choice(sizes))
                src += [a] * k
                dst += [b] * k
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    t = rng.integers(0, 2000, src.shape[0]).astype(np.int64)
    o = np.argsort(t, kind="stable")
    return W.TemporalGraph(16, src[o], dst[o], t[o])


@pytest.mark.parametrize("which", ["tiny", "long_runs", "config1", "medium_small"])
def test_batch_of_plain_queries_against_the_oracle(F, which):
    """The fused batched threshold (queries without per-edge outputs): one pass over the
    bins per direction variant for all queries, pairs and certificate totals equal the
    oracle's; repeated deltas, every quantifier, universe and direction variant."""
    rng = np.random.default_rng(51)
    if which == "tiny":
        graphs = [W.random_small_graph(rng, int(rng.integers(3, 14)), int(rng.integers(10, 120)), 25)
                  for _ in range(6)]
        deltas = (0, 1, 3, 7, 40)
    elif which == "long_runs":
        graphs = [_long_run_graph(17), _long_run_graph(18)]
        deltas = (0, 5, 60, 400, 3000)
    elif which == "config1":
        graphs = [W.config_graph(1)]
        deltas = (3600, 100_000, 1_000_000)
    else:
        graphs = [W.config_graph(2, scale=0.01)]
        deltas = (600, 3600, 86400, 604800)
    for g in graphs:
        qs = _plain(_full_mix(deltas)) + W.random_query_mix(40, rng)
        qs += [W.Query(deltas[-1], k, 10, W.Q_FORALL_T, W.DIR_OUT, W.U_COMMON, False) for k in (0, 3, 10)]
        bat, _ = _lib_results(F, g, qs, batch=True)
        with oracle.OracleGraph.of(g) as og:
            for q, r in zip(qs, bat):
                _assert_pairs(r, og.query(q), str(q))
                assert r["edge_count"] is None or len(r["edge_count"]) == 0


def test_batch_more_queries_than_one_fused_pass(F, monkeypatch):
    """More than 256 plain queries of one direction variant (several fused passes over the
    same bins), with a first solution buffer too small for the pass (a second pass with
    room for all), mixed with queries that want per-edge counts (the prefix path)."""
    monkeypatch.setenv("FOLTY_BATCH_SOLUTION_CAP", "7")
    g = W.config_graph(2, scale=0.01)
    rng = np.random.default_rng(52)
    qs = [dataclasses.replace(q, dir=W.DIR_OUT) for q in W.random_query_mix(300, rng)]
    qs += [W.Query(86400, 1, 2, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True),
           W.Query(604800, 1, 5, W.Q_EXISTS, W.DIR_EITHER, W.U_TAIL, True)]
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        bat = G.query_batch(qs)
        seq = [G.query(q) for q in qs]
    for q, a, b in zip(qs, seq, bat):
        _assert_pairs(b, a, str(q))
        if q.want_edge_counts:
            np.testing.assert_array_equal(a["edge_count"], b["edge_count"])
    assert sum(len(r["u"]) for r in bat) > 7
    with oracle.OracleGraph.of(g) as og:
        for i in rng.choice(len(qs), 25, replace=False):
            _assert_pairs(bat[i], og.query(qs[i]), str(qs[i]))


def test_batch_of_plain_queries_with_32_bit_bins_and_long_lists(F):
    """Plain batched queries with 32-bit bins (a hub of degree past 2^16) and with solution
    lists longer than the pinned stage (the copy-out path of the fused pass)."""
    rng = np.random.default_rng(12)
    n, leaves = 70_000, 66_000
    src = np.concatenate([np.zeros(leaves, np.int32), rng.integers(1, 3000, 40_000).astype(np.int32)])
    dst = np.concatenate([np.arange(1, leaves + 1, dtype=np.int32), rng.integers(1, 3000, 40_000).astype(np.int32)])
    t = rng.integers(0, 5000, src.shape[0]).astype(np.int64)
    o = np.argsort(t, kind="stable")
    hub = W.TemporalGraph(n, src[o], dst[o], t[o])
    qs = [W.Query(d, 1, 10, W.Q_FORALL_T, dr, W.U_COMMON, False) for d in (5, 100, 2000)
          for dr in (W.DIR_OUT, W.DIR_EITHER)] + [W.Query(3000, 1, 2, W.Q_EXISTS, W.DIR_IN, W.U_HEAD, False)]
    clique = _clique_graph()
    qc = [W.Query(100, 1, 2, W.Q_EXISTS, W.DIR_OUT, W.U_HEAD, False),
          W.Query(100, 1, 3, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON, False),
          W.Query(3, 1, 1, W.Q_FORALL_T, W.DIR_IN, W.U_TAIL, False)]
    for g, queries in ((hub, qs), (clique, qc)):
        bat, info = _lib_results(F, g, queries, batch=True)
        with oracle.OracleGraph.of(g) as og:
            want = [og.query(q) for q in queries]
        for q, r, w in zip(queries, bat, want):
            _assert_pairs(r, w, str(q))
    assert max(len(w["u"]) for w in want) > (1 << 16)


def test_plain_single_queries_through_captured_plans(F, monkeypatch):
    """Plain single queries replay a CUDA graph captured once per graph and query shape,
    with the window and rho in a device parameter block: results equal the oracle's and,
    bit for bit, those of the same queries launched one kernel at a time
    (FOLTY_QUERY_GRAPHS=0); several windows and rhos replay each shape."""
    rng = np.random.default_rng(61)
    graphs = [W.random_small_graph(rng, 12, 90, 20) for _ in range(3)]
    graphs += [W.config_graph(1), W.config_graph(2, scale=0.01), wide_time_span_graph(15), _long_run_graph(19),
               _clique_graph()]
    for g in graphs:
        span = int(g.t.max() - g.t.min()) if g.m else 1
        deltas = sorted({0, 3, max(1, span // 50), max(1, span // 5), span + 1})
        qs = [W.Query(d, k, 10, quant, dr, uni, False) for d in deltas
              for (k, quant, dr, uni) in ((5, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD), (1, W.Q_EXISTS, W.DIR_IN, W.U_TAIL),
                                          (3, W.Q_FORALL_T, W.DIR_EITHER, W.U_COMMON),
                                          (9, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD))]
        with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
            before = F.folty_kernel_launches()
            got = [G.query(q) for q in qs]
            assert F.folty_kernel_launches() > before
            monkeypatch.setenv("FOLTY_QUERY_GRAPHS", "0")
            ref = [G.query(q) for q in qs]
            monkeypatch.delenv("FOLTY_QUERY_GRAPHS")
            again = [G.query(q) for q in reversed(qs)][::-1]
        with oracle.OracleGraph.of(g) as og:
            for q, a, b, c in zip(qs, got, ref, again):
                for k in ("u", "v", "count", "ncert"):
                    np.testing.assert_array_equal(a[k], b[k], err_msg=str(q))
                    np.testing.assert_array_equal(c[k], b[k], err_msg=str(q))
                assert a["n_cert_edges"] == b["n_cert_edges"] == c["n_cert_edges"]
                _assert_pairs(a, og.query(q), str(q))


def test_autotuned_shapes_give_identical_results(F):
    """Every kernel shape the autotuner may pick (thread-versus-warp split of the triangle
    passes, probe tile and grid) gives the same per-edge counts, pairs, batch results and
    triangle statistics; a tuned graph records its trial times, and a second graph of the
    same statistics takes its shapes from the cache."""
    import torch
    rng = np.random.default_rng(71)
    graphs = [W.config_graph(2, scale=0.02), W.config_graph(3, scale=0.004), _long_run_graph(20)]
    shapes = [(24, 4, 0), (48, 8, 0), (96, 8, 2), (1 << 30, 4, 4), (1, 4, 1)]
    for g in graphs:
        qs = [W.Query(d, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, True) for d in (600, 86400, 10 ** 7)
              for dr in (W.DIR_OUT, W.DIR_EITHER)]
        plain = _plain(qs) + W.random_query_mix(12, rng)
        outs = []
        try:
            for sh in shapes:
                F.folty_tuning_force(*sh)
                with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
                    t = F.folty_graph_tuning(G.handle)
                    assert (t["tri_heavy"], t["tri_source"]) == (sh[0], "forced")
                    res = [G.query(q) for q in qs] + [G.query(q) for q in plain] + G.query_batch(plain)
                    t = F.folty_graph_tuning(G.handle)
                    assert (t["probe_items"], t["probe_blocks_per_sm"]) == sh[1:]
                    outs.append((res, G.info()))
        finally:
            F.folty_tuning_force(0, 0, 0)
        base, info = outs[0]
        for res, inf in outs[1:]:
            assert inf["triangles"] == info["triangles"] and inf["probes"] == info["probes"]
            for a, b in zip(base, res):
                assert pairs_of(a) == pairs_of(b) and a["n_cert_edges"] == b["n_cert_edges"]
                if a["edge_count"] is not None:
                    np.testing.assert_array_equal(a["edge_count"], b["edge_count"])
    # tuned by trials once, then from the cache
    F.folty_tuning_clear_cache()
    g = graphs[0]
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        G.query(W.Query(3600))
        t1 = F.folty_graph_tuning(G.handle)
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        G.query(W.Query(3600))
        t2 = F.folty_graph_tuning(G.handle)
    assert t1["tri_source"] == "timed trials" and t1["probe_source"] == "timed trials"
    assert all(x > 0 for x in t1["tri_trial_ms"]) and all(x > 0 for x in t1["probe_trial_ms"])
    assert t2["tri_source"] == "cache" and t2["probe_source"] == "cache"
    assert (t2["tri_heavy"], t2["probe_items"], t2["probe_blocks_per_sm"]) == \
        (t1["tri_heavy"], t1["probe_items"], t1["probe_blocks_per_sm"])
    with pytest.raises(F.FoltyError):
        F.folty_tuning_force(48, 5, 0)
