"""folty_edge_counts_noalloc: per-edge counts of one query with no allocation inside the
library, checked against folty_query through the C ABI.

Callers that cannot allocate device memory at query time -- a serving process that
reserved its memory budget at start-up, latency-bound code that must not run into the
implicit device synchronisation of cudaMalloc/cudaFree, a host whose allocator must not
be re-entered from a library call -- use this entry point; its working counters live in
one file-scope device array shared by every call. This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_17215_gb300 as F
    return F


def _counting_allocator(F, calls):
    import torch

    @F.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    @F.FREE_FN
    def free(ptr, stream, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    return F.folty_allocator(alloc, free, None), (alloc, free)


def _load(F, g, a):
    h = ctypes.c_void_p()
    st = F.lib.folty_load_temporal_graph(g.n, g.m, g.src.ctypes.data, g.dst.ctypes.data, g.t.ctypes.data,
                                         ctypes.byref(a), F.current_stream(), ctypes.byref(h))
    assert st == F.FOLTY_OK, F.folty_last_error()
    F.folty_preprocess(h.value)
    return h.value


def test_noalloc_counts_equal_query_counts_on_calls_in_a_row(F):
    import torch
    g = W.config_graph(2, scale=0.04)  # 40,000 vertices, 800,000 edges
    calls = {"alloc": 0, "free": 0}
    a, keep = _counting_allocator(F, calls)
    h = _load(F, g, a)
    try:
        assert F.folty_graph_get_info(h)["m_kept"] <= F.NOALLOC_MAX_EDGES
        cases = [(3600, W.DIR_OUT), (86400, W.DIR_EITHER), (3600, W.DIR_OUT), (600, W.DIR_IN)]
        outs = [torch.full((g.m,), -7, dtype=torch.int32, device="cuda") for _ in cases]
        torch.cuda.synchronize()
        before = dict(calls)
        for (delta, dr), out in zip(cases, outs):  # consecutive calls, no synchronisation between
            F.folty_edge_counts_noalloc(h, delta, dr, out)
        torch.cuda.synchronize()
        assert calls == before, "the allocation-free path must not call the allocator"
        for (delta, dr), out in zip(cases, outs):
            want = F.folty_query(h, W.Query(delta, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, True))["edge_count"]
            np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert int(outs[1].max()) > 0
    finally:
        F.folty_free(h)
    del keep


def test_noalloc_rejects_graphs_above_its_limit(F):
    import torch
    g = W.config_graph(2, scale=0.06)  # 1,200,000 edges > 2^20
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        assert G.info()["m_kept"] > F.NOALLOC_MAX_EDGES
        out = torch.zeros(g.m, dtype=torch.int32, device="cuda")
        with pytest.raises(F.FoltyError) as ei:
            F.folty_edge_counts_noalloc(G.handle, 3600, W.DIR_OUT, out)
        assert ei.value.status == F.FOLTY_EINVAL
        assert "at most" in str(ei.value)


def test_noalloc_on_the_64_bit_timestamp_store(F):
    """A time span past 2^32 keeps 64-bit timestamps; windows below and above 2^32."""
    import torch
    from _support import WIDE_DELTAS, wide_time_span_graph
    g = wide_time_span_graph(14)
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        for delta in WIDE_DELTAS:
            for dr in (W.DIR_OUT, W.DIR_IN, W.DIR_EITHER):
                out = torch.full((g.m,), -7, dtype=torch.int32, device="cuda")
                F.folty_edge_counts_noalloc(G.handle, delta, dr, out)
                want = G.query(W.Query(delta, 1, 2, W.Q_FORALL_T, dr, W.U_HEAD, True))["edge_count"]
                np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_noalloc_refuses_buffers_it_cannot_write(F):
    """Host arrays, the wrong dtype or a short buffer are refused by the binding; host
    memory handed to the C entry point directly is refused by the library (FOLTY_EINVAL)
    before any kernel runs."""
    import torch
    g = W.config_graph(1)
    with F.TemporalGraph(g.n, g.src, g.dst, g.t) as G:
        with pytest.raises(TypeError):
            F.folty_edge_counts_noalloc(G.handle, 3600, W.DIR_OUT, np.zeros(g.m, np.int32))
        with pytest.raises(TypeError):
            F.folty_edge_counts_noalloc(G.handle, 3600, W.DIR_OUT, torch.zeros(g.m, dtype=torch.int64, device="cuda"))
        with pytest.raises(ValueError):
            F.folty_edge_counts_noalloc(G.handle, 3600, W.DIR_OUT, torch.zeros(g.m - 1, dtype=torch.int32, device="cuda"))
        for host in (np.zeros(g.m, np.int32), torch.zeros(g.m, dtype=torch.int32).pin_memory()):
            ptr = host.ctypes.data if isinstance(host, np.ndarray) else host.data_ptr()
            st = F.lib.folty_edge_counts_noalloc(G.handle, 3600, W.DIR_OUT, ptr, F.current_stream())
            assert st == F.FOLTY_EINVAL, F.folty_last_error()
            assert "device memory" in F.folty_last_error()
        # the graph still answers afterwards
        out = torch.zeros(g.m, dtype=torch.int32, device="cuda")
        F.folty_edge_counts_noalloc(G.handle, 10 ** 6, W.DIR_OUT, out)
        want = G.query(W.Query(10 ** 6, 1, 2, W.Q_FORALL_T, W.DIR_OUT, W.U_HEAD, True))["edge_count"]
        np.testing.assert_array_equal(out.cpu().numpy(), want)
