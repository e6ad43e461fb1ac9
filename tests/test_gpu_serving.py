"""Serving: queries for several resident graphs submitted concurrently, batched per graph
by the server, must give exactly the results of folty_query alone on the same graph."""
import threading

import numpy as np
import pytest

import workloads as W
from _support import pairs_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_17215_gb300 as F
    return F


@pytest.fixture(scope="module")
def graphs(F):
    gs = [W.config_graph(1), W.medium_graph_of_size(200_000, 7), W.medium_graph_of_size(600_000, 8)]
    handles = [F.TemporalGraph(g.n, g.src, g.dst, g.t, allocator=None) for g in gs]
    yield handles
    for h in handles:
        h.close()


def _mix(rng, count):
    qs = W.random_query_mix(count, rng, want_edge_counts=False)
    return [W.Query(q.delta, q.rho_num, q.rho_den, q.quant, q.dir, int(rng.integers(0, 3)), False)
            for q in qs]


def _same(a, b):
    return pairs_of(a) == pairs_of(b) and a["n_cert_edges"] == b["n_cert_edges"]


def test_results_alone_equal_results_in_the_mix(F, graphs):
    rng = np.random.default_rng(21)
    jobs = [(int(rng.integers(0, len(graphs))), q) for q in _mix(rng, 150)]
    sv = F.folty_server_create([G.handle for G in graphs])
    try:
        tickets = [None] * len(jobs)

        def submit(part):
            for i in part:
                gi, q = jobs[i]
                tickets[i] = F.folty_server_submit(sv, gi, q)

        threads = [threading.Thread(target=submit, args=(range(k, len(jobs), 4),)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        got = [F.folty_server_wait(sv, t, timeout_ms=120_000) for t in tickets]
        stats = F.folty_server_get_stats(sv)
    finally:
        F.folty_server_destroy(sv)
    assert stats["queries"] == len(jobs)
    assert stats["batches"] < len(jobs), "queued queries must share batches"
    assert max(r["info"]["batch_size"] for r in got) > 1
    for (gi, q), r in zip(jobs, got):
        alone = graphs[gi].query(q)
        assert _same(r, alone), (gi, q)
        assert r["info"]["graph_index"] == gi
        assert r["info"]["latency_ms"] >= r["info"]["run_ms"] >= 0


def test_poisson_arrivals_results_equal_results_alone(F, graphs):
    """Queries arriving one by one at Poisson times (3,000 per second over 2 s, each for a
    uniformly drawn graph), submitted from one thread as they arrive and collected by
    another: every result equals folty_query alone, and queries that arrived while a batch
    ran were batched together."""
    import queue
    import time
    rng = np.random.default_rng(23)
    arrivals = np.cumsum(rng.exponential(1.0 / 3000.0, 6000))
    arrivals = arrivals[arrivals < 2.0]
    qs = _mix(rng, len(arrivals))
    gis = rng.integers(0, len(graphs), len(arrivals))
    sv = F.folty_server_create([G.handle for G in graphs])
    got = []
    try:
        pending = queue.Queue()

        def collect():
            while True:
                t = pending.get()
                if t is None:
                    return
                got.append(F.folty_server_wait(sv, t, timeout_ms=120_000))

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for at, q, gi in zip(arrivals, qs, gis):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            pending.put(F.folty_server_submit(sv, int(gi), q))
        pending.put(None)
        th.join()
        stats = F.folty_server_get_stats(sv)
    finally:
        F.folty_server_destroy(sv)
    assert len(got) == len(arrivals) and stats["queries"] == len(arrivals)
    assert max(r["info"]["batch_size"] for r in got) > 1
    alone = {}
    for q, gi, r in zip(qs, gis, got):
        assert r["info"]["graph_index"] == gi
        key = (int(gi), q)
        if key not in alone:
            alone[key] = graphs[int(gi)].query(q)
        assert _same(r, alone[key]), (gi, q)


def test_memory_budget_admits_one_query_at_a_time(F, graphs):
    rng = np.random.default_rng(22)
    jobs = [(int(rng.integers(0, len(graphs))), q) for q in _mix(rng, 30)]
    sv = F.folty_server_create([G.handle for G in graphs], memory_budget_bytes=1)
    try:
        tickets = [F.folty_server_submit(sv, gi, q) for gi, q in jobs]
        got = [F.folty_server_wait(sv, t) for t in tickets]
    finally:
        F.folty_server_destroy(sv)
    assert all(r["info"]["batch_size"] == 1 for r in got)
    for (gi, q), r in zip(jobs, got):
        assert _same(r, graphs[gi].query(q))


def test_ticket_errors(F, graphs):
    sv = F.folty_server_create([G.handle for G in graphs])
    try:
        with pytest.raises(F.FoltyError) as ei:
            F.folty_server_wait(sv, 987654, timeout_ms=0)
        assert ei.value.status == F.FOLTY_EINVAL
        t = F.folty_server_submit(sv, 0, W.Query(3600))
        F.folty_server_wait(sv, t, timeout_ms=60_000)
        with pytest.raises(F.FoltyError) as ei:
            F.folty_server_wait(sv, t, timeout_ms=0)  # collected already
        assert ei.value.status == F.FOLTY_EINVAL
        with pytest.raises(F.FoltyError) as ei:
            F.folty_server_submit(sv, len(graphs), W.Query(3600))
        assert ei.value.status == F.FOLTY_EINVAL
        with pytest.raises(F.FoltyError) as ei:
            F.folty_server_submit(sv, 0, W.Query(3600, 3, 2))
        assert ei.value.status == F.FOLTY_EINVAL
        # uncollected tickets are run and freed by destroy
        F.folty_server_submit(sv, 1, W.Query(600))
    finally:
        F.folty_server_destroy(sv)
