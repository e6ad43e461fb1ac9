#!/usr/bin/env python
"""Benchmark of the temporal-graph triadic query path on GB300.

Workload (default): the medium synthetic temporal graph -- 1,000,000 vertices,
20,000,000 temporal edges, Chung-Lu exponent 2.1, Zipf(1.5) multiplicities capped at
1000, bursty lognormal timestamps over one year -- and its three queries
exists u exists v forall_{1/2} w in N(u) with delta in {600, 3600, 86400} s ("out"
motif). One step = the whole path on one batch of input: load (copy + validation),
preprocessing (sort, static graph, peeling, orientation, triangle listing) and the
three queries (probes, counts, threshold, solution pairs back on the host).

value  = (queries x temporal edges) processed per second over all ranks, inputs
         resident in HBM when the timed region starts (device CUDA-event time);
e2e    = the same through the C ABI from pinned host buffers: host->device copy of the
         edge list and device->host copy of the results inside every step;
roofline = the window-probe kernel, model bytes per launch / its event-timed duration.

Multi-GPU: every rank runs its own replica of the workload (the query path has no
exchange step); value sums the ranks' work over the slowest rank's time.

--impl reference times the CPU oracle (test infrastructure; plain C + OpenMP) on the
host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "temporal edges/s per FOL triadic query on 1xGB300"
UNIT = "temporal edges/s"
WORKLOAD = ("medium synthetic temporal graph: n=1,000,000, m=20,000,000, Chung-Lu gamma=2.1, "
            "Zipf(1.5) multiplicity capped at 1000, bursty lognormal(6,2) times over 1 year; "
            "3 queries exists-exists-forall_{1/2} over N(u), delta in {600,3600,86400} s")


STAGE_KERNELS = {
    "probe": "window-probe stage: k_live_tri, scans, k_live_compact, k_live_tiles, k_probe_live",
    "sort": "radix sort spans: k_rs_hist_all + k_rs_bases (all digit histograms), or one k_rs_onesweep digit pass",
    "peel": "k_peel (cooperative) + k_tail_* + k_peel_tail",
    "threshold": "k_threshold",
}


def stage_traffic(stage, model_bytes):
    """DRAM bytes per span of a stage from the committed ncu summary, when it was taken
    on the current sources (profiles/traffic_medium_workload.md lists 'traffic <stage>
    <bytes> <sha256 of the stage's sources>'); None otherwise."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "traffic_medium_workload.md")
    if not os.path.exists(path):
        return None
    for m in re.finditer(r"^traffic (\w+) (\d+) ([0-9a-f]{64})$", open(path).read(), re.M):
        if m.group(1) != stage:
            continue
        h = hashlib.sha256()
        for f in STAGE_SOURCES.get(stage, ()):
            h.update(open(os.path.join(ROOT, "paper_2507_17215_gb300", "csrc", f), "rb").read())
        return int(m.group(2)) if h.hexdigest() == m.group(3) else None
    return None


STAGE_SOURCES = {"probe": ("live.cu", "probe.cuh"), "sort": ("prims.cu",),
                 "peel": ("preprocess.cu",), "threshold": ("query.cu",)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running; start()
    returns once the first sample is in, mark() opens the timed region, and stop() summarises
    the samples taken after mark() (the last earlier one when none came after it)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.time() + 5.0
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.first:] or self.lines[max(0, self.first - 1):self.first]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample_time(g, queries, budget_s: float, seed: int = 0):
    """Oracle on a bounded sample: full build of its edge lists and neighbourhoods, then
    the per-edge counts of uniformly drawn temporal edges for every query. Returns the
    extrapolated seconds for the whole step and a description."""
    import oracle
    t0 = time.perf_counter()
    og = oracle.OracleGraph.of(g)
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    size = 4000
    t0 = time.perf_counter()
    for q in queries:
        og.counts(q.delta, q.dir, idx=rng.integers(0, g.m, size))
    calib = time.perf_counter() - t0
    per = calib / (size * len(queries))
    size = int(min(g.m, max(size, budget_s / max(per, 1e-9) / len(queries))))
    t0 = time.perf_counter()
    for q in queries:
        og.counts(q.delta, q.dir, idx=rng.integers(0, g.m, size))
    eval_s = time.perf_counter() - t0
    og.close()
    per = eval_s / (size * len(queries))
    step_s = build_s + per * g.m * len(queries)
    sample = (f"oracle build on all {g.m} edges ({build_s:.1f} s) + per-edge counts of "
              f"{size} uniformly drawn edges x {len(queries)} queries ({eval_s:.1f} s), "
              f"extrapolated to all edges")
    return step_s, sample, oracle.threads()


def run_reference(args, g, queries):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    sample = ""
    cores = 1
    for i in range(args.warmup + args.steps):
        step_s, sample, cores = oracle_sample_time(g, queries, budget_s=args.ref_budget, seed=i)
        if i >= args.warmup:
            vals.append(step_s)
    mean_s = sum(vals) / len(vals)
    value = len(queries) * g.m / mean_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "queries": len(queries), "m": g.m, "n": g.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- ranks

def max_over_ranks(x: float, world: int, device: str) -> float:
    """Slowest rank's figure (all_reduce MAX); identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Weak scaling over replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ----------------------------------------------------------------------------- GPU arm

SERVE_SIZES = (100_000, 500_000, 1_000_000, 2_000_000, 5_000_000, 10_000_000, 15_000_000, 20_000_000)


def measure_serving(F, seconds, rate=200.0, sizes=SERVE_SIZES, seed=5):
    """Poisson arrivals (rate per second) of mixed queries over resident graphs of the
    medium recipe (n = m / 20), each query for a uniformly drawn graph; latency is
    arrival -> results on the host, as stamped by the server."""
    import queue as _queue
    gens = [W.medium_graph_of_size(m, 5000 + i) for i, m in enumerate(sizes)]
    handles = [F.TemporalGraph(g.n, g.src, g.dst, g.t, allocator=None) for g in gens]
    ms = [g.m for g in gens]
    del gens
    rng = np.random.default_rng(seed)
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        arrivals.append(t)
    qs = W.random_query_mix(len(arrivals), rng)
    gi = rng.integers(0, len(sizes), len(arrivals))
    sv = F.folty_server_create([h.handle for h in handles])
    try:
        for i in range(len(sizes)):  # warm-up: one query per graph
            F.folty_server_wait(sv, F.folty_server_submit(sv, i, qs[0]))
        pending = _queue.Queue()
        infos = []

        def collect():
            while True:
                item = pending.get()
                if item is None:
                    return
                res = F.folty_server_wait(sv, item[0])
                infos.append((res["info"], item[1]))

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for at, q, g in zip(arrivals, qs, gi):
            delay = t0 + at - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            pending.put((F.folty_server_submit(sv, int(g), q), int(g)))
        pending.put(None)
        th.join()
        elapsed = time.perf_counter() - t0
        stats = F.folty_server_get_stats(sv)
    finally:
        F.folty_server_destroy(sv)
        for h in handles:
            h.close()
    lat = np.array([inf["latency_ms"] for inf, _ in infos])
    edges = sum(ms[g] for _, g in infos)
    return {"workload": "8 resident graphs of the medium recipe, m in " + ",".join(str(m) for m in sizes)
            + "; Poisson arrivals, mixed queries", "seconds": seconds, "rate_qps": rate,
            "queries": len(infos), "throughput_qps": len(infos) / elapsed,
            "edges_per_s": edges / elapsed,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_batch": float(np.mean([inf["batch_size"] for inf, _ in infos])) if infos else None,
            "batches": stats["batches"], "max_batches_in_flight": stats["max_batches_in_flight"],
            "peak_memory_bytes": stats["peak_memory_bytes"]}


def measure_batch(F, g, d_src, d_dst, d_t, sh, nq, stream, reps=3):
    """nq mixed queries (delta log-uniform on [60 s, 7 d], rho = k/10, quantifier and
    direction uniform) on the preprocessed graph: folty_query_batch against nq
    back-to-back folty_query calls, results compared pair list by pair list."""
    import torch
    rng = np.random.default_rng(4)
    qs = W.random_query_mix(nq, rng)
    h = F.folty_load_temporal_graph(g.n, d_src, d_dst, d_t, stream=sh)
    try:
        F.folty_preprocess(h, sh)
        F.folty_query_batch(h, qs, sh)  # warm-up (allocator, module load)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        batch_ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev[0].record(stream)
            res_b = F.folty_query_batch(h, qs, sh)
            ev[1].record(stream)
            torch.cuda.synchronize()
            batch_ms.append(ev[0].elapsed_time(ev[1]))
        torch.cuda.synchronize()
        ev[0].record(stream)
        res_s = [F.folty_query(h, q, sh) for q in qs]
        ev[1].record(stream)
        torch.cuda.synchronize()
        seq_ms = ev[0].elapsed_time(ev[1])
    finally:
        F.folty_free(h)
    same = all(a["n_cert_edges"] == b["n_cert_edges"] and all(np.array_equal(a[k], b[k]) for k in
               ("u", "v", "count", "ncert")) for a, b in zip(res_b, res_s))
    bm = float(np.median(batch_ms))
    return {"queries": nq, "workload": "medium graph, mixed queries (delta log-uniform 60 s..7 d, "
            "rho k/10, exists/forall, out/in/either, universe N(u))",
            "batch_ms": bm, "sequential_ms": seq_ms, "speedup": seq_ms / bm,
            "edges_per_s": nq * g.m / (bm / 1e3), "results_equal": bool(same),
            "solution_pairs_total": int(sum(len(r["u"]) for r in res_b))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="folty", choices=["folty", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=4.0,
                    help="seconds of sampled oracle evaluation per step")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (debug only)")
    ap.add_argument("--batch", type=int, default=256,
                    help="queries of the batched measurement (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the serving measurement (0 = skip; 60 for the full run)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    g = W.config_graph(2, scale=args.scale)
    queries = [W.Query(q.delta, q.rho_num, q.rho_den, q.quant, q.dir, q.universe, False)
               for q in W.config_queries(2)]
    if args.impl == "reference":
        run_reference(args, g, queries)
        return

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import paper_2507_17215_gb300 as F

    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)
    d_src = torch.from_numpy(g.src).cuda()
    d_dst = torch.from_numpy(g.dst).cuda()
    d_t = torch.from_numpy(g.t).cuda()
    h_src = torch.from_numpy(g.src).pin_memory()
    h_dst = torch.from_numpy(g.dst).pin_memory()
    h_t = torch.from_numpy(g.t).pin_memory()
    torch.cuda.synchronize()

    def step(src, dst, t):
        h = F.folty_load_temporal_graph(g.n, src, dst, t, stream=sh)
        try:
            F.folty_preprocess(h, sh)
            out = [F.folty_query(h, q, sh) for q in queries]
        finally:
            F.folty_free(h)
        return out

    for _ in range(args.warmup):
        res = step(d_src, d_dst, d_t)
    # graph figures for the roofline (outside the timed region)
    h = F.folty_load_temporal_graph(g.n, d_src, d_dst, d_t, stream=sh)
    F.folty_preprocess(h, sh)
    info = F.folty_graph_get_info(h)
    tm = F.folty_graph_traffic_model(h, W.DIR_OUT, sh)
    F.folty_free(h)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = F.folty_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.mark()
    ev0.record(stream)
    for _ in range(args.steps):
        res = step(d_src, d_dst, d_t)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = F.folty_kernel_launches() - launches0
    clk = clocks.stop()
    t_ms = max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
    value = replica_throughput(args.steps * len(queries) * g.m, world, t_ms / 1e3)

    # ---- the same steps again with the library's per-stage CUDA events on (the
    # roofline's stage durations); kept out of the timed region above, whose host-side
    # event bookkeeping it would otherwise include
    prof_steps = max(1, min(args.steps, 10))
    F.folty_profile_enable(True)
    for _ in range(prof_steps):
        step(d_src, d_dst, d_t)
    torch.cuda.synchronize()
    prof = F.folty_profile_read()
    F.folty_profile_enable(False)

    # ---- batched queries: 256 mixed queries on the same graph vs one at a time
    batched = None
    if args.batch > 0:
        batched = measure_batch(F, g, d_src, d_dst, d_t, sh, args.batch, stream)

    serving = None
    if args.serve_seconds > 0 and world == 1:
        serving = measure_serving(F, args.serve_seconds)

    # ---- end-to-end through the C ABI from pinned host buffers
    ke = args.e2e_steps if args.e2e_steps is not None else args.steps
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_e = []
    for _ in range(ke):
        res_e = step(h_src, h_dst, h_t)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = replica_throughput(ke * len(queries) * g.m, world, e2e_s) if ke > 0 else None
    h2d = g.m * (4 + 4 + 8)
    d2h = sum(16 * len(r["u"]) + 8 for r in res_e) + 8 * (4 + 3 * 2)

    peak, peak_kind = _peaks()
    stages = {}
    for name, p in prof.items():
        if p["launches"] == 0 or p["ms"] <= 0:
            continue
        gbs = p["bytes"] / (p["ms"] / 1e3) / 1e9
        stages[name] = {"ms_per_step": p["ms"] / prof_steps, "spans_per_step": p["launches"] / prof_steps,
                        "model_bytes_per_span": p["bytes"] / p["launches"], "achieved_gbs": gbs,
                        "frac": gbs / peak}
    dom = max(stages, key=lambda k: stages[k]["ms_per_step"]) if stages else None
    roofline = None
    if dom is not None:
        d = prof[dom]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": stage_traffic(dom, d["bytes"] / d["launches"]),
                    "stage": dom, "kernel": STAGE_KERNELS[dom], "peak_kind": f"{peak_kind} hbm_gbs",
                    "model_bytes_per_launch": d["bytes"] / d["launches"],
                    "launch_ms": d["ms"] / d["launches"]}
        if dom == "peel":
            roofline["note"] = ("the peel is bound by the latency of its dependent rounds (304 on this graph: "
                                "grid, cluster and single-CTA phases), not by bandwidth; its model bytes are "
                                "tiny, so the fraction is near zero by construction. The sort, probe and "
                                "threshold stages in 'stages' are the bandwidth-bound ones")
    probe_ms = prof["probe"]["ms"] / max(prof["probe"]["launches"], 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "queries": len(queries),
                   "deltas": [q.delta for q in queries], "rho": "1/2", "universe": "N(u)",
                   "motif": "out", "parallelism": f"replicas x{world}",
                   "l2": "inputs (320 MB) and timestamp store larger than the 129 MB L2",
                   "static_edges": info["static_edges"], "triangles": info["triangles"],
                   "probes_per_query": info["probes"], "degeneracy": info["degeneracy"],
                   "peel_rounds": info["peel_rounds"], "solution_pairs": [len(r["u"]) for r in res],
                   "probe_ms_per_query": probe_ms,
                   "probe_model_bytes_all_roles": tm["probe_bytes"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "stages": stages,
        "clocks": clk,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        step_s, sample, cores = oracle_sample_time(g, queries, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": len(queries) * g.m / step_s, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
