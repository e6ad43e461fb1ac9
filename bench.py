#!/usr/bin/env python
"""Benchmark of the temporal-graph triadic query path on GB300.

Workload (default, "paper"): the paper-scale synthetic temporal graph -- 5,000,000
vertices, 70,000,000 temporal edges, Chung-Lu exponent 2.0 plus 50 planted
300-vertex communities (intra-pair probability 0.7), Zipf(1.3) multiplicities (capped at
10,000, 16 inside the communities), bursty lognormal timestamps over one year -- and its
query exists u exists v forall_{3/10} w in N(u) with delta = 3600 s ("out" motif).
"--workload medium" runs the medium graph (1,000,000 vertices, 20,000,000 edges) and its
three queries (delta in {600, 3600, 86400} s, rho = 1/2) instead.

One step = the whole path on one batch of input: load (copy + validation),
preprocessing (sort, static graph, peeling, orientation, triangle listing, role summary)
and the workload's queries (selection, probes, counts, threshold, solution pairs back on
the host).

value    = (queries x temporal edges) per second of whole steps, over all ranks, inputs
           resident in HBM when the timed region starts (device CUDA-event time);
query    = the per-query metric m / t_query: device time of folty_query alone on a
           preprocessed graph (preprocessing reported beside it as preprocess_ms);
e2e      = the same steps through the C ABI from pinned host buffers: host->device copy
           of the edge list and device->host copy of the results inside every step;
roofline = the step's dominant stage (largest device time per step): model bytes per
           span over its CUDA-event duration against the measured HBM peak;
query_roofline = the same for the dominant stage of the query path.

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
WORKLOADS = {
    "paper": (3, "paper-scale synthetic temporal graph: n=5,000,000, m=70,000,000, Chung-Lu gamma=2.0 plus 50 "
                 "planted 300-vertex communities (p=0.7), Zipf(1.3) multiplicity capped at 10,000 (16 inside "
                 "the communities), bursty lognormal(6,2) times over 1 year; query exists-exists-forall_{3/10} "
                 "over N(u), delta=3600 s", "3/10"),
    "medium": (2, "medium synthetic temporal graph: n=1,000,000, m=20,000,000, Chung-Lu gamma=2.1, "
                  "Zipf(1.5) multiplicity capped at 1000, bursty lognormal(6,2) times over 1 year; "
                  "3 queries exists-exists-forall_{1/2} over N(u), delta in {600,3600,86400} s", "1/2"),
}

STAGE_KERNELS = {
    "probe": "k_probe_live (persistent window probes over the kept roles)",
    "select": "k_live_sums + k_live_offsets + k_live_write (selection of the kept triangles by their liveness bytes)",
    "sort": "radix sort spans: k_rs_hist_all + k_rs_bases (all digit histograms), or one k_rs_onesweep digit pass",
    "peel": "k_peel (cooperative) + k_tail_* + k_peel_tail + k_solo_* + k_peel_solo",
    "threshold": "k_threshold",
    "triangles": "k_tri_bound + k_tri_write (one pass into the bounded layout; k_tri_count first on small graphs)",
    "roles": "k_run_ends + k_tri_live_copy (liveness bytes while the triangles move to the dense layout)",
    "batch": "k_batch_threshold",
    "store": "temporal store beside the peel: k_store_ids, k_store_hist, the id sort's k_rs_onesweep passes "
             "(contains sort spans)",
}
STAGE_SOURCES = {"probe": ("live.cu", "probe.cuh"), "select": ("live.cu", "scan.cuh"), "sort": ("prims.cu",),
                 "peel": ("preprocess.cu",), "threshold": ("query.cu",), "triangles": ("preprocess.cu",),
                 "roles": ("live.cu", "liveness.cuh"), "batch": ("batch.cu",), "store": ("preprocess.cu", "prims.cu")}
QUERY_STAGES = ("select", "probe", "threshold")


def stage_traffic(stage, workload):
    """DRAM bytes per span of a stage from the committed ncu summary of the workload, when
    it was taken on the current sources (profiles/traffic_<workload>_workload.md lists
    'traffic <stage> <bytes> <sha256 of the stage's sources>'); None otherwise."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}_workload.md")
    if not os.path.exists(path):
        return None
    for m in re.finditer(r"^traffic (\w+) (\d+) ([0-9a-f]{64})$", open(path).read(), re.M):
        if m.group(1) != stage:
            continue
        return int(m.group(2)) if source_hash(stage) == m.group(3) else None
    return None


def source_hash(stage):
    import hashlib
    h = hashlib.sha256()
    for f in STAGE_SOURCES.get(stage, ()):
        h.update(open(os.path.join(ROOT, "paper_2507_17215_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


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

class OracleArm:
    """The CPU oracle on the host cores: its edge lists and neighbourhoods are built once
    for the whole graph (timed), then every sample draws temporal edges uniformly and
    computes their counts for each query; a step's time is extrapolated as the build plus
    the per-edge time times all edges and queries."""

    def __init__(self, g):
        import oracle
        self.oracle = oracle
        self.g = g
        t0 = time.perf_counter()
        self.og = oracle.OracleGraph.of(g)
        self.build_s = time.perf_counter() - t0
        self.cores = oracle.threads()

    def step_seconds(self, queries, budget_s: float, seed: int = 0):
        g = self.g
        rng = np.random.default_rng(seed)
        size = 4000
        t0 = time.perf_counter()
        for q in queries:
            self.og.counts(q.delta, q.dir, idx=rng.integers(0, g.m, size))
        per = (time.perf_counter() - t0) / (size * len(queries))
        size = int(min(g.m, max(size, budget_s / max(per, 1e-9) / len(queries))))
        t0 = time.perf_counter()
        for q in queries:
            self.og.counts(q.delta, q.dir, idx=rng.integers(0, g.m, size))
        eval_s = time.perf_counter() - t0
        per = eval_s / (size * len(queries))
        step_s = self.build_s + per * g.m * len(queries)
        sample = (f"oracle build on all {g.m} edges ({self.build_s:.1f} s, once) + per-edge counts of "
                  f"{size} uniformly drawn edges x {len(queries)} queries ({eval_s:.1f} s), extrapolated "
                  f"to all edges")
        return step_s, sample

    def close(self):
        self.og.close()


def run_reference(args, g, queries, workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    arm = OracleArm(g)
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        step_s, sample = arm.step_seconds(queries, budget_s=args.ref_budget, seed=i)
        if i >= args.warmup:
            vals.append(step_s)
    arm.close()
    mean_s = sum(vals) / len(vals)
    value = len(queries) * g.m / mean_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[workload][1], "queries": len(queries), "m": g.m, "n": g.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": arm.cores, "kind": "oracle",
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


def measure_batch(F, g, sh, nq, stream, reps=3):
    """nq mixed queries (delta log-uniform on [60 s, 7 d], rho = k/10, quantifier and
    direction uniform) on the preprocessed graph: folty_query_batch against nq
    back-to-back folty_query calls, results compared pair list by pair list."""
    import torch
    rng = np.random.default_rng(4)
    qs = W.random_query_mix(nq, rng)
    d = [torch.from_numpy(a).cuda() for a in (g.src, g.dst, g.t)]
    h = F.folty_load_temporal_graph(g.n, *d, stream=sh)
    try:
        F.folty_preprocess(h, sh)
        del d
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
        F.folty_profile_enable(True)
        F.folty_query_batch(h, qs, sh)
        prof = F.folty_profile_read()
        F.folty_profile_enable(False)
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
    stages = {k: {"ms": v["ms"], "spans": v["launches"], "model_bytes": v["bytes"]}
              for k, v in prof.items() if v["launches"]}
    return {"queries": nq, "workload": "medium graph, mixed queries (delta log-uniform 60 s..7 d, "
            "rho k/10, exists/forall, out/in/either, universe N(u))",
            "batch_ms": bm, "sequential_ms": seq_ms, "speedup": seq_ms / bm,
            "edges_per_s": nq * g.m / (bm / 1e3), "results_equal": bool(same),
            "solution_pairs_total": int(sum(len(r["u"]) for r in res_b)), "stages": stages}


def stage_table(prof, steps, peak):
    out = {}
    for name, p in prof.items():
        if p["launches"] == 0 or p["ms"] <= 0:
            continue
        gbs = p["bytes"] / (p["ms"] / 1e3) / 1e9
        out[name] = {"ms_per_step": p["ms"] / steps, "spans_per_step": p["launches"] / steps,
                     "model_bytes_per_span": p["bytes"] / p["launches"],
                     "ms_per_span": p["ms"] / p["launches"], "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def roofline_of(prof, stage, peak, peak_kind, workload):
    d = prof[stage]
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": stage_traffic(stage, workload), "stage": stage, "kernel": STAGE_KERNELS[stage],
            "peak_kind": f"{peak_kind} hbm_gbs (of {peak_kind})",
            "model_bytes_per_launch": d["bytes"] / d["launches"], "launch_ms": d["ms"] / d["launches"]}


def time_queries(F, g, d_src, d_dst, d_t, sh, stream, queries, reps=10):
    """Load and preprocessing alone (events around each call, median of 3), then every
    query of the workload alone on the preprocessed graph (median of reps), and what each
    query's probe pass keeps."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    load_ms, pre_ms = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        ev[0].record(stream)
        h = F.folty_load_temporal_graph(g.n, d_src, d_dst, d_t, stream=sh)
        ev[1].record(stream)
        F.folty_preprocess(h, sh)
        ev[2].record(stream)
        torch.cuda.synchronize()
        load_ms.append(ev[0].elapsed_time(ev[1]))
        pre_ms.append(ev[1].elapsed_time(ev[2]))
        F.folty_free(h)
    h = F.folty_load_temporal_graph(g.n, d_src, d_dst, d_t, stream=sh)
    F.folty_preprocess(h, sh)
    info = F.folty_graph_get_info(h)
    q_ms = []
    kept = []
    for q in queries:
        F.folty_query(h, q, sh)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev[0].record(stream)
            F.folty_query(h, q, sh)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        q_ms.append(float(np.median(ts)))
        st = F.folty_graph_probe_stats(h, q.delta, q.dir, sh)
        kept.append({"delta": q.delta, "kept_triangles": st["kept_triangles"], "kept_roles": st["kept_roles"],
                     "kept_probes": st["kept_probes"], "all_probes": st["all_probes"],
                     "kept_probe_fraction": st["kept_probes"] / max(st["all_probes"], 1),
                     "kept_role_fraction": st["kept_roles"] / max(st["all_roles"], 1),
                     "select_model_bytes": st["select_bytes"], "probe_model_bytes": st["probe_bytes"]})
    tm = F.folty_graph_traffic_model(h, W.DIR_OUT, sh)
    tuning = F.folty_graph_tuning(h)
    F.folty_free(h)
    return {"load_ms": float(np.median(load_ms)), "preprocess_ms": float(np.median(pre_ms)),
            "query_ms": q_ms, "kept": kept, "info": info, "all_roles_probe_model_bytes": tm["probe_bytes"],
            "tuning": tuning}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="folty", choices=["folty", "reference"])
    ap.add_argument("--workload", default="paper", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=2.0,
                    help="seconds of sampled oracle evaluation per step")
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (debug only)")
    ap.add_argument("--batch", type=int, default=256,
                    help="queries of the batched measurement on the medium graph (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the serving measurement (0 = skip)")
    ap.add_argument("--no-medium", action="store_true",
                    help="skip the medium graph's step figures when the workload is the paper-scale one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    cfg_k, cfg_desc, rho_txt = WORKLOADS[args.workload]
    g = W.config_graph(cfg_k, scale=args.scale)
    queries = [W.Query(q.delta, q.rho_num, q.rho_den, q.quant, q.dir, q.universe, False)
               for q in W.config_queries(cfg_k)]
    if args.impl == "reference":
        run_reference(args, g, queries, args.workload)
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

    # ---- per-query figures (the metric m / t_query), preprocessing alone, kept roles
    qt = time_queries(F, g, d_src, d_dst, d_t, sh, stream, queries)
    info = qt["info"]

    # ---- end-to-end through the C ABI from pinned host buffers
    ke = args.e2e_steps if args.e2e_steps is not None else min(args.steps, 20)
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
    del d_src, d_dst, d_t, h_src, h_dst, h_t

    # ---- the medium graph's step (when the headline is the paper-scale one), the batch
    # and the serving measurements (both over medium-recipe graphs)
    medium = None
    g2 = None
    if (args.batch > 0 or (args.workload != "medium" and not args.no_medium)) and world == 1:
        g2 = W.config_graph(2, scale=args.scale)
    if args.workload != "medium" and not args.no_medium and world == 1:
        q2 = [W.Query(q.delta, q.rho_num, q.rho_den, q.quant, q.dir, q.universe, False) for q in W.config_queries(2)]
        s2 = [torch.from_numpy(a).cuda() for a in (g2.src, g2.dst, g2.t)]

        def step2():
            h = F.folty_load_temporal_graph(g2.n, *s2, stream=sh)
            try:
                F.folty_preprocess(h, sh)
                return [F.folty_query(h, q, sh) for q in q2]
            finally:
                F.folty_free(h)

        for _ in range(3):
            step2()
        torch.cuda.synchronize()
        n2 = 20
        ev0.record(stream)
        for _ in range(n2):
            step2()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms2 = ev0.elapsed_time(ev1) / n2
        qt2 = time_queries(F, g2, *s2, sh, stream, q2)
        medium = {"workload": WORKLOADS["medium"][1], "ms_per_step": ms2,
                  "edges_per_s": len(q2) * g2.m / (ms2 / 1e3), "load_ms": qt2["load_ms"],
                  "preprocess_ms": qt2["preprocess_ms"], "query_ms": qt2["query_ms"],
                  "query_edges_per_s": [g2.m / (x / 1e3) for x in qt2["query_ms"]],
                  "kept": qt2["kept"], "triangles": qt2["info"]["triangles"], "degeneracy": qt2["info"]["degeneracy"]}
        del s2
    batched = None
    if args.batch > 0 and world == 1:
        batched = measure_batch(F, g2, sh, args.batch, stream)
    serving = None
    if args.serve_seconds > 0 and world == 1:
        serving = measure_serving(F, args.serve_seconds)

    peak, peak_kind = _peaks()
    stages = stage_table(prof, prof_steps, peak)
    roofline = query_roofline = None
    if stages:
        # the store span contains sort spans and runs beside the peel: not a stage of its own
        dom = max((k for k in stages if k != "store"), key=lambda k: stages[k]["ms_per_step"])
        roofline = roofline_of(prof, dom, peak, peak_kind, args.workload)
        if dom == "peel":
            roofline["note"] = (f"the peel is bound by the latency of its dependent rounds ({info['peel_rounds']} "
                                "on this graph: grid, cluster and single-CTA phases), not by bandwidth; its model "
                                "bytes are tiny, so the fraction is near zero by construction")
        qs_ = [k for k in QUERY_STAGES if k in stages]
        if qs_:
            qdom = max(qs_, key=lambda k: stages[k]["ms_per_step"])
            query_roofline = roofline_of(prof, qdom, peak, peak_kind, args.workload)
    q_ms = qt["query_ms"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": cfg_desc, "n": g.n, "m": g.m, "queries": len(queries),
                   "deltas": [q.delta for q in queries], "rho": rho_txt, "universe": "N(u)",
                   "motif": "out", "parallelism": f"replicas x{world}",
                   "l2": f"inputs ({g.m * 16 // 10**6} MB) and timestamp store larger than the 129 MB L2",
                   "static_edges": info["static_edges"], "triangles": info["triangles"],
                   "probes_per_query_all_roles": info["probes"], "degeneracy": info["degeneracy"],
                   "max_degree": info["max_degree"], "sigma_max": info["sigma_max"],
                   "peel_rounds": info["peel_rounds"], "solution_pairs": [len(r["u"]) for r in res]},
        "query": {"metric": "m / t_query (device time of folty_query alone, preprocessing excluded)",
                  "query_ms": q_ms, "edges_per_s": [g.m / (x / 1e3) for x in q_ms],
                  "load_ms": qt["load_ms"], "preprocess_ms": qt["preprocess_ms"], "kept": qt["kept"],
                  "all_roles_probe_model_bytes": qt["all_roles_probe_model_bytes"],
                  "note": "the probe stage's algorithmic bytes count the kept roles only (kept_* and "
                          "probe_model_bytes per query); all_roles_probe_model_bytes is the model of probing "
                          "every role, which the liveness selection avoids"},
        "tuning": qt["tuning"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "query_roofline": query_roofline,
        "stages": stages,
        "clocks": clk,
        "medium": medium,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        arm = OracleArm(g)
        step_s, sample = arm.step_seconds(queries, budget_s=args.ref_budget)
        arm.close()
        line["cpu_baseline"] = {"value": len(queries) * g.m / step_s, "unit": UNIT, "cores": arm.cores,
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
