#!/usr/bin/env python
"""Benchmark of the GB300 optimal-cycle-mean solver.

One step = one complete solve (initial policy, every Howard iteration of
evaluation + improvement sweep, critical-cycle extraction) of the workload,
with its CSR graph already resident in HBM.  The default workload is the
largest single graph, locality32m (n = 2^25, m = 2.68e8, minimum cycle
mean).  The metric is edge-iterations per second: m * (number of improvement
sweeps) / solve time, summed over all GPUs for multi-GPU runs (each GPU solves
its own replica: one graph does not shard, so N > 1 is replicas only).

The same JSON line carries two sub-records for the other forms of the solver:
``batch4096`` (the batched form: graphs/s of one batched call against a loop
of the plain solver, every member compared with the oracle's stored answer;
sharded over the ranks by edge count when N > 1) and ``diff1m_grad`` (forward
+ backward against the finite-difference loop of plain solves).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference     # the CPU oracle on the same workload

Prints one JSON line (rank 0).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "edge-iters/s"
LOCALITY_LOG2 = [25]     # --locality-log2 (smaller sizes for profiling captures)
L2_FLUSH_BYTES = 256 << 20


BATCH_WORKLOADS = {
    "batch4096": (4096, 200000,
                  "4096 graphs, n_g log-uniform in [100, 200000], ring + U{0..7} extra edges, "
                  "w U[1,10000], max"),
    "batch4096-20k": (4096, 20000,
                      "4096 graphs, n_g log-uniform in [100, 20000], ring + U{0..7} extra edges, "
                      "w U[1,10000], max"),
}


def _workloads():
    return {
        "product4": (synth.product4,
                     "state-space product of 4 processes x 38-state rings + 2 chords/state, "
                     "BFS-numbered, 2,085,136 states, w U[0,1000], max"),
        "ring10k": (synth.ring10k, "ring + U{0..4} uniform extra edges, n=10,000, w U[1,100], max"),
        "locality32m": (lambda: synth.locality32m(1 << LOCALITY_LOG2[0]),
                        "locality graph n=2^25, deg 4/16/64, targets i+1+|N(0,4096)|, "
                        "w U[-1000,1000], min"),
        "diff1m": (synth.diff1m_base, "ring + U{0..7} extra edges, n=2^20, w 1024*U[0,1000], max"),
        "hub4m": (synth.hub4m, "ring + 3 uniform extra edges, n=2^20, one vertex with 4,000,000 more "
                               "(skewed degrees), w U[-1000,1000], max"),
    }


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.15)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# reference arm: the CPU oracle, as it stands
# --------------------------------------------------------------------------

def run_reference(args, g, desc):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    iters = args.ref_iters
    ms = []
    for step in range(args.warmup + args.steps):
        t = time.perf_counter()
        try:
            oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, max_iter=iters)
        except oracle.OracleError as e:
            if e.code != -5:
                raise
        dt = time.perf_counter() - t
        if step >= args.warmup:
            ms.append(dt * 1e3)
    t_step = sum(ms) / len(ms) / 1e3
    value = g.m * iters / t_step
    sample = (f"first {iters} Howard iterations (evaluation + improvement sweep each) of the "
              f"oracle on the full {args.workload} graph, per step")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edge-iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "n": g.n, "m": g.m, "mode": g.mode},
        "cpu_baseline": {"value": value, "unit": "edge-iters/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edge-iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def algorithmic_bytes(cls: str, n: int, m: int, launches: int) -> float:
    """Bytes a kernel class must move at least, summed over its launches.

    sweep:    row_ptr 4(n+1) + col_idx and w 8m + the record {V, rank} of
              every target vertex once 12n + the policy read and written 8n,
              i.e. 8m + 24n + 4 per sweep
    evaluate: floor of an O(n) evaluation of one policy, 40 B per vertex:
              policy edge, its target and weight read (12), root, value,
              rank and cycle flag written (28)
    """
    if cls == "sweep":
        return launches * (4.0 * (n + 1) + 8.0 * m + 12.0 * n + 8.0 * n)
    if cls == "evaluate":
        return launches * 40.0 * n
    return 0.0


CLASSES = ["init", "sweep", "evaluate", "extract"]

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from an
# ncu capture of the kernel, with the sha256 prefix of its sources at the time;
# reported only while the sources are unchanged.  The locality32m figures are
# taken on the same recipe at n = 2^23 (a capture of the full 2^25 graph holds
# too much device memory for ncu's save-and-restore passes) and scaled by 4,
# the ratio of the vertex and edge counts; the traffic of both kernels grows in
# proportion to n (evaluation) and n + m (sweep) once the graph exceeds L2.
KERNEL_SOURCES = {"evaluate": ("evaluate.cu", "grid_sync.cuh", "common.cuh"),
                  "sweep": ("sweep.cu", "common.cuh")}
TRAFFIC = {
    # n = 2^23 capture (launches from the middle of a solve, mean; the
    # evaluation's two launches, local_chunk_kernel + evaluate_local_kernel;
    # the sweep's full instance) x 4
    ("locality32m", "evaluate"): (4 * (0.067920e9 + 0.174084e9 + 0.191438e9 + 0.133894e9),
                                  "d516308f4f43a93f"),
    ("locality32m", "sweep"): (4 * (0.862757e9 + 0.122895e9), "7327f46a463627d3"),
}


def job_rate(units_per_step: float, steps: int, local_ms: float, world: int, device):
    """Whole-job rate of `world` replicas that each ran `steps` steps of
    `units_per_step` units in `local_ms` (their own timed region): the job
    took as long as its slowest rank (max over ranks), and its rate counts
    the units of all ranks.  Returns (rate per second, job milliseconds)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    job_ms = float(t.item())
    return world * steps * units_per_step / (job_ms / 1e3), job_ms


def _source_hash(kernel: str) -> str | None:
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1111_0627_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str):
    entry = TRAFFIC.get((workload, kernel))
    if entry is None or _source_hash(kernel) != entry[1]:
        return None
    return entry[0]


def _stored_answer(workload: str):
    """(num, den, cycle length, cycle digest) of the oracle's stored answer for
    a single-graph workload (tests/golden/oracle_values.txt, written by
    tests/golden/make_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_values.txt")
    try:
        with open(path) as f:
            for line in f:
                tok = line.split()
                if tok and tok[0] == workload:
                    kv = dict(t.split("=", 1) for t in tok[1:] if "=" in t)
                    return (int(kv["num"]), int(kv["den"]), int(kv["len"]),
                            int(kv["cycle_digest"]))
    except OSError:
        pass
    return None


def cpu_sample(g, workload: str, single: bool, iters: int) -> dict:
    """The oracle's first `iters` Howard iterations (evaluation + improvement
    sweep each) on the full graph, single-threaded: edge-iterations/s."""
    import oracle
    t0 = time.perf_counter()
    fn = oracle.howard_single if single else oracle.howard
    sweeps = iters
    try:
        h = fn(g.row_ptr, g.col_idx, g.w, g.mode, max_iter=iters)
        sweeps = h.iterations + 1          # converged inside the sample
    except oracle.OracleError as e:
        if e.code != -5:          # not converged within the sample: expected
            raise
    dt = time.perf_counter() - t0
    return {"value": g.m * sweeps / dt, "unit": "edge-iters/s", "cores": 1, "kind": "oracle",
            "sample": f"first {iters} Howard iterations of the oracle on the full {workload} graph "
                      f"({dt:.1f} s, single-threaded, initial pass included)"}


def run_ours(args, g, desc):
    import ctypes

    import torch
    import torch.distributed as dist

    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300 import _native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _native.load()
    stream = torch.cuda.current_stream(dev)

    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col_idx).to(dev)
    w = torch.from_numpy(g.w).to(dev)
    single = bool(args.single_lambda)
    ws = ocm.make_workspace(g.n, g.m, dev, single_lambda=single)
    cyc = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def solve(flags=0):
        return ocm.solve(rp, col, w, g.mode, workspace=ws, cycle_out=cyc, stream=stream,
                         flags=flags, single_lambda=single)

    for _ in range(args.warmup):
        sol = solve()
    sweeps = sol.stats["iterations"] + 1
    units = g.m * sweeps                    # edge-iterations per solve

    # ---- timed region: inputs resident, L2 flushed before every step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clocks:
        barrier()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            s = solve()
            ev[k][1].record(stream)
            launches += s.stats["launches"]
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value, total_ms = job_rate(units, args.steps, sum(step_ms), world, dev)

    # ---- the same solve with the loop driven from the host (one stream
    #      synchronisation per improvement step), for comparison only
    host_ms = []
    for k in range(min(args.steps, 5)):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solve(ocm.ocm.OCM_FLAG_HOST_LOOP)
        b.record(stream)
        b.synchronize()
        host_ms.append(a.elapsed_time(b))

    # ---- kernel-class durations (events around each launch), same workload
    prof_steps = max(1, min(args.steps, 5))
    lib.ocm_profile_enable(1)
    lib.ocm_profile_collect(None, None)
    for k in range(prof_steps):
        flush.fill_(k & 0xFF)
        solve()
    ms_arr = (ctypes.c_double * len(CLASSES))()
    n_arr = (ctypes.c_int64 * len(CLASSES))()
    lib.ocm_profile_collect(ms_arr, n_arr)
    lib.ocm_profile_enable(0)
    classes = {c: {"ms_total": ms_arr[i], "launches": int(n_arr[i])} for i, c in enumerate(CLASSES)}
    peak, peak_kind = _peaks()
    for c, d in classes.items():
        b = algorithmic_bytes(c, g.n, g.m, d["launches"])
        d["algorithmic_bytes"] = b
        d["gbs"] = (b / (d["ms_total"] / 1e3) / 1e9) if d["ms_total"] > 0 and b > 0 else None
    dom = max(classes, key=lambda c: classes[c]["ms_total"])

    def kernel_roofline(c):
        d = classes[c]
        achieved = d["gbs"]
        return {"bound": "hbm", "kernel": c, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                # (the counters were taken on the default form's launches)
                "traffic": None if single else measured_traffic(args.workload, c),
                "peak_kind": peak_kind,
                "avg_launch_us": d["ms_total"] * 1e3 / max(d["launches"], 1),
                "algorithmic_bytes_per_launch": d["algorithmic_bytes"] / max(d["launches"], 1)}

    # the dominant class, and the other of the two per-step classes beside it
    other = "sweep" if dom != "sweep" else "evaluate"
    rooflines = {dom: kernel_roofline(dom), other: kernel_roofline(other)}
    rooflines["sweep"]["note"] = ("averaged over every sweep of the solve: the frontier sweeps of "
                                  "the last iterations, which skip most vertices, count at the "
                                  "full sweep's algorithmic bytes; traffic is the full sweep's")
    if "evaluate" in rooflines:
        rooflines["evaluate"]["note"] = ("algorithmic bytes: the 40 B per vertex floor of one "
                                         "evaluation; both launches of the two-level form")
    roofline = rooflines[dom]
    share = {c: round(v["ms_total"] / max(sum(x["ms_total"] for x in classes.values()), 1e-12), 4)
             for c, v in classes.items()}

    # ---- end to end through the public API with host buffers
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_col = torch.from_numpy(g.col_idx).pin_memory()
    h_w = torch.from_numpy(g.w).pin_memory()
    h_cyc = torch.empty(g.n, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    d_rp, d_col, d_w = torch.empty_like(rp), torch.empty_like(col), torch.empty_like(w)
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(e2e_steps)]
    d2h = 0
    barrier()
    for k in range(e2e_steps):
        flush.fill_(k & 0xFF)
        e_ev[k][0].record(stream)
        d_rp.copy_(h_rp, non_blocking=True)
        d_col.copy_(h_col, non_blocking=True)
        d_w.copy_(h_w, non_blocking=True)
        s = ocm.solve(d_rp, d_col, d_w, g.mode, workspace=ws, cycle_out=cyc, stream=stream,
                      single_lambda=single)
        L = s.cycle.numel()
        h_cyc[:L].copy_(s.cycle, non_blocking=True)
        e_ev[k][1].record(stream)
        d2h = 4 * L + 16
    barrier()
    e2e_value, _ = job_rate(units, e2e_steps, sum(a.elapsed_time(b) for a, b in e_ev), world, dev)

    # ---- the answer against the oracle's stored answer for this graph
    stored = _stored_answer(args.workload if args.locality_log2 == 25 or
                            args.workload != "locality32m" else "")
    matches = None
    if stored is not None and not single:
        c = sol.cycle.cpu().numpy().astype(np.int32)
        matches = (sol.num, sol.den, int(c.shape[0]), synth.digest(c)) == stored

    # ---- CPU baseline: the oracle as it stands, rank 0 at N = 1, on a bounded
    #      sample of the same workload: its first Howard iterations on the
    #      full graph (about 10-30 s of one host core)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(g, args.workload, single, args.cpu_iters)

    # ---- the other forms of the solver, as sub-records of the same line
    sub = {}
    if args.subrecords:
        del rp, col, w, ws, cyc, d_rp, d_col, d_w
        torch.cuda.empty_cache()
        sub["batch4096"] = measure_batch(args, "batch4096", dev, world, rank, local,
                                         steps=min(args.steps, 5), compare_loop=world == 1)
        sub["diff1m_grad"] = measure_grad(args, dev, world, rank, steps=min(args.steps, 10))

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "edge-iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "n": g.n, "m": g.m,
                       "mode": g.mode, "sweeps_per_solve": sweeps,
                       "lambda": f"{sol.num}/{sol.den}", "critical_cycle_len": int(sol.cycle.numel()),
                       "matches_stored_oracle_answer": matches,
                       "l2": "flushed before every timed step (256 MiB write, outside the timing)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "step_ms_median": statistics.median(step_ms),
                       "step_ms_min": min(step_ms),
                       "loop": "cuda_graph" if sol.stats["graph_loop"] else "host",
                       "host_loop_ms_median": statistics.median(host_ms),
                       "iteration": ("single-lambda (Alg. 1 rebuild around the chosen cycle)"
                                     if single else "multichain (one mean per policy cycle)")},
            "roofline": roofline,
            "roofline_" + other: rooflines[other],
            "kernel_share": share,
            "kernels": {c: {"ms_per_solve": v["ms_total"] / prof_steps,
                            "launches_per_solve": v["launches"] / prof_steps,
                            "gbs": v["gbs"]} for c, v in classes.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "edge-iters/s",
                    "h2d_bytes_per_step": 4 * (g.n + 1) + 8 * g.m, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "stats": sol.stats,
        }
        out.update(sub)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _gpu_setup():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    return torch, dist, world, rank, local, torch.device("cuda", local)


def _batch_golden() -> dict:
    """The oracle's stored per-member answers of batch4096 (written by
    tests/golden/make_batch_values.py): g -> (num, den, len, digest, first edge)."""
    rows = {}
    path = os.path.join(ROOT, "tests", "golden", "batch4096_values.txt")
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            g, n, m, num, den, L, iters, digest, first = (int(x) for x in line.split())
            rows[g] = (num, den, L, digest, first)
    return rows


def _member_answers(vptr, rp, num, den, clen, cyc_all):
    """(num, den, len, digest, first edge) of every member, cycle edges local
    to the member graph, as the stored oracle answers hold them."""
    out = {}
    for g in range(vptr.shape[0] - 1):
        v0 = int(vptr[g])
        e0 = int(rp[v0])
        c = (np.asarray(cyc_all[v0:v0 + int(clen[g])], dtype=np.int64) - e0).astype(np.int32)
        out[g] = (int(num[g]), int(den[g]), int(clen[g]), synth.digest(c),
                  int(c[0]) if c.shape[0] else -1)
    return out


def measure_batch(args, workload, dev, world, rank, local, steps, compare_loop=True,
                  warmup=3) -> dict:
    """Batched form: graphs/s of one ocm_solve_batch call over the G graphs
    (N > 1: each rank solves its LPT share by edge count, the job rate counts
    all G graphs over the slowest rank), against a loop of ocm_solve over the
    same graphs (same stream, warm workspace; N = 1 only).  batch4096 members
    are compared with the oracle's stored answers."""
    import torch
    import torch.distributed as dist

    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300 import shard
    G, nmax, desc = BATCH_WORKLOADS[workload]
    graphs = synth.batch_graphs(G=G, nmin=100, nmax=nmax)
    full = synth.concat(graphs, name=workload)
    costs = full.row_ptr[full.graph_vptr[1:]].astype(np.int64) - \
        full.row_ptr[full.graph_vptr[:-1]]
    mine = shard.lpt_partition(costs, world)[rank]
    sub = shard.take_graphs(full.graph_vptr, full.row_ptr, full.col_idx, full.w, mine)
    b = synth.Batch(sub.graph_vptr, sub.row_ptr, sub.col_idx, sub.w, full.mode)
    vp, rp, col, w = [torch.from_numpy(x).to(dev) for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    ws = torch.empty(ocm.workspace_bytes_batch(b.G, b.N, b.M), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(3, warmup)):
        sol = ocm.solve_batch(vp, rp, col, w, b.mode, workspace=ws, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    launches = 0
    barrier()
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        sol = ocm.solve_batch(vp, rp, col, w, b.mode, workspace=ws, stream=stream)
        ev[k][1].record(stream)
        launches += sol.stats["launches"]
    barrier()
    local_ms = sum(a.elapsed_time(bb) for a, bb in ev)
    value, total_ms = job_rate(G / world, steps, local_ms, world, dev)

    # results of every graph, gathered on the host in the input order
    parts = shard.gather(shard.local_results(sub, sol.num.cpu().numpy(), sol.den.cpu().numpy(),
                                             sol.cycle_len.cpu().numpy(),
                                             sol.cycle_out.cpu().numpy()))
    res = shard.assemble(parts, full.graph_vptr)
    matches = None
    if workload == "batch4096":
        gold = _batch_golden()
        got = _member_answers(full.graph_vptr, full.row_ptr, res.num, res.den, res.cycle_len,
                              res.cycle_out)
        matches = sum(1 for gi in range(G) if got[gi] == gold[gi])

    loop = None
    if compare_loop:
        wsl = torch.empty(max(ocm.workspace_bytes(gr.n, gr.m) for gr in graphs),
                          dtype=torch.uint8, device=dev)
        cyc = torch.empty(max(gr.n for gr in graphs), dtype=torch.int32, device=dev)
        devg = [tuple(torch.from_numpy(x).to(dev) for x in (gr.row_ptr, gr.col_idx, gr.w))
                for gr in graphs]
        for r_, c_, w_ in devg[:3]:
            ocm.solve(r_, c_, w_, b.mode, workspace=wsl, cycle_out=cyc, stream=stream)
        identical = True
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # every graph of the loop is new to the solver's loop-graph cache, so
        # the loop is timed both with the CUDA-graph loop and host-driven, and
        # the faster of the two is the baseline
        loop_ms_by = {}
        for loop_name, flags in (("cuda_graph", 0), ("host", ocm.ocm.OCM_FLAG_HOST_LOOP)):
            barrier()
            e0.record(stream)
            for i, (r_, c_, w_) in enumerate(devg):
                x = ocm.solve(r_, c_, w_, b.mode, workspace=wsl, cycle_out=cyc, stream=stream,
                              flags=flags)
                identical &= (x.num, x.den) == (int(res.num[i]), int(res.den[i]))
                if i < 64:   # cycles of a sample of graphs compared edge by edge
                    off = int(full.row_ptr[int(full.graph_vptr[i])])
                    identical &= (res.cycle(i, full.graph_vptr) - off).tolist() == \
                        x.cycle.cpu().tolist()
            e1.record(stream)
            barrier()
            loop_ms_by[loop_name] = e0.elapsed_time(e1)
        loop_ms = min(loop_ms_by.values())
        loop = {"graphs_per_s": G / (loop_ms / 1e3), "ms": loop_ms, "ms_by_loop": loop_ms_by,
                "identical_results": bool(identical)}
        del devg, wsl

    # end to end: host CSR -> device, batched solve, results back
    h = [torch.from_numpy(x).pin_memory() for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    d = [torch.empty_like(x) for x in (vp, rp, col, w)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for src, dst in zip(h, d):
        dst.copy_(src, non_blocking=True)
    s2 = ocm.solve_batch(*d, b.mode, workspace=ws, stream=stream)
    outs = [s2.num.cpu(), s2.den.cpu(), s2.cycle_len.cpu(), s2.cycle_out.cpu()]
    e1.record(stream)
    barrier()
    e2e_value, _ = job_rate(G / world, 1, e0.elapsed_time(e1), world, dev)
    ms_batch = total_ms / steps
    return {
        "metric": "graphs/s", "value": value, "unit": "graphs/s", "n_gpus": world,
        "steps": steps, "ms_per_step": ms_batch,
        "config": {"workload": f"{workload}: {desc}", "G": G, "N": full.N, "M": full.M,
                   "mode": full.mode, "iterations": sol.stats["iterations"],
                   "loop": "cuda_graph" if sol.stats["graph_loop"] else "host",
                   "parallelism": (f"sharded over {world} GPUs by edge count (LPT), host gather"
                                   if world > 1 else "single GPU"),
                   "l2": "flushed before every timed step (256 MiB write, outside the timing)"},
        "members_matching_oracle": matches,
        "loop_of_plain_solver": loop,
        "speedup_vs_loop": (loop["ms"] / ms_batch) if loop else None,
        "e2e": {"value": e2e_value, "unit": "graphs/s",
                "h2d_bytes_per_step": sum(x.numel() * 4 for x in h),
                "d2h_bytes_per_step": sum(x.numel() * x.element_size() for x in outs)},
        "gpu_launches": launches, "stats": sol.stats}


def run_batch(args):
    torch, dist, world, rank, local, dev = _gpu_setup()
    with ClockSampler(local) as clocks:
        r = measure_batch(args, args.workload, dev, world, rank, local, args.steps,
                          compare_loop=world == 1, warmup=args.warmup)
    if rank == 0:
        r.update({"warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                  "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                  "clocks": clocks.summary()})
        print(json.dumps(r), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_grad(args, dev, world, rank, steps, warmup=3) -> dict:
    """Differentiation form on diff1m: forward + backward kernel against finite
    differences by looping the plain solver over 64 random edges plus the
    critical cycle (integer +1 perturbations, exact)."""
    import torch
    import torch.distributed as dist

    import paper_1111_0627_gb300 as ocm
    base = synth.diff1m_base()
    # the unique-optimum construction needs the base graph's critical cycle; the
    # solver's own answer is used here (the tests check it against the oracle)
    rp, col = torch.from_numpy(base.row_ptr).to(dev), torch.from_numpy(base.col_idx).to(dev)
    w0 = torch.from_numpy(base.w).to(dev)
    ws = ocm.make_workspace(base.n, base.m, dev)
    c0 = ocm.solve(rp, col, w0, "max", workspace=ws).cycle.long()
    w = w0.clone()
    w[c0] += 1
    stream = torch.cuda.current_stream(dev)
    gl = torch.ones(1, device=dev)
    for _ in range(max(3, warmup)):
        sol = ocm.solve(rp, col, w, "max", workspace=ws, stream=stream)
        g = ocm.backward(sol.cycle, gl, base.m, stream=stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sol = ocm.solve(rp, col, w, "max", workspace=ws, stream=stream)
        g = ocm.backward(sol.cycle, gl, base.m, stream=stream)
    e1.record(stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    rate, job_ms = job_rate(1, steps, e0.elapsed_time(e1), world, dev)
    fb_ms = job_ms / steps
    eb = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    eb[0].record(stream)
    for _ in range(steps):
        g = ocm.backward(sol.cycle, gl, base.m, stream=stream)
    eb[1].record(stream)
    torch.cuda.synchronize(dev)
    bw_ms = eb[0].elapsed_time(eb[1]) / steps
    rng = np.random.default_rng(1111062704)
    edges = np.unique(np.concatenate([rng.integers(0, base.m, 64), sol.cycle.cpu().numpy()]))
    lam0 = sol.value
    gh = g.cpu().numpy()
    e0.record(stream)
    max_rel = 0.0
    wp = torch.empty_like(w)
    for e in edges:
        wp.copy_(w)
        wp[int(e)] += 1
        fd = float(ocm.solve(rp, col, wp, "max", workspace=ws, stream=stream).value - lam0)
        if fd != 0.0:
            max_rel = max(max_rel, abs(gh[int(e)] - fd) / abs(fd))
        elif gh[int(e)] != 0.0:
            max_rel = float("inf")
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fd_ms = e0.elapsed_time(e1)
    return {
        "metric": "gradient evaluations/s", "value": rate, "unit": "1/s",
        "n_gpus": world, "steps": steps, "ms_per_step": fb_ms,
        "config": {"workload": "diff1m: n=2^20, ring + U{0..7} extras, w 1024*U[0,1000] with +1 "
                               "on the critical cycle (unique optimum), max",
                   "n": base.n, "m": base.m, "critical_cycle_len": int(sol.cycle.numel()),
                   "fd_edges": int(len(edges))},
        "backward_kernel_ms": bw_ms,
        "finite_difference_loop": {"ms": fd_ms, "solves": int(len(edges)),
                                   "max_rel_err_vs_gradient": max_rel},
        "speedup_vs_fd_loop": fd_ms / fb_ms}


def run_grad(args):
    torch, dist, world, rank, local, dev = _gpu_setup()
    r = measure_grad(args, dev, world, rank, args.steps, warmup=args.warmup)
    if rank == 0:
        r.update({"warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                  "vs_baseline": None, "dtype": "int64+f32", "data": "synthetic"})
        print(json.dumps(r), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_scc(args):
    """SCC front-end: decomposition plus the per-component solve of a sparse
    random digraph with many components and vertices without out-edges,
    vertices/s; the oracle's Tarjan decomposition timed beside it."""
    import paper_1111_0627_gb300 as ocm
    torch, dist, world, rank, local, dev = _gpu_setup()
    n = 10_000_000
    g = synth.random_digraph(np.random.default_rng(1111062799), n, 1.5, sink_frac=0.05)
    rp, col, w = [torch.from_numpy(x).to(dev) for x in (g.row_ptr, g.col_idx, g.w)]
    lib = ocm.load()
    ws = torch.empty(int(lib.ocm_workspace_size_solve_scc(g.n, g.m)), dtype=torch.uint8,
                     device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        sol = ocm.solve_scc(rp, col, w, g.mode, workspace=ws, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    launches = 0
    with ClockSampler(local) as clocks:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            sol = ocm.solve_scc(rp, col, w, g.mode, workspace=ws, stream=stream)
            ev[k][1].record(stream)
            launches += sol.stats["launches"]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
    value, total_ms = job_rate(n, args.steps, sum(a.elapsed_time(b) for a, b in ev), world, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    labels, count = ocm.scc(rp, col, workspace=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    scc_ms = e0.elapsed_time(e1)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        k_cpu, _ = oracle.tarjan_scc(g.row_ptr, g.col_idx)
        dt = time.perf_counter() - t0
        assert k_cpu == count, "oracle and GPU disagree on the number of components"
        cpu = {"value": n / dt, "unit": "vertices/s", "cores": 1, "kind": "oracle",
               "sample": f"Tarjan's decomposition of the same graph ({dt:.2f} s, single-threaded; "
                         f"decomposition only)"}
    h = [torch.from_numpy(x).pin_memory() for x in (g.row_ptr, g.col_idx, g.w)]
    d = [torch.empty_like(x) for x in (rp, col, w)]
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for src, dst in zip(h, d):
        dst.copy_(src, non_blocking=True)
    s2 = ocm.solve_scc(*d, g.mode, workspace=ws, stream=stream)
    out = [s2.num.cpu(), s2.den.cpu(), s2.root.cpu()]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    if rank == 0:
        print(json.dumps({
            "metric": "vertices/s", "value": value,
            "unit": "vertices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "digraph-scc: random digraph, n=10^7, out-degree Poisson(1.5), "
                                   "5% vertices without out-edges, w U[-50,50], max",
                       "n": g.n, "m": g.m, "components": count,
                       "components_with_cycle": int(sol.root.numel()),
                       "decomposition_ms": scc_ms,
                       "l2": "flushed before every timed step (256 MiB write, outside the timing)"},
            "cpu_baseline": cpu,
            "e2e": {"value": n / (e2e_ms / 1e3), "unit": "vertices/s",
                    "h2d_bytes_per_step": sum(x.numel() * 4 for x in h),
                    "d2h_bytes_per_step": sum(x.numel() * x.element_size() for x in out)},
            "gpu_launches": launches, "clocks": clocks.summary()}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="locality32m",
                    choices=sorted(_workloads()) + sorted(BATCH_WORKLOADS) +
                    ["diff1m-grad", "digraph-scc"])
    ap.add_argument("--ref-iters", type=int, default=0,
                    help="Howard iterations per reference (oracle) step (0: 1 on locality32m, "
                         "else 2)")
    ap.add_argument("--cpu-iters", type=int, default=2,
                    help="Howard iterations of the oracle in the cpu_baseline sample")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="skip the batch4096 and diff1m_grad sub-records of the default run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-lambda", action="store_true",
                    help="the paper's single-lambda form of the iteration (single-graph workloads)")
    ap.add_argument("--locality-log2", type=int, default=25,
                    help="log2 of the vertex count of the locality workload (default 25)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)      # at least three untimed warm-up steps
    if args.ref_iters <= 0:
        args.ref_iters = 1 if args.workload == "locality32m" else 2
    # the sub-records ride on the default single-graph line only
    args.subrecords = (not args.no_subrecords and args.workload == "locality32m"
                       and args.locality_log2 == 25 and not args.single_lambda)
    LOCALITY_LOG2[0] = args.locality_log2
    if args.workload in BATCH_WORKLOADS and args.impl == "ours":
        return run_batch(args)
    if args.workload == "diff1m-grad" and args.impl == "ours":
        return run_grad(args)
    if args.workload == "digraph-scc" and args.impl == "ours":
        return run_scc(args)
    if args.workload in BATCH_WORKLOADS or args.workload in ("diff1m-grad", "digraph-scc"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm is run on the single-graph workloads only"}))
        return 0
    make, desc = _workloads()[args.workload]
    g = make()
    if args.impl == "reference":
        return run_reference(args, g, desc)
    return run_ours(args, g, desc)


if __name__ == "__main__":
    sys.exit(main())
