"""Autotuner for the improvement sweep's layout and launch parameters.

The sweep has two layouts.  Edge tiles: the CSR edge array is cut into tiles
of 32 * edges_per_lane edges, one warp each (edges_per_lane 4 or 8).
Degree classes: a vertex of out-degree d is served by a group of g lanes (the
smallest power of two with d <= edges_per_lane * g, at most 32).  Both run in
blocks of ``sweep_threads``.  Which combination is fastest depends on the
degree distribution and on how local the targets are, so :func:`tune` runs
one full solve per candidate on the caller's graph, reads the sweep kernels'
time from the library's own CUDA-event instrumentation (``ocm_profile_*``),
and keeps the fastest.  Results are cached per graph signature (size and
degree buckets) in a JSON table (``OCM_TUNE_FILE``, default
``~/.cache/ocm_gb300/tune.json``); ``solve(..., tune=True)`` looks the
signature up.  The solver's results never depend on these parameters -- only
its speed does.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import threading

import torch

from . import _native

TILES, CLASSES, WINDOW = 2, 1, 3   # OCM_SWEEP_TILES, _CLASSES, _WINDOW (include/ocm.h)
CANDIDATES = ([(TILES, epl, thr) for epl in (4, 8) for thr in (64, 128, 256)] +
              [(CLASSES, epl, thr) for epl in (2, 4, 8, 16, 32) for thr in (128, 256, 512)] +
              [(WINDOW, epl, 512) for epl in (2, 4, 8, 16)])
SWEEP_CLASS = 1       # profiling class of the improvement sweep (include/ocm.h)
_lock = threading.Lock()


def table_path() -> str:
    return os.environ.get("OCM_TUNE_FILE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ocm_gb300", "tune.json"))


def signature(row_ptr: torch.Tensor) -> str:
    """Size and degree-shape buckets: log2 of n, of the mean degree (half
    steps) and of the largest degree."""
    deg = (row_ptr[1:] - row_ptr[:-1]).to(torch.float64)
    n = int(deg.numel())
    mean = float(deg.mean()) if n else 1.0
    mx = float(deg.max()) if n else 1.0
    return (f"n{math.ceil(math.log2(max(n, 2)))}_d{round(2 * math.log2(max(mean, 1.0)))}"
            f"_x{math.ceil(math.log2(max(mx, 1.0)))}")


def _load_table() -> dict:
    try:
        with open(table_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_table(tab: dict) -> None:
    path = table_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(tab, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(row_ptr: torch.Tensor) -> tuple[int, int, int] | None:
    with _lock:
        entry = _load_table().get(signature(row_ptr))
    if not entry or "sweep_kind" not in entry:
        return None
    return int(entry["sweep_kind"]), int(entry["edges_per_lane"]), int(entry["sweep_threads"])


def tune(row_ptr: torch.Tensor, col_idx: torch.Tensor, w: torch.Tensor, mode="max", *,
         candidates=CANDIDATES, save: bool = True) -> dict:
    """Time the sweep for every (sweep_kind, edges_per_lane, sweep_threads)
    candidate and record the fastest for this graph's signature."""
    from .ocm import solve
    lib = _native.load()
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    timings = {}
    ref = None
    ws = None
    prev = lib.ocm_profile_enable(0)
    try:
        for kind, epl, thr in candidates:
            sol = solve(row_ptr, col_idx, w, mode, workspace=ws, edges_per_lane=epl,
                        sweep_threads=thr, sweep_kind=kind)   # warm-up, and the result to compare
            if ws is None:
                from .ocm import make_workspace
                ws = make_workspace(row_ptr.numel() - 1, col_idx.numel(), row_ptr.device)
            if ref is None:
                ref = (sol.num, sol.den)
            elif (sol.num, sol.den) != ref:
                raise RuntimeError("launch parameters changed the result")
            lib.ocm_profile_enable(1)
            lib.ocm_profile_collect(None, None)
            solve(row_ptr, col_idx, w, mode, workspace=ws, edges_per_lane=epl, sweep_threads=thr,
                  sweep_kind=kind)
            lib.ocm_profile_collect(ms, cnt)
            lib.ocm_profile_enable(0)
            timings[f"{kind}x{epl}x{thr}"] = ms[SWEEP_CLASS] / max(cnt[SWEEP_CLASS], 1)
    finally:
        lib.ocm_profile_enable(prev)
    best = min(timings, key=timings.get)
    kind, epl, thr = (int(x) for x in best.split("x"))
    result = {"sweep_kind": kind, "edges_per_lane": epl, "sweep_threads": thr,
              "sweep_ms": timings[best], "timings_ms": timings, "signature": signature(row_ptr)}
    if save:
        with _lock:
            tab = _load_table()
            tab[result["signature"]] = {k: result[k] for k in ("sweep_kind", "edges_per_lane",
                                                               "sweep_threads", "sweep_ms")}
            _save_table(tab)
    return result


# ----------------------------------------------------------------------------
# Batched form: the size limit of the per-block path (ocm_options.
# batch_small_vertices: 0 automatic, < 0 union only, else a vertex count) and
# the union path's sweep layout, timed as whole ocm_solve_batch calls.
# ----------------------------------------------------------------------------
BATCH_CANDIDATES = ([(small, CLASSES, 8, 512) for small in (0, -1, 4096, 65536)] +
                    [(-1, CLASSES, epl, thr) for epl in (4, 16) for thr in (256, 512)])


def batch_signature(graph_vptr: torch.Tensor, row_ptr: torch.Tensor) -> str:
    """Batch shape buckets: log2 of the graph count, of the total vertex count,
    of the largest graph and of the mean degree (half steps)."""
    sizes = (graph_vptr[1:] - graph_vptr[:-1]).to(torch.float64)
    G = int(sizes.numel())
    N = int(row_ptr.numel() - 1)
    M = int(row_ptr[-1])
    mean = M / max(N, 1)
    return (f"batch_g{math.ceil(math.log2(max(G, 2)))}_n{math.ceil(math.log2(max(N, 2)))}"
            f"_x{math.ceil(math.log2(max(float(sizes.max()), 2.0)))}"
            f"_d{round(2 * math.log2(max(mean, 1.0)))}")


def lookup_batch(graph_vptr: torch.Tensor, row_ptr: torch.Tensor):
    with _lock:
        entry = _load_table().get(batch_signature(graph_vptr, row_ptr))
    if not entry or "batch_small_vertices" not in entry:
        return None
    return (int(entry["batch_small_vertices"]), int(entry["sweep_kind"]),
            int(entry["edges_per_lane"]), int(entry["sweep_threads"]))


def tune_batch(graph_vptr: torch.Tensor, row_ptr: torch.Tensor, col_idx: torch.Tensor,
               w: torch.Tensor, mode="max", *, candidates=BATCH_CANDIDATES, reps: int = 2,
               save: bool = True) -> dict:
    """Time ocm_solve_batch (CUDA events on the current stream, best of
    `reps` after a warm-up) for every (batch_small_vertices, sweep_kind,
    edges_per_lane, sweep_threads) candidate, check that every candidate gives
    the same results, and record the fastest for this batch's signature."""
    from .ocm import solve_batch, workspace_bytes_batch
    G, N, M = graph_vptr.numel() - 1, row_ptr.numel() - 1, col_idx.numel()
    ws = torch.empty(workspace_bytes_batch(G, N, M), dtype=torch.uint8, device=row_ptr.device)
    stream = torch.cuda.current_stream(row_ptr.device)
    timings, ref = {}, None
    for small, kind, epl, thr in candidates:
        kw = dict(workspace=ws, stream=stream, small_vertices=small, sweep_kind=kind,
                  edges_per_lane=epl, sweep_threads=thr)
        sol = solve_batch(graph_vptr, row_ptr, col_idx, w, mode, **kw)
        got = (sol.num.clone(), sol.den.clone(), sol.cycle_len.clone())
        if ref is None:
            ref = got
        elif not all(torch.equal(a, b) for a, b in zip(ref, got)):
            raise RuntimeError("launch parameters changed the result")
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            solve_batch(graph_vptr, row_ptr, col_idx, w, mode, **kw)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        timings[f"{small}x{kind}x{epl}x{thr}"] = best
    pick = min(timings, key=timings.get)
    small, kind, epl, thr = (int(x) for x in pick.split("x"))
    result = {"batch_small_vertices": small, "sweep_kind": kind, "edges_per_lane": epl,
              "sweep_threads": thr, "batch_ms": timings[pick], "timings_ms": timings,
              "signature": batch_signature(graph_vptr, row_ptr)}
    if save:
        with _lock:
            tab = _load_table()
            tab[result["signature"]] = {k: result[k] for k in (
                "batch_small_vertices", "sweep_kind", "edges_per_lane", "sweep_threads",
                "batch_ms")}
            _save_table(tab)
    return result
