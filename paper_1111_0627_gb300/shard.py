"""The batched form across several GPUs, one process per GPU.

The graphs of a batch are independent (the paper solves its regions
concurrently, Sec. 3.3), so the batch shards without any exchange during the
solve: the graphs are split over the ranks by LPT bin packing on their edge
counts, every rank solves its share with ``ocm_solve_batch`` on its own
device, and the per-graph results (value, cycle length, cycle) are gathered on
the host in the input order.  No collective runs on the data path and no rank
reads another rank's memory; the only exchange is the final host-side gather.

Host logic only (numpy and ``torch.distributed``); every solve runs in the
CUDA library through :func:`paper_1111_0627_gb300.ocm.solve_batch`.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def lpt_partition(costs, world: int) -> list[np.ndarray]:
    """Longest-processing-time-first bin packing: graphs in decreasing cost
    (ties: smaller index first) go one by one to the rank with the smallest
    load so far (ties: smaller rank).  Returns, per rank, its graph indices in
    increasing order.  The largest load is at most the mean load plus the
    largest single cost, and deterministic for a given input."""
    if world < 1:
        raise ValueError("world must be >= 1")
    c = np.asarray(costs, dtype=np.int64)
    order = np.lexsort((np.arange(c.shape[0]), -c))
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(c.shape[0], dtype=np.int64)
    for g in order:
        r = int(np.argmin(load))          # first minimum: the smallest rank among equals
        owner[g] = r
        load[r] += c[g]
    return [np.flatnonzero(owner == r) for r in range(world)]


@dataclass
class SubBatch:
    """Graphs ``members`` of a disjoint-union batch as a batch of their own."""
    members: np.ndarray      # int64 [G_r], indices into the full batch, increasing
    graph_vptr: np.ndarray   # int32 [G_r + 1]
    row_ptr: np.ndarray      # int32 [N_r + 1]
    col_idx: np.ndarray      # int32 [M_r]
    w: np.ndarray            # int32 [M_r]
    edge_base: np.ndarray    # int64 [G_r]: first edge of each member in the full batch
    local_edge_base: np.ndarray  # int64 [G_r]: the same in the sub-batch


def take_graphs(graph_vptr, row_ptr, col_idx, w, members) -> SubBatch:
    """Host-side extraction of the member graphs (vertex and edge ids are
    renumbered; every edge stays inside its graph by the batch's contract)."""
    vp = np.asarray(graph_vptr, dtype=np.int64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    mem = np.asarray(members, dtype=np.int64)
    v0, v1 = vp[mem], vp[mem + 1]
    e0, e1 = rp[v0], rp[v1]
    nv, ne = v1 - v0, e1 - e0
    new_vp = np.zeros(mem.shape[0] + 1, dtype=np.int64)
    np.cumsum(nv, out=new_vp[1:])
    new_ep = np.zeros(mem.shape[0] + 1, dtype=np.int64)
    np.cumsum(ne, out=new_ep[1:])
    if new_vp[-1] >= 2**31 or new_ep[-1] >= 2**31:
        raise ValueError("sub-batch too large for int32 indices")
    vids = np.concatenate([np.arange(a, b) for a, b in zip(v0, v1)]) if mem.size else \
        np.zeros(0, np.int64)
    eids = np.concatenate([np.arange(a, b) for a, b in zip(e0, e1)]) if mem.size else \
        np.zeros(0, np.int64)
    vshift = np.repeat(new_vp[:-1] - v0, nv)       # new vertex id = old + shift
    eshift = np.repeat(new_ep[:-1] - e0, nv)       # the same for the edges of each vertex
    new_rp = np.empty(vids.shape[0] + 1, dtype=np.int64)
    new_rp[:-1] = rp[vids] + eshift
    new_rp[-1] = new_ep[-1]
    col = np.asarray(col_idx)[eids].astype(np.int64) + np.repeat(new_vp[:-1] - v0, ne)
    return SubBatch(mem, new_vp.astype(np.int32), new_rp.astype(np.int32), col.astype(np.int32),
                    np.asarray(w)[eids].astype(np.int32), e0, new_ep[:-1])


@dataclass
class GatheredBatch:
    """Per-graph results of a sharded solve, in the input order, with the
    layout of a single ``ocm_solve_batch`` call (host arrays)."""
    num: np.ndarray          # int64 [G]
    den: np.ndarray          # int32 [G]
    cycle_len: np.ndarray    # int32 [G]
    cycle_out: np.ndarray    # int32 [N]: graph g's cycle (global edge ids) at graph_vptr[g]
    owner: np.ndarray        # int32 [G]: rank that solved each graph

    def cycle(self, g: int, graph_vptr) -> np.ndarray:
        s = int(graph_vptr[g])
        return self.cycle_out[s:s + int(self.cycle_len[g])]


def local_results(sub: SubBatch, num, den, cycle_len, cycle_out):
    """One rank's results as (member, num, den, cycle in global edge ids)."""
    num = np.asarray(num, dtype=np.int64)
    den = np.asarray(den, dtype=np.int32)
    clen = np.asarray(cycle_len, dtype=np.int32)
    cyc = np.asarray(cycle_out, dtype=np.int64)
    out = []
    for i, g in enumerate(sub.members):
        s = int(sub.graph_vptr[i])
        c = cyc[s:s + int(clen[i])] - sub.local_edge_base[i] + sub.edge_base[i]
        out.append((int(g), int(num[i]), int(den[i]), c.astype(np.int32)))
    return out


def assemble(parts, graph_vptr) -> GatheredBatch:
    """Joins the per-rank result lists (``parts[r]`` from rank r) in the input
    order; every graph must appear exactly once."""
    vp = np.asarray(graph_vptr, dtype=np.int64)
    G, N = vp.shape[0] - 1, int(vp[-1])
    num = np.zeros(G, np.int64)
    den = np.zeros(G, np.int32)
    clen = np.zeros(G, np.int32)
    cyc = np.full(N, -1, np.int32)
    owner = np.full(G, -1, np.int32)
    for r, part in enumerate(parts):
        for g, a, b, c in part:
            if owner[g] != -1:
                raise ValueError(f"graph {g} solved twice")
            owner[g] = r
            num[g], den[g], clen[g] = a, b, c.shape[0]
            cyc[vp[g]:vp[g] + c.shape[0]] = c
    if (owner < 0).any():
        raise ValueError("graphs missing from the gather: "
                         f"{np.flatnonzero(owner < 0)[:8].tolist()}")
    return GatheredBatch(num, den, clen, cyc, owner)


def gather(local, group=None) -> list:
    """All ranks' result lists, in rank order (a host-side object gather; the
    one exchange of the sharded batch).  Without an initialised process group
    this is the single-rank case."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return [local]
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, local, group=group)
    return parts


def solve_batch_sharded(graph_vptr, row_ptr, col_idx, w, mode="max", *, device=None,
                        group=None, **kw) -> GatheredBatch:
    """Solves a batch given as host arrays across the ranks of ``group`` (all
    ranks call it with the same batch; each solves its LPT share on its
    current CUDA device) and returns every graph's result on every rank."""
    import torch
    import torch.distributed as dist

    from . import ocm
    world, rank = 1, 0
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    vp = np.asarray(graph_vptr, dtype=np.int64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    costs = rp[vp[1:]] - rp[vp[:-1]]
    mine = lpt_partition(costs, world)[rank]
    local = []
    if mine.size:
        sub = take_graphs(graph_vptr, row_ptr, col_idx, w, mine)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        t = [torch.from_numpy(x).to(dev) for x in (sub.graph_vptr, sub.row_ptr, sub.col_idx, sub.w)]
        sol = ocm.solve_batch(*t, mode, **kw)
        local = local_results(sub, sol.num.cpu().numpy(), sol.den.cpu().numpy(),
                              sol.cycle_len.cpu().numpy(), sol.cycle_out.cpu().numpy())
    return assemble(gather(local, group), graph_vptr)
