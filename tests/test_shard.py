"""Sharding of the batched form over ranks (host logic, CPU): the LPT split by
edge count, the extraction of each rank's member graphs, and the host-side
gather that puts every graph's result back in the input order.  The two-rank
test runs gloo processes and stands the CPU oracle in for the GPU solver of
each rank, so partition, renumbering and gather are checked end to end."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1111_0627_gb300 import shard


def test_lpt_partition_is_a_balanced_deterministic_split():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 8):
        costs = rng.integers(1, 10_000, size=333)
        parts = shard.lpt_partition(costs, world)
        allg = np.sort(np.concatenate(parts))
        assert allg.tolist() == list(range(333))          # every graph exactly once
        loads = [int(costs[p].sum()) for p in parts]
        assert max(loads) <= costs.sum() / world + costs.max()   # the LPT bound
        assert all((np.diff(p) > 0).all() for p in parts)
        again = shard.lpt_partition(costs, world)
        assert all((a == b).all() for a, b in zip(parts, again))
    # hand case: costs 7,5,4,3,1 on two ranks -> {7,3} = 10 and {5,4,1} = 10
    parts = shard.lpt_partition([7, 5, 4, 3, 1], 2)
    assert [p.tolist() for p in parts] == [[0, 3], [1, 2, 4]]


def test_more_ranks_than_graphs_leaves_ranks_empty():
    parts = shard.lpt_partition([3, 9], 4)
    assert [p.tolist() for p in parts] == [[1], [0], [], []]


def test_take_graphs_rebuilds_each_member_exactly():
    graphs = synth.batch_graphs(G=9, nmin=5, nmax=60)
    b = synth.concat(graphs)
    members = np.array([1, 4, 5, 8])
    sub = shard.take_graphs(b.graph_vptr, b.row_ptr, b.col_idx, b.w, members)
    sb = synth.Batch(sub.graph_vptr, sub.row_ptr, sub.col_idx, sub.w, b.mode)
    for i, g in enumerate(members):
        a, c = sb.member(i), graphs[g]
        assert (a.row_ptr == c.row_ptr).all() and (a.col_idx == c.col_idx).all()
        assert (a.w == c.w).all()
        assert sub.edge_base[i] == b.row_ptr[b.graph_vptr[g]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    graphs = synth.batch_graphs(G=40, nmin=10, nmax=400)
    b = synth.concat(graphs)
    costs = b.row_ptr[b.graph_vptr[1:]].astype(np.int64) - b.row_ptr[b.graph_vptr[:-1]]
    mine = shard.lpt_partition(costs, world)[rank]
    sub = shard.take_graphs(b.graph_vptr, b.row_ptr, b.col_idx, b.w, mine)
    sb = synth.Batch(sub.graph_vptr, sub.row_ptr, sub.col_idx, sub.w, b.mode)
    # the oracle stands in for this rank's GPU batch solve (local edge ids)
    num, den, clen = [], [], []
    cyc = np.full(sb.N, -1, np.int32)
    for i in range(sb.G):
        gr = sb.member(i)
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        num.append(h.num), den.append(h.den), clen.append(len(h.cycle))
        s = int(sub.graph_vptr[i])
        cyc[s:s + len(h.cycle)] = np.asarray(h.cycle) + int(sub.local_edge_base[i])
    local = shard.local_results(sub, num, den, clen, cyc)
    res = shard.assemble(shard.gather(local), b.graph_vptr)
    out[rank] = (res.num.tolist(), res.den.tolist(), res.cycle_len.tolist(),
                 res.cycle_out.tolist(), res.owner.tolist(), mine.tolist())
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_every_graph_in_input_order():
    import oracle
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    graphs = synth.batch_graphs(G=40, nmin=10, nmax=400)
    b = synth.concat(graphs)
    assert res[0][:5] == res[1][:5]                       # every rank holds the whole answer
    num, den, clen, cyc, owner, _ = res[0]
    assert sorted(res[0][5] + res[1][5]) == list(range(40))
    for g, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (num[g], den[g], clen[g]) == (h.num, h.den, len(h.cycle)), g
        s, e0 = int(b.graph_vptr[g]), int(b.row_ptr[b.graph_vptr[g]])
        assert [x - e0 for x in cyc[s:s + clen[g]]] == [int(x) for x in h.cycle], g
        assert g in res[owner[g]][5]
    # both ranks got work, and the split is the LPT one
    assert set(owner) == {0, 1}


def test_assemble_rejects_missing_and_duplicate_graphs():
    vp = np.array([0, 2, 5])
    part = [(0, 1, 1, np.array([0, 1], np.int32))]
    with pytest.raises(ValueError):
        shard.assemble([part], vp)
    with pytest.raises(ValueError):
        shard.assemble([part, part + [(1, 2, 1, np.array([3], np.int32))]], vp)
