"""Batched form (needs a GB300): every graph of a disjoint-union batch gets
exactly the value and critical cycle that the oracle gives for that graph
alone, independent of the order of the graphs in the batch."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _solve_batch(b):
    d = torch.device("cuda")
    return ocm.solve_batch(torch.from_numpy(b.graph_vptr).to(d), torch.from_numpy(b.row_ptr).to(d),
                           torch.from_numpy(b.col_idx).to(d), torch.from_numpy(b.w).to(d), b.mode)


def _check_against_oracle(b, sol, graphs):
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    for g, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (int(num[g]), int(den[g])) == (h.num, h.den), g
        e0 = int(b.row_ptr[int(b.graph_vptr[g])])
        cyc = (sol.cycle(g).cpu().numpy() - e0).tolist()
        assert cyc == [int(x) for x in h.cycle], g


def test_batch_of_random_graphs_matches_per_graph_oracle():
    graphs = synth.batch_graphs(G=64, nmin=20, nmax=3000)
    b = synth.concat(graphs)
    sol = _solve_batch(b)
    _check_against_oracle(b, sol, graphs)


@pytest.mark.parametrize("mode", ["max", "min"])
def test_batch_mixed_tiny_graphs_and_modes(mode):
    rng = np.random.default_rng(77 + (mode == "min"))
    graphs = [synth.tiny_random(rng, int(rng.integers(1, 30)), max_extra=3, wlo=-50, whi=50,
                                mode=mode) for _ in range(200)]
    b = synth.concat(graphs)
    sol = _solve_batch(b)
    _check_against_oracle(b, sol, graphs)


def test_batch_order_independence():
    graphs = synth.batch_graphs(G=24, nmin=50, nmax=2000)
    perm = np.random.default_rng(3).permutation(len(graphs))
    b1 = synth.concat(graphs)
    b2 = synth.concat([graphs[i] for i in perm])
    s1, s2 = _solve_batch(b1), _solve_batch(b2)
    for k, i in enumerate(perm):
        assert int(s1.num[i]) == int(s2.num[k]) and int(s1.den[i]) == int(s2.den[k])
        c1 = s1.cycle(int(i)).cpu().numpy() - int(b1.row_ptr[int(b1.graph_vptr[i])])
        c2 = s2.cycle(k).cpu().numpy() - int(b2.row_ptr[int(b2.graph_vptr[k])])
        assert c1.tolist() == c2.tolist()


def test_batch_equals_single_solves_on_gpu():
    graphs = synth.batch_graphs(G=16, nmin=1000, nmax=60000)
    b = synth.concat(graphs)
    sol = _solve_batch(b)
    d = torch.device("cuda")
    for g, gr in enumerate(graphs):
        s = ocm.solve(torch.from_numpy(gr.row_ptr).to(d), torch.from_numpy(gr.col_idx).to(d),
                      torch.from_numpy(gr.w).to(d), gr.mode)
        assert (int(sol.num[g]), int(sol.den[g])) == (s.num, s.den)
        e0 = int(b.row_ptr[int(b.graph_vptr[g])])
        assert (sol.cycle(g).cpu() - e0).tolist() == s.cycle.cpu().tolist()


def test_batch_rejects_edges_between_graphs_and_bad_offsets():
    graphs = synth.batch_graphs(G=3, nmin=10, nmax=20)
    b = synth.concat(graphs)
    col = b.col_idx.copy()
    col[0] = int(b.graph_vptr[2])          # an edge of graph 0 into graph 2
    bad = synth.Batch(b.graph_vptr, b.row_ptr, col, b.w, b.mode)
    with pytest.raises(ocm.OCMError) as ei:
        _solve_batch(bad)
    assert ei.value.status == -2
    vp = b.graph_vptr.copy()
    vp[1] = vp[0]                           # empty graph
    with pytest.raises(ocm.OCMError) as ei:
        _solve_batch(synth.Batch(vp, b.row_ptr, b.col_idx, b.w, b.mode))
    assert ei.value.status == -2


def test_batch_backward_matches_per_graph_gradients():
    graphs = synth.batch_graphs(G=20, nmin=50, nmax=3000)
    b = synth.concat(graphs)
    sol = _solve_batch(b)
    gl = torch.arange(1, b.G + 1, dtype=torch.float32, device="cuda")
    grad = ocm.backward_batch(sol, gl, b.M).cpu().numpy()
    ref = np.zeros(b.M)
    for g, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        e0 = int(b.row_ptr[int(b.graph_vptr[g])])
        ref[e0:e0 + gr.m] = (g + 1) * oracle.gradient(gr.m, h.cycle)
    assert np.allclose(grad, ref, rtol=2**-22, atol=0)


def _batch_golden():
    rows = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "batch4096_values.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            g, n, m, num, den, L, iters, digest, first = (int(x) for x in line.split())
            rows[g] = (n, m, num, den, L, digest, first)
    return rows


def test_full_batch_config_every_member_against_oracle():
    """The full batched workload (4096 graphs, sizes log-uniform in [100,
    200000]) in one call, as the benchmark runs it: every member's value, cycle
    length, first cycle edge and cycle digest equal the oracle's stored answer
    for that graph alone (tests/golden/batch4096_values.txt, written by
    make_batch_values.py from oracle/ and synth/ only)."""
    gold = _batch_golden()
    assert len(gold) == 4096
    b = synth.batch4096()
    sol = _solve_batch(b)
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    clen = sol.cycle_len.cpu().numpy()
    cyc_all = sol.cycle_out.cpu().numpy()
    vptr, rp = b.graph_vptr, b.row_ptr
    bad = []
    for g in range(b.G):
        n, m, gnum, gden, L, digest, first = gold[g]
        v0 = int(vptr[g])
        assert int(vptr[g + 1]) - v0 == n and int(rp[int(vptr[g + 1])]) - int(rp[v0]) == m, g
        e0 = int(rp[v0])
        c = (cyc_all[v0:v0 + int(clen[g])] - e0).astype(np.int32)
        got = (int(num[g]), int(den[g]), int(clen[g]), synth.digest(c), int(c[0]) if len(c) else -1)
        if got != (gnum, gden, L, digest, first):
            bad.append((g, got, (gnum, gden, L, digest, first)))
    assert not bad, bad[:5]


def test_sharded_batch_on_one_rank_equals_the_batched_call():
    """paper_1111_0627_gb300.shard on a single rank (no process group): the LPT
    share is the whole batch, and the gathered host results equal one
    ocm_solve_batch call graph by graph."""
    from paper_1111_0627_gb300 import shard
    graphs = synth.batch_graphs(G=48, nmin=20, nmax=4000)
    b = synth.concat(graphs)
    res = shard.solve_batch_sharded(b.graph_vptr, b.row_ptr, b.col_idx, b.w, b.mode)
    sol = _solve_batch(b)
    assert (res.num == sol.num.cpu().numpy()).all() and (res.den == sol.den.cpu().numpy()).all()
    assert (res.cycle_len == sol.cycle_len.cpu().numpy()).all()
    for g in range(b.G):
        assert res.cycle(g, b.graph_vptr).tolist() == sol.cycle(g).cpu().tolist()
    assert (res.owner == 0).all()


@pytest.mark.parametrize("small", [-1, 64, 1500, 1 << 20])
def test_per_block_path_and_union_path_agree(small):
    """The persistent per-graph kernel (one block runs every iteration of a
    graph) and the disjoint-union path give every graph the same value and
    cycle as the oracle, whatever the size threshold that splits the batch
    between them (-1: union only; 1 << 20: every graph per block)."""
    rng = np.random.default_rng(1111062777)
    graphs = synth.batch_graphs(G=40, nmin=10, nmax=6000)
    graphs += [synth.tiny_random(rng, int(rng.integers(1, 12)), max_extra=3, wlo=-50, whi=50)
               for _ in range(40)]
    b = synth.concat(graphs)
    d = torch.device("cuda")
    args = [torch.from_numpy(x).to(d) for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    sol = ocm.solve_batch(*args, b.mode, small_vertices=small)
    _check_against_oracle(b, sol, graphs)
    sizes = np.diff(b.graph_vptr)
    edges = np.diff(b.row_ptr[b.graph_vptr])
    expect = int(((sizes <= small) & (edges <= 16 * small)).sum()) if small > 0 else 0
    assert sol.stats["batch_small_graphs"] == expect
    # the iteration count is the largest over the graphs, on either path
    iters = max(oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode).iterations for g in graphs)
    assert sol.stats["iterations"] == iters


def test_per_block_path_reports_the_iteration_cap():
    graphs = synth.batch_graphs(G=12, nmin=200, nmax=900)
    b = synth.concat(graphs)
    d = torch.device("cuda")
    args = [torch.from_numpy(x).to(d) for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    need = max(oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode).iterations for g in graphs)
    with pytest.raises(ocm.OCMError) as ei:
        ocm.solve_batch(*args, b.mode, small_vertices=1 << 20, max_iters=need)
    assert ei.value.status == -5
    sol = ocm.solve_batch(*args, b.mode, small_vertices=1 << 20, max_iters=need + 1)
    _check_against_oracle(b, sol, graphs)


@pytest.mark.parametrize("small", [-1, 1 << 20])
def test_batch_members_with_hub_vertices(small):
    """Members with a vertex of thousands of out-edges: the per-block sweep
    serves such a vertex with a whole warp; values and cycles are the oracle's."""
    graphs = [synth.hub4m(n=n, hub_deg=deg, seed=1111062790 + i)
              for i, (n, deg) in enumerate([(300, 40), (2000, 5000), (50, 33), (4000, 70000)])]
    graphs += synth.batch_graphs(G=6, nmin=30, nmax=500)
    b = synth.concat(graphs)
    d = torch.device("cuda")
    args = [torch.from_numpy(x).to(d) for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    sol = ocm.solve_batch(*args, b.mode, small_vertices=small)
    _check_against_oracle(b, sol, graphs)
    if small > 0:
        assert sol.stats["batch_small_graphs"] == len(graphs)


def test_automatic_split_sends_a_batch_of_small_graphs_to_the_per_block_path():
    graphs = synth.batch_graphs(G=30, nmin=50, nmax=3000)
    b = synth.concat(graphs)
    sol = _solve_batch(b)
    assert sol.stats["batch_small_graphs"] == len(graphs)


def test_batch_autotuner_picks_a_candidate_and_results_stay_exact(tmp_path, monkeypatch):
    """autotune.tune_batch times the per-block/union split and the union's
    sweep layout on the caller's batch, checks that every candidate gives the
    same results, and solve_batch(tune=True) uses the recorded choice."""
    monkeypatch.setenv("OCM_TUNE_FILE", str(tmp_path / "tune.json"))
    graphs = synth.batch_graphs(G=40, nmin=20, nmax=5000)
    b = synth.concat(graphs)
    d = torch.device("cuda")
    args = [torch.from_numpy(x).to(d) for x in (b.graph_vptr, b.row_ptr, b.col_idx, b.w)]
    cands = [(0, 1, 8, 512), (-1, 1, 4, 256), (1000, 1, 16, 512)]
    res = ocm.autotune.tune_batch(*args, b.mode, candidates=cands)
    picked = (res["batch_small_vertices"], res["sweep_kind"], res["edges_per_lane"],
              res["sweep_threads"])
    assert picked in cands and len(res["timings_ms"]) == 3
    assert ocm.autotune.lookup_batch(args[0], args[1]) == picked
    sol = ocm.solve_batch(*args, b.mode, tune=True)
    _check_against_oracle(b, sol, graphs)
