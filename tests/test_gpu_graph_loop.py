"""The policy-iteration loop as a CUDA graph (needs a GB300).

By default a solve runs its loop -- evaluate, improve, stop when no vertex
switched (Alg. 1) -- as one launch of a graph whose conditional WHILE node
repeats a captured step; OCM_FLAG_HOST_LOOP drives the same launches from the
host.  Both must give the oracle's result bit for bit, with the same
iteration and switch counts, and the graph's exits (iteration cap, a bounded
wait that gave up) must report the same errors as the host loop."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_STALL


def _dev(g):
    d = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
            torch.from_numpy(g.w).to(d))


def _both(g, **kw):
    rp, col, w = _dev(g)
    a = ocm.solve(rp, col, w, g.mode, **kw)
    b = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_HOST_LOOP, **kw)
    return a, b


def _same(a, b, h):
    assert (a.num, a.den) == (b.num, b.den) == (h.num, h.den)
    ref = [int(x) for x in h.cycle]
    assert a.cycle.cpu().tolist() == ref and b.cycle.cpu().tolist() == ref
    for k in ("iterations", "switched", "cycles", "detect_rounds", "value_rounds",
              "detect_items", "value_items"):
        assert a.stats[k] == b.stats[k], k
    assert a.stats["iterations"] == h.iterations
    assert a.stats["graph_loop"] == 1 and b.stats["graph_loop"] == 0


@pytest.mark.parametrize("mode", ["max", "min"])
def test_graph_loop_equals_host_loop_on_tiny_graphs(mode):
    rng = np.random.default_rng(77001 + (mode == "min"))
    for trial in range(60):
        n = int(rng.integers(1, 40))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-25, whi=25, ring=bool(trial % 2),
                              mode=mode)
        a, b = _both(g)
        _same(a, b, oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode))


@pytest.mark.parametrize("name", ["ring10k", "product4"])
def test_graph_loop_equals_host_loop_on_workloads(name):
    g = getattr(synth, name)()
    a, b = _both(g, certificate=True)
    _same(a, b, oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode))
    for k in ("eta_num", "eta_den", "potential", "policy"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k


def test_cached_graph_is_reused_and_rekeyed():
    """Repeated solves on one workspace reuse the instantiated graph; a
    different graph on the same workspace, or other launch parameters, must
    not run a stale one."""
    g1 = synth.ring10k()
    rng = np.random.default_rng(5)
    g2 = synth.tiny_random(rng, 5000, max_extra=3, wlo=1, whi=100, ring=True, mode="max")
    ws = ocm.make_workspace(max(g1.n, g2.n), max(g1.m, g2.m) + 1)
    h1 = oracle.howard(g1.row_ptr, g1.col_idx, g1.w, g1.mode)
    h2 = oracle.howard(g2.row_ptr, g2.col_idx, g2.w, g2.mode)
    d1, d2 = _dev(g1), _dev(g2)
    for rnd in range(3):
        for g, d, h in ((g1, d1, h1), (g2, d2, h2)):
            for epl, thr in ((0, 0), (2, 128)):
                s = ocm.solve(*d, g.mode, workspace=ws, edges_per_lane=epl, sweep_threads=thr)
                assert (s.num, s.den) == (h.num, h.den), (g.name, rnd, epl)
                assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle]
                assert s.stats["graph_loop"] == 1


def test_graph_loop_on_another_stream():
    g = synth.ring10k()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    rp, col, w = _dev(g)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sol = ocm.solve(rp, col, w, g.mode)
    assert (sol.num, sol.den) == (h.num, h.den)
    assert sol.stats["graph_loop"] == 1


def test_graph_loop_iteration_cap():
    g = synth.ring10k()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert h.iterations >= 2
    rp, col, w = _dev(g)
    for flags in (0, OCM_FLAG_HOST_LOOP):
        with pytest.raises(ocm.OCMError) as ei:
            ocm.solve(rp, col, w, g.mode, max_iters=1, flags=flags)
        assert ei.value.status == -5
        # a cap exactly at the oracle's count is enough
        sol = ocm.solve(rp, col, w, g.mode, max_iters=h.iterations + 1, flags=flags)
        assert (sol.num, sol.den) == (h.num, h.den)


def test_graph_loop_bounded_wait_expires_cleanly():
    """The evaluation's first grid barrier waits for a block that does not
    exist (test flag) inside the graph: the WHILE loop must stop, the solve
    must report OCM_ERR_TIMEOUT, and the next solve must succeed."""
    g = synth.ring10k()
    rp, col, w = _dev(g)
    with pytest.raises(ocm.OCMError) as ei:
        ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_TEST_STALL)
    assert ei.value.status == -6
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    sol = ocm.solve(rp, col, w, g.mode)
    assert (sol.num, sol.den) == (h.num, h.den)
    assert sol.stats["graph_loop"] == 1


def test_wait_limit_option_bounds_the_stalled_wait():
    """ocm_options.wait_limit_ms sets the limit of every device-side wait: the
    stalled barrier of the test flag gives up after about that long (GPU wall
    clock), in both loop forms, and the context stays usable."""
    import time
    g = synth.ring10k()
    rp, col, w = _dev(g)
    for flags in (OCM_FLAG_TEST_STALL, OCM_FLAG_TEST_STALL | OCM_FLAG_HOST_LOOP):
        took = {}
        for ms in (5, 400):
            torch.cuda.synchronize()
            t = time.perf_counter()
            with pytest.raises(ocm.OCMError) as ei:
                ocm.solve(rp, col, w, g.mode, flags=flags, wait_limit_ms=ms)
            took[ms] = time.perf_counter() - t
            assert ei.value.status == -6
        assert took[400] >= 0.38, took
        assert took[5] < 0.25, took
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    sol = ocm.solve(rp, col, w, g.mode, wait_limit_ms=50)
    assert (sol.num, sol.den) == (h.num, h.den)


def test_injected_loop_graph_failure_falls_back_to_the_host_loop(monkeypatch):
    """OCM_FAULT=alloc: the loop graph cannot be instantiated, the solve runs
    the host-driven loop and gives the same answer."""
    g = synth.ring10k()
    rp, col, w = _dev(g)
    monkeypatch.setenv("OCM_FAULT", "alloc")
    sol = ocm.solve(rp, col, w, g.mode)
    monkeypatch.delenv("OCM_FAULT")
    ref = ocm.solve(rp, col, w, g.mode)
    assert sol.stats["graph_loop"] == 0 and ref.stats["graph_loop"] == 1
    assert (sol.num, sol.den) == (ref.num, ref.den)
    assert sol.cycle.tolist() == ref.cycle.tolist()
    assert sol.stats["iterations"] == ref.stats["iterations"]


def test_batch_graph_loop_equals_host_loop():
    graphs = synth.batch_graphs(G=48, nmin=20, nmax=4000)
    b = synth.concat(graphs)
    d = torch.device("cuda")
    args = (torch.from_numpy(b.graph_vptr).to(d), torch.from_numpy(b.row_ptr).to(d),
            torch.from_numpy(b.col_idx).to(d), torch.from_numpy(b.w).to(d), b.mode)
    a = ocm.solve_batch(*args)
    c = ocm.solve_batch(*args, flags=OCM_FLAG_HOST_LOOP)
    assert a.stats["graph_loop"] == 1 and c.stats["graph_loop"] == 0
    assert torch.equal(a.num, c.num) and torch.equal(a.den, c.den)
    assert torch.equal(a.cycle_len, c.cycle_len)
    for g, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (int(a.num[g]), int(a.den[g])) == (h.num, h.den), g
        e0 = int(b.row_ptr[int(b.graph_vptr[g])])
        assert (a.cycle(g).cpu() - e0).tolist() == [int(x) for x in h.cycle], g
        assert torch.equal(a.cycle(g), c.cycle(g))
