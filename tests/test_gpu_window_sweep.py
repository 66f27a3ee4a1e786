"""The window sweep (needs a GB300): one block per SM walks a chunk of
vertices in tiles, the records of the vertices around the tile held in shared
memory by bulk copies, targets outside the window read from global memory.
It must switch exactly the vertices the degree-class sweep switches, so every
solve equals the oracle -- value, critical cycle, iteration count, and the
certificate of the per-vertex outputs -- whether the targets lie inside the
window (locality graphs), outside it (uniform targets), at chunk and vertex
range ends (tiny graphs: windows reaching below vertex 0 and past n), or at
heavy vertices (left to the heavy kernels)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import OCM_SWEEP_CLASSES, OCM_SWEEP_WINDOW


def _dev(g):
    d = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
            torch.from_numpy(g.w).to(d))


def _check(g, h=None, certificate=False, **kw):
    h = h or oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, sweep_kind=OCM_SWEEP_WINDOW, certificate=certificate, **kw)
    assert s.stats["sweep_kind"] == OCM_SWEEP_WINDOW
    assert (s.num, s.den) == (h.num, h.den), g.name
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle], g.name
    assert s.stats["iterations"] == h.iterations, g.name
    if certificate:
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, s.eta_num.cpu().numpy(),
                                     s.eta_den.cpu().numpy(), s.potential.cpu().numpy(),
                                     s.num, s.den, s.cycle.cpu().numpy())
        assert rc == 0, (g.name, rc, bad)
    return s


@pytest.mark.parametrize("mode", ["max", "min"])
def test_tiny_graphs(mode):
    rng = np.random.default_rng(1111062970 + (mode == "min"))
    for trial in range(120):
        n = int(rng.integers(1, 60))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-30, whi=30, ring=bool(trial % 2),
                              mode=mode)
        _check(g)


@pytest.mark.parametrize("mode", ["max", "min"])
def test_graphs_with_and_without_locality(mode):
    rng = np.random.default_rng(1111062980 + (mode == "min"))
    cases = [
        synth.locality(20000, 8, -100, 100, seed=1111062981, mode=mode),        # all in window
        synth.locality(70000, 4096, -1000, 1000, seed=1111062982, mode=mode),   # most in window
        synth.locality(50000, 30000, -1000, 1000, seed=1111062983, mode=mode),  # most outside
        synth.ring_extra(40000, 0, 5, -50, 50, 1, seed=1111062984, mode=mode),  # uniform targets
        synth.tiny_random(rng, 30000, max_extra=3, wlo=-9, whi=9, mode=mode),   # short cycles
    ]
    for g in cases:
        _check(g, certificate=True)


def test_lane_loads_and_heavy_vertices():
    g = synth.locality32m(1 << 16)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    for epl in (1, 2, 4, 16, 64):
        _check(g, h, edges_per_lane=epl)
    from test_gpu_heavy import hub_graph
    rng = np.random.default_rng(1111062990)
    for hubs, lo, hi in ((1, 60000, 60000), (7, 1025, 5000), (40, 1000, 3000)):
        _check(hub_graph(rng, 20000, hubs, lo, hi), certificate=True)


def test_window_and_classes_give_the_same_bits():
    """On a locality graph the window sweep gives the degree classes' bits
    (policy, potentials, cycle, iteration count); the default layout is the
    degree classes."""
    g = synth.locality32m(1 << 18)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, certificate=True, sweep_kind=OCM_SWEEP_WINDOW)
    assert s.stats["sweep_kind"] == OCM_SWEEP_WINDOW
    ref = ocm.solve(rp, col, w, g.mode, certificate=True)
    assert ref.stats["sweep_kind"] == OCM_SWEEP_CLASSES
    assert (s.num, s.den) == (ref.num, ref.den)
    assert torch.equal(s.cycle, ref.cycle) and torch.equal(s.policy, ref.policy)
    assert torch.equal(s.potential, ref.potential)
    assert s.stats["iterations"] == ref.stats["iterations"]


def test_cycle_ratio_keeps_the_degree_classes():
    g = synth.locality(20000, 64, -100, 100, seed=1111062992)
    t = np.random.default_rng(5).integers(1, 9, g.m).astype(np.int32)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, transit=torch.from_numpy(t).cuda(),
                  sweep_kind=OCM_SWEEP_WINDOW)
    assert s.stats["sweep_kind"] == OCM_SWEEP_CLASSES
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=t)
    assert (s.num, s.den) == (h.num, h.den)


def test_batch_union_with_the_window_sweep():
    graphs = synth.batch_graphs(G=40, nmin=50, nmax=6000)
    b = synth.concat(graphs)
    d = torch.device("cuda")
    sol = ocm.solve_batch(torch.from_numpy(b.graph_vptr).to(d), torch.from_numpy(b.row_ptr).to(d),
                          torch.from_numpy(b.col_idx).to(d), torch.from_numpy(b.w).to(d), b.mode,
                          small_vertices=-1, sweep_kind=OCM_SWEEP_WINDOW)
    assert sol.stats["sweep_kind"] == OCM_SWEEP_WINDOW
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    for i, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (int(num[i]), int(den[i])) == (h.num, h.den), i
        e0 = int(b.row_ptr[int(b.graph_vptr[i])])
        assert (sol.cycle(i).cpu().numpy() - e0).tolist() == [int(x) for x in h.cycle], i
