"""The band-by-band task order of the degree-class sweep and the initial pass
(needs a GB300).  Graphs of more than 2^22 vertices take their warp tasks
band by band (all classes of 2^18 vertices, then the next band), each warp
keeping a cursor on the table of (band, class) groups; the test flag cuts the
bands to 1,024 vertices so that graphs small enough for the oracle cross
hundreds of bands, with empty groups, bands ending inside a class, heavy
vertices (outside the classes), the cycle-ratio instance and the batched
union.  Every solve must equal the oracle, and the unbanded order bit for
bit (policy and potentials)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_SMALL_BANDS


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def _check(g, t=None, init=None, **kw):
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=t, init_policy=init)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    extra = {}
    if t is not None:
        extra["transit"] = _dev(t)[0]
    if init is not None:
        extra["init_policy"] = _dev(init)[0]
    s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_TEST_SMALL_BANDS, certificate=True,
                  **extra, **kw)
    assert (s.num, s.den) == (h.num, h.den), g.name
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle], g.name
    assert s.stats["iterations"] == h.iterations, g.name
    ref = ocm.solve(rp, col, w, g.mode, certificate=True, **extra, **kw)
    assert torch.equal(s.policy, ref.policy) and torch.equal(s.potential, ref.potential), g.name
    return s


@pytest.mark.parametrize("mode", ["max", "min"])
def test_small_bands_on_graphs_with_mixed_degrees(mode):
    rng = np.random.default_rng(1111063000 + (mode == "min"))
    cases = [
        synth.locality(60000, 4096, -1000, 1000, seed=1111063001, mode=mode),  # degrees 4/16/64
        synth.ring_extra(50000, 0, 40, -50, 50, 1, seed=1111063002, mode=mode),  # many classes
        synth.tiny_random(rng, 40000, max_extra=3, wlo=-9, whi=9, mode=mode),   # short cycles
    ]
    for g in cases:
        _check(g)


def test_small_bands_with_heavy_vertices_ratio_warm_start_and_lane_loads():
    from test_gpu_heavy import hub_graph
    rng = np.random.default_rng(1111063010)
    _check(hub_graph(rng, 30000, 7, 1025, 5000))
    g = synth.locality(30000, 512, -100, 100, seed=1111063011)
    _check(g, t=rng.integers(1, 9, g.m).astype(np.int32))
    _check(g, init=synth.random_policy(rng, g.row_ptr))
    for epl in (1, 4, 32):
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
        for flags in (OCM_FLAG_TEST_SMALL_BANDS, OCM_FLAG_TEST_SMALL_BANDS | OCM_FLAG_HOST_LOOP):
            s = ocm.solve(rp, col, w, g.mode, flags=flags, edges_per_lane=epl)
            assert (s.num, s.den) == (h.num, h.den)
            assert s.stats["iterations"] == h.iterations


def test_small_bands_in_the_batched_union():
    graphs = synth.batch_graphs(G=30, nmin=500, nmax=8000)
    b = synth.concat(graphs)
    vptr, rp, col, w = _dev(b.graph_vptr, b.row_ptr, b.col_idx, b.w)
    sol = ocm.solve_batch(vptr, rp, col, w, b.mode, small_vertices=-1,
                          flags=OCM_FLAG_TEST_SMALL_BANDS)
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    for i, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (int(num[i]), int(den[i])) == (h.num, h.den), i
        e0 = int(b.row_ptr[int(b.graph_vptr[i])])
        assert (sol.cycle(i).cpu().numpy() - e0).tolist() == [int(x) for x in h.cycle], i
