"""The frontier sweep (needs a GB300).  After an evaluation the record pass can
mark the records it changed, and the next sweep then skips every vertex none
of whose targets' records changed: such a vertex would choose as it did in the
last sweep.  The test flag makes both happen after every evaluation but the
first, so every sweep after the first is a frontier sweep; the solves must
equal the oracle exactly -- value, critical cycle, iteration count (a skipped
vertex that should have switched would change the trajectory) and the
certificate -- in both evaluation forms, for the mean and the ratio, with
heavy vertices, from warm starts and in a batch."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import (OCM_FLAG_EVAL_GLOBAL, OCM_FLAG_EVAL_LOCAL,
                                           OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_FRONTIER,
                                           OCM_FLAG_TEST_SMALL_BANDS)


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def _check(g, flags=0, t=None, init=None, certificate=True):
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=t, init_policy=init)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    extra = {}
    if t is not None:
        extra["transit"] = _dev(t)[0]
    if init is not None:
        extra["init_policy"] = _dev(init)[0]
    s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_TEST_FRONTIER | flags,
                  certificate=certificate, **extra)
    assert (s.num, s.den) == (h.num, h.den), g.name
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle], g.name
    assert s.stats["iterations"] == h.iterations, g.name
    if certificate:
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, s.eta_num.cpu().numpy(),
                                     s.eta_den.cpu().numpy(), s.potential.cpu().numpy(),
                                     s.num, s.den, s.cycle.cpu().numpy(), transit=t)
        assert rc == 0, (g.name, rc, bad)
    return s


@pytest.mark.parametrize("mode", ["max", "min"])
def test_frontier_on_tiny_graphs(mode):
    rng = np.random.default_rng(1111063100 + (mode == "min"))
    for trial in range(150):
        n = int(rng.integers(1, 50))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-30, whi=30, ring=bool(trial % 2),
                              mode=mode)
        _check(g, certificate=False)


@pytest.mark.parametrize("mode", ["max", "min"])
def test_frontier_in_both_evaluation_forms(mode):
    rng = np.random.default_rng(1111063110 + (mode == "min"))
    cases = [
        synth.locality(60000, 4096, -1000, 1000, seed=1111063111, mode=mode),
        synth.ring_extra(40000, 0, 6, -50, 50, 1, seed=1111063112, mode=mode),
        synth.tiny_random(rng, 30000, max_extra=3, wlo=-9, whi=9, mode=mode),
    ]
    for g in cases:
        for flags in (OCM_FLAG_EVAL_LOCAL, OCM_FLAG_EVAL_GLOBAL,
                      OCM_FLAG_EVAL_LOCAL | OCM_FLAG_HOST_LOOP | OCM_FLAG_TEST_SMALL_BANDS):
            _check(g, flags)


def test_frontier_with_ratio_heavy_vertices_and_warm_start():
    from test_gpu_heavy import hub_graph
    rng = np.random.default_rng(1111063120)
    _check(hub_graph(rng, 20000, 7, 1025, 5000))
    g = synth.locality(30000, 512, -100, 100, seed=1111063121)
    _check(g, t=rng.integers(1, 9, g.m).astype(np.int32))
    _check(g, init=synth.random_policy(rng, g.row_ptr))


def test_frontier_in_a_batch():
    graphs = synth.batch_graphs(G=30, nmin=200, nmax=6000)
    b = synth.concat(graphs)
    vptr, rp, col, w = _dev(b.graph_vptr, b.row_ptr, b.col_idx, b.w)
    sol = ocm.solve_batch(vptr, rp, col, w, b.mode, small_vertices=-1,
                          flags=OCM_FLAG_TEST_FRONTIER)
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    for i, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        assert (int(num[i]), int(den[i])) == (h.num, h.den), i
        e0 = int(b.row_ptr[int(b.graph_vptr[i])])
        assert (sol.cycle(i).cpu().numpy() - e0).tolist() == [int(x) for x in h.cycle], i


def test_default_frontier_on_the_2p20_locality_graph():
    """By default the frontier sweep takes over once few vertices switch; the
    stored oracle answer (value, cycle, iterations) must hold."""
    from test_gpu_parity import golden_values
    kv = golden_values()["locality_2^20"]
    g = synth.locality32m(1 << 20)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    s = ocm.solve(rp, col, w, g.mode)
    assert (s.num, s.den) == (int(kv["num"]), int(kv["den"]))
    assert synth.digest(s.cycle.cpu().numpy().astype(np.int32)) == int(kv["cycle_digest"])
    assert s.stats["iterations"] == int(kv["iters"])


def test_single_lambda_form_keeps_full_sweeps():
    """The single-lambda rebuild writes records after the record pass, so the
    frontier is off in that form even with the test flag; results stay exact."""
    rng = np.random.default_rng(1111063130)
    for trial in range(40):
        g = synth.tiny_random(rng, int(rng.integers(2, 60)), max_extra=3, wlo=-20, whi=20,
                              ring=True)
        h = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
        rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
        s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_TEST_FRONTIER, single_lambda=True)
        assert (s.num, s.den) == (h.num, h.den)
        assert s.stats["iterations"] == h.iterations

