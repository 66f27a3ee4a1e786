"""The two-level policy evaluation (needs a GB300): blocks resolve the policy
paths inside their own vertex ranges first, the cycles that cross ranges are
found on the graph of the "exit" vertices.  It must give exactly what the
one-level evaluation and the oracle give -- value, critical cycle, iteration
count, per-vertex means and potentials -- on graphs with and without locality
(forced on small graphs, where ranges hold a few hundred vertices and nearly
every cycle crosses them)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import (OCM_FLAG_EVAL_GLOBAL, OCM_FLAG_EVAL_LOCAL,
                                           OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_NO_BITMAP)


def _dev(g):
    d = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
            torch.from_numpy(g.w).to(d))


def _check(g, flags, h=None):
    h = h or oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, flags=flags, certificate=True)
    assert (s.num, s.den) == (h.num, h.den)
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle]
    assert s.stats["iterations"] == h.iterations
    assert (s.eta_num.cpu().numpy() == h.eta_p).all()
    assert (s.eta_den.cpu().numpy() == h.eta_q).all()
    assert (s.potential.cpu().numpy() == h.V).all()
    return s


@pytest.mark.parametrize("mode", ["max", "min"])
def test_forced_local_evaluation_on_random_graphs(mode):
    rng = np.random.default_rng(1111062900 + (mode == "min"))
    for trial in range(12):
        n = int(rng.integers(2000, 60000))
        if trial % 3 == 0:    # uniform targets: every policy edge leaves its range
            g = synth.ring_extra(n, 0, 4, -50, 50, 1, seed=1111062900 + trial, mode=mode)
        elif trial % 3 == 1:  # local targets, ranges of n / blocks vertices
            g = synth.locality(n, int(rng.integers(2, 400)), -1000, 1000,
                               seed=1111062950 + trial, mode=mode)
        else:                 # many short cycles, self-loops and parallel edges
            g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, mode=mode)
        _check(g, OCM_FLAG_EVAL_LOCAL)


@pytest.mark.parametrize("mode", ["max", "min"])
def test_local_evaluation_without_bitmaps(mode):
    """The form large ranges take (no shared-memory bitmaps: no leaf trimming,
    every vertex in the jump rounds), forced on small graphs."""
    rng = np.random.default_rng(1111062930 + (mode == "min"))
    for trial in range(6):
        n = int(rng.integers(2000, 40000))
        if trial % 2 == 0:
            g = synth.locality(n, int(rng.integers(2, 400)), -1000, 1000,
                               seed=1111062960 + trial, mode=mode)
        else:
            g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, mode=mode)
        _check(g, OCM_FLAG_EVAL_LOCAL | OCM_FLAG_TEST_NO_BITMAP)


def test_local_and_global_evaluation_agree_in_both_loop_forms():
    g = synth.locality32m(1 << 18)
    rp, col, w = _dev(g)
    ref = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_GLOBAL, certificate=True)
    for flags in (OCM_FLAG_EVAL_LOCAL, OCM_FLAG_EVAL_LOCAL | OCM_FLAG_HOST_LOOP):
        s = ocm.solve(rp, col, w, g.mode, flags=flags, certificate=True)
        assert (s.num, s.den) == (ref.num, ref.den)
        assert torch.equal(s.cycle, ref.cycle)
        assert torch.equal(s.potential, ref.potential) and torch.equal(s.policy, ref.policy)
        assert s.stats["iterations"] == ref.stats["iterations"]


def test_forced_local_evaluation_on_the_2p20_locality_graph():
    """The stored oracle answer of the 2^20 locality graph (value, cycle,
    iterations) and the oracle's certificate, with the two-level evaluation."""
    from test_gpu_parity import golden_values
    kv = golden_values()["locality_2^20"]
    g = synth.locality32m(1 << 20)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_LOCAL, certificate=True)
    assert (s.num, s.den) == (int(kv["num"]), int(kv["den"]))
    assert synth.digest(s.cycle.cpu().numpy().astype(np.int32)) == int(kv["cycle_digest"])
    assert s.stats["iterations"] == int(kv["iters"])
    rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, s.eta_num.cpu().numpy(),
                                 s.eta_den.cpu().numpy(), s.potential.cpu().numpy(),
                                 s.num, s.den, s.cycle.cpu().numpy())
    assert rc == 0, bad


def test_flags_for_the_evaluation_are_exclusive():
    g = synth.ring10k()
    rp, col, w = _dev(g)
    with pytest.raises(ocm.OCMError) as ei:
        ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_LOCAL | OCM_FLAG_EVAL_GLOBAL)
    assert ei.value.status == -1
    # single-lambda and cycle-ratio solves ignore the request (one-level only)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_LOCAL, single_lambda=True)
    assert (s.num, s.den) == (h.num, h.den)
