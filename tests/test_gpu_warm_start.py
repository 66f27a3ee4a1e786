"""Warm start (needs a GB300): the CUDA path started from a caller-given
policy follows exactly the oracle's Howard iteration started from the same
policy (value, critical cycle, iteration count), for single graphs and
batches; an initial policy edge that does not leave its vertex is rejected
before any output is written."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


@pytest.mark.parametrize("mode", ["max", "min"])
def test_random_start_policies_follow_the_oracle(mode):
    rng = np.random.default_rng(1111062760 + (mode == "min"))
    for trial in range(150):
        n = int(rng.integers(1, 40))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-50, whi=50, ring=bool(trial % 2),
                              mode=mode)
        init = synth.random_policy(rng, g.row_ptr)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, mode, init_policy=init)
        rp, col, w, ip = _dev(g.row_ptr, g.col_idx, g.w, init)
        s = ocm.solve(rp, col, w, mode, init_policy=ip)
        assert (s.num, s.den) == (h.num, h.den), trial
        assert s.cycle.cpu().tolist() == h.cycle.tolist(), trial
        assert s.stats["iterations"] == h.iterations, trial


@pytest.mark.parametrize("name", ["ring10k", "product4"])
def test_resolve_after_weight_change_from_previous_policy(name):
    g = getattr(synth, name)()
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    first = ocm.solve(rp, col, w, g.mode, certificate=True)
    rng = np.random.default_rng(1111062762)
    w2 = g.w.copy()
    idx = rng.integers(0, g.m, size=64)
    w2[idx] += rng.integers(-30, 31, size=64).astype(np.int32)
    (w2d,) = _dev(w2)
    warm = ocm.solve(rp, col, w2d, g.mode, init_policy=first.policy, certificate=True)
    cold = ocm.solve(rp, col, w2d, g.mode)
    h = oracle.howard(g.row_ptr, g.col_idx, w2, g.mode,
                      init_policy=first.policy.cpu().numpy())
    assert (warm.num, warm.den) == (h.num, h.den) == (cold.num, cold.den)
    assert warm.cycle.cpu().tolist() == h.cycle.tolist()
    assert warm.stats["iterations"] == h.iterations
    assert warm.stats["iterations"] < cold.stats["iterations"]
    rc, bad = oracle.certificate(g.row_ptr, g.col_idx, w2, g.mode, warm.eta_num.cpu().numpy(),
                                 warm.eta_den.cpu().numpy(), warm.potential.cpu().numpy(),
                                 warm.num, warm.den, warm.cycle.cpu().numpy())
    assert rc == 0, (rc, bad)


def test_start_from_the_final_policy_stops_at_once():
    g = synth.ring10k()
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    s = ocm.solve(rp, col, w, g.mode, certificate=True)
    s2 = ocm.solve(rp, col, w, g.mode, init_policy=s.policy)
    assert s2.stats["iterations"] == 0
    assert (s2.num, s2.den) == (s.num, s.den)
    assert s2.cycle.cpu().tolist() == s.cycle.cpu().tolist()


def test_foreign_start_edge_is_rejected_and_outputs_untouched():
    g = synth.from_edges(3, [(0, 1, 1), (1, 2, 1), (2, 0, 1), (2, 2, 5)])
    rp, col, w, bad = _dev(g.row_ptr, g.col_idx, g.w, np.array([0, 0, 2], np.int32))
    out = torch.full((3,), 77, dtype=torch.int32, device=rp.device)
    with pytest.raises(ocm.OCMError) as e:
        ocm.solve(rp, col, w, init_policy=bad, cycle_out=out)
    assert e.value.status == -1
    assert out.cpu().tolist() == [77, 77, 77]
    (good,) = _dev(np.array([0, 1, 2], np.int32))
    assert ocm.solve(rp, col, w, init_policy=good).num == 5


@pytest.mark.parametrize("mode", ["max", "min"])
def test_batch_warm_start_follows_the_oracle_per_graph(mode):
    rng = np.random.default_rng(1111062764 + (mode == "min"))
    graphs = [synth.tiny_random(rng, int(rng.integers(1, 60)), max_extra=4, wlo=-40, whi=40,
                                mode=mode) for _ in range(120)]
    inits = [synth.random_policy(rng, gr.row_ptr) for gr in graphs]
    b = synth.concat(graphs)
    # global edge ids: shift each graph's start policy by its first edge
    init = np.concatenate([ini + int(b.row_ptr[int(b.graph_vptr[k])])
                           for k, ini in enumerate(inits)]).astype(np.int32)
    vp, rp, col, w, ip = _dev(b.graph_vptr, b.row_ptr, b.col_idx, b.w, init)
    sol = ocm.solve_batch(vp, rp, col, w, mode, init_policy=ip)
    num, den = sol.num.cpu().numpy(), sol.den.cpu().numpy()
    for k, gr in enumerate(graphs):
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, mode, init_policy=inits[k])
        assert (int(num[k]), int(den[k])) == (h.num, h.den), k
        e0 = int(b.row_ptr[int(b.graph_vptr[k])])
        assert (sol.cycle(k).cpu().numpy() - e0).tolist() == h.cycle.tolist(), k
