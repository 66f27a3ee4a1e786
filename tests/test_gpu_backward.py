"""Backward form: d lambda*/dw from the CUDA backward kernel, checked against
the oracle's gradient and against exact finite differences on the
differentiation workload (needs a GB300)."""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import golden_values

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def diff1m():
    """Differentiation workload: the 2^20-vertex graph with weights 1024*U[0,1000]
    and +1 on each edge of its (oracle-computed, stored) critical cycle, which
    makes that cycle the unique optimum."""
    base = synth.diff1m_base()
    cyc = np.array(golden_values()["diff1m_base_cycle"], dtype=np.int64)
    w = base.w.copy()
    w[cyc] += 1
    return synth.Graph(base.row_ptr, base.col_idx, w, "max", "diff1m"), cyc


def test_backward_matches_oracle_gradient():
    for g in (synth.ring10k(), synth.locality32m(1 << 18)):
        rp, col, w = _dev(g.row_ptr), _dev(g.col_idx), _dev(g.w)
        sol = ocm.solve(rp, col, w, g.mode)
        grad = ocm.backward(sol.cycle, torch.ones(1, device="cuda"), g.m).cpu().numpy()
        ref = oracle.gradient(g.m, oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode).cycle)
        # fp32(1/L) vs the float64 reference: within one fp32 rounding
        assert np.allclose(grad, ref, rtol=2**-23, atol=0)
        assert np.count_nonzero(grad) == sol.cycle.numel()


def test_autograd_function_and_upstream_scale():
    g = synth.ring10k()
    rp, col, w = _dev(g.row_ptr), _dev(g.col_idx), _dev(g.w)
    wf = w.to(torch.float32).requires_grad_(True)
    lam = ocm.OCMFunction.apply(wf, rp, col, w, g.mode)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert abs(float(lam) - h.num / h.den) <= abs(h.num / h.den) * 2**-23
    (3.0 * lam).backward()
    ref = 3.0 * oracle.gradient(g.m, h.cycle)
    assert np.allclose(wf.grad.cpu().numpy(), ref, rtol=2**-22, atol=0)


def test_unique_cycle_construction_and_fd_on_diff1m():
    """Finite differences with integer +1 perturbations, 64 random edges plus
    every critical-cycle edge.  With the unique optimum C*, +1 on an edge of C*
    raises lambda* by exactly 1/|C*| and +1 elsewhere leaves it unchanged, so
    the fp32 gradient must match the exact difference to 1e-6 relative."""
    g, base_cycle = diff1m()
    gv = golden_values()["diff1m"]
    rp, col, w = _dev(g.row_ptr), _dev(g.col_idx), _dev(g.w)
    ws = ocm.make_workspace(g.n, g.m)
    sol = ocm.solve(rp, col, w, "max", workspace=ws)
    assert (sol.num, sol.den) == (int(gv["num"]), int(gv["den"]))
    cyc = sol.cycle.cpu().numpy()
    assert cyc.tolist() == base_cycle.tolist()
    lam0 = sol.value
    grad = ocm.backward(sol.cycle, torch.ones(1, device="cuda"), g.m).cpu().numpy()
    rng = np.random.default_rng(1111062704)
    edges = np.unique(np.concatenate([rng.integers(0, g.m, 64), cyc]))
    on_cycle = set(cyc.tolist())
    L = len(cyc)
    for e in edges:
        w_pert = w.clone()
        w_pert[int(e)] += 1
        fd = ocm.solve(rp, col, w_pert, "max", workspace=ws).value - lam0
        expect = Fraction(1, L) if int(e) in on_cycle else Fraction(0)
        assert fd == expect, int(e)
        if expect == 0:
            assert grad[int(e)] == 0.0
        else:
            assert abs(grad[int(e)] - float(expect)) <= 1e-6 * float(expect)
