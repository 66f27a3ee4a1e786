"""Pins for the CPU oracle (no GPU): the oracle is checked against things other
than itself -- brute-force enumeration of every simple cycle, Karp's
independent recurrence, hand-computed closed forms (tests/golden), the
structure of Fig. 1, the LP-dual certificate (Eq. 1, Prop. 2.1), Prop. 2.2,
and invariances of the cycle mean (shift, scale, duality, relabelling,
monotonicity).  A dropped term, a wrong sign or index, or a transposed operand
in Howard's evaluation or improvement step changes the value or the cycle on
some of these thousands of graphs."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from golden_io import closed_forms, fig1, ratio_closed_forms, relabel, single_lambda_traces
import hub_graphs


def _frac(num, den):
    return Fraction(int(num), int(den))


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("mode", ["max", "min"])
def test_howard_matches_brute_force_and_karp_on_tiny_graphs(mode):
    rng = np.random.default_rng(1111062700 + (mode == "min"))
    for trial in range(1500):
        n = int(rng.integers(1, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=bool(trial % 3 == 0),
                              mode=mode)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, mode)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode)
        k = oracle.karp(g.row_ptr, g.col_idx, g.w, mode)
        assert h.value == b.value == k, (trial, n)
        # Howard's critical cycle is one of the optimal simple cycles, listed
        # from its smallest vertex
        assert tuple(int(e) for e in h.cycle) in b.optimal, (trial, h.cycle, b.optimal)
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, mode, h.eta_p, h.eta_q, h.V,
                                     h.num, h.den, h.cycle)
        assert rc == 0, (trial, rc, bad)


def test_howard_on_wide_weights_matches_brute_force():
    rng = np.random.default_rng(7)
    for trial in range(300):
        n = int(rng.integers(2, 8))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-2**31 + 1, whi=2**31 - 1)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, "max")
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, "max")
        assert h.value == b.value
        assert tuple(int(e) for e in h.cycle) in b.optimal


def test_brute_force_counts_cycles_of_complete_digraph():
    # K_4 with self-loops: simple cycles = 4 loops + C(4,2)*1 + C(4,3)*2 + C(4,4)*6 = 4+6+8+6
    edges = [(i, j, 1) for i in range(4) for j in range(4)]
    g = synth.from_edges(4, edges)
    b = oracle.brute(g.row_ptr, g.col_idx, g.w)
    assert b.ncycles == 24
    assert b.value == 1 and len(b.optimal) == 24


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("cf", closed_forms(), ids=lambda c: c.name)
def test_closed_forms(cf):
    g = cf.graph
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (h.num, h.den) == (cf.num, cf.den)
    assert oracle.karp(g.row_ptr, g.col_idx, g.w, g.mode) == _frac(cf.num, cf.den)
    if cf.cycle is not None:
        assert tuple(int(e) for e in h.cycle) == cf.cycle


def test_single_ring_closed_form_any_size():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 64, 1000):
        w = rng.integers(-1000, 1000, size=n)
        g = synth.from_edges(n, [(i, (i + 1) % n, int(w[i])) for i in range(n)])
        h = oracle.howard(g.row_ptr, g.col_idx, g.w)
        assert h.value == Fraction(int(w.sum()), n)
        assert list(h.cycle) == list(range(n))


def test_fig1_sccs_and_prop_2_2():
    f = fig1()
    k, comp = oracle.tarjan_scc(f.graph_max.row_ptr, f.graph_max.col_idx)
    assert k == 4
    groups = {}
    for v, c in enumerate(comp):
        groups.setdefault(int(c), set()).add(f.names[v])
    assert sorted(map(sorted, groups.values())) == sorted(map(sorted, f.sccs))
    for g, val, cyc in ((f.graph_max, f.max_value, f.max_cycle),
                        (f.graph_min, f.min_value, f.min_cycle)):
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        assert (h.num, h.den) == val
        assert tuple(int(e) for e in h.cycle) == cyc
        # Prop. 2.2: optimum over G = optimum over the optimal cycle means of its SCCs
        best = None
        for members in groups.values():
            ids = sorted(f.names.index(x) for x in members)
            sub = [(ids.index(s), ids.index(int(g.col_idx[e])), int(g.w[e]))
                   for s in ids for e in range(g.row_ptr[s], g.row_ptr[s + 1])
                   if int(g.col_idx[e]) in ids]
            if not sub:
                continue  # single vertex without a self-loop has no cycle
            sg = synth.from_edges(len(ids), sub, g.mode)
            if (np.diff(sg.row_ptr) == 0).any():
                continue
            v = oracle.brute(sg.row_ptr, sg.col_idx, sg.w, g.mode).value
            best = v if best is None else (max(best, v) if g.mode == "max" else min(best, v))
        assert best == _frac(*val)


def test_prop_2_2_random_non_strongly_connected():
    rng = np.random.default_rng(11)
    for trial in range(200):
        n = int(rng.integers(2, 9))
        g = synth.tiny_random(rng, n, max_extra=2, wlo=-20, whi=20)
        k, comp = oracle.tarjan_scc(g.row_ptr, g.col_idx)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w)
        best = None
        for c in range(k):
            ids = [v for v in range(n) if comp[v] == c]
            sub = [(ids.index(s), ids.index(int(g.col_idx[e])), int(g.w[e]))
                   for s in ids for e in range(g.row_ptr[s], g.row_ptr[s + 1])
                   if comp[g.col_idx[e]] == c]
            if not sub:
                continue
            deg = np.bincount([s for s, _, _ in sub], minlength=len(ids))
            if (deg == 0).any():
                continue
            sg = synth.from_edges(len(ids), sub)
            v = oracle.karp(sg.row_ptr, sg.col_idx, sg.w)
            best = v if best is None else max(best, v)
        assert h.value == best


# ------------------------------------------------------------------ invariants
def _graph_with(g, w):
    return synth.Graph(g.row_ptr, g.col_idx, np.asarray(w, dtype=np.int32), g.mode)


def test_invariants_shift_scale_duality_relabel_monotone():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(1, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-50, whi=50)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w)
        lam, cyc = h.value, tuple(h.cycle)
        # shift: lambda(w + c) = lambda(w) + c, same cycle
        c = int(rng.integers(-100, 100))
        hs = oracle.howard(g.row_ptr, g.col_idx, g.w + c)
        assert hs.value == lam + c and tuple(hs.cycle) == cyc
        # scale: lambda(k w) = k lambda(w), same cycle
        k = int(rng.integers(1, 50))
        hk = oracle.howard(g.row_ptr, g.col_idx, g.w * k)
        assert hk.value == lam * k and tuple(hk.cycle) == cyc
        # duality: min(w) = -max(-w), same cycle
        hm = oracle.howard(g.row_ptr, g.col_idx, -g.w, "min")
        assert hm.value == -lam and tuple(hm.cycle) == cyc
        # relabelling does not change the value
        perm = rng.permutation(n)
        r = relabel(g, perm)
        assert oracle.howard(r.row_ptr, r.col_idx, r.w).value == lam
        # adding an edge never lowers the maximum
        s, t = int(rng.integers(0, n)), int(rng.integers(0, n))
        edges = [(v, int(g.col_idx[e]), int(g.w[e])) for v in range(n)
                 for e in range(g.row_ptr[v], g.row_ptr[v + 1])]
        edges.append((s, t, int(rng.integers(-50, 50))))
        g2 = synth.from_edges(n, edges)
        assert oracle.howard(g2.row_ptr, g2.col_idx, g2.w).value >= lam


# ----------------------------------------------------------------- certificate
def test_certificate_rejects_planted_mistakes():
    """Plant mistakes in an oracle answer; the certificate must catch each."""
    rng = np.random.default_rng(9)
    caught = {1: 0, 2: 0, 5: 0, 6: 0}
    for trial in range(300):
        n = int(rng.integers(3, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=True)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w)
        args = (g.row_ptr, g.col_idx, g.w, "max")
        assert oracle.certificate(*args, h.eta_p, h.eta_q, h.V, h.num, h.den, h.cycle)[0] == 0
        # a value that is too small: the optimal cycle then violates (b) or (d)
        rc = oracle.certificate(*args, h.eta_p, h.eta_q, h.V, h.num - 1, h.den, h.cycle)[0]
        assert rc in (5, 6)
        caught[rc if rc in caught else 5] += 1
        # a potential perturbed at one vertex breaks a reduced-weight inequality
        # unless that vertex's constraints all have slack; try every vertex
        broke = False
        for v in range(n):
            V2 = h.V.copy()
            V2[v] += 1
            rc = oracle.certificate(*args, h.eta_p, h.eta_q, V2, h.num, h.den, h.cycle)[0]
            if rc:
                assert rc == 2
                broke = True
        assert broke  # at least the critical cycle's vertices are tight
        # claim a larger mean at one vertex only: (a) fails on an edge into it
        # or (d) fails
        v = int(rng.integers(0, n))
        ep = h.eta_p.copy()
        ep[v] += h.eta_q[v]
        rc = oracle.certificate(*args, ep, h.eta_q, h.V, h.num, h.den, h.cycle)[0]
        assert rc in (1, 2, 6)
    assert caught[5] + caught[6] == 300


def test_certificate_rejects_non_cycles():
    cf = {c.name: c for c in closed_forms()}["k3"]
    g = cf.graph
    h = oracle.howard(g.row_ptr, g.col_idx, g.w)
    args = (g.row_ptr, g.col_idx, g.w, "max", h.eta_p, h.eta_q, h.V, h.num, h.den)
    assert oracle.certificate(*args, h.cycle)[0] == 0
    assert oracle.certificate(*args, np.array([3], np.int32))[0] == 3       # not closed
    assert oracle.certificate(*args, np.array([3, 4], np.int32))[0] == 3    # not chained
    assert oracle.certificate(*args, np.array([3, 5, 3, 5], np.int32))[0] == 3  # longer than n
    assert oracle.certificate(*args, np.array([0, 2], np.int32))[0] == 5    # wrong mean
    sl = {c.name: c for c in closed_forms()}["selfloop"].graph
    hs = oracle.howard(sl.row_ptr, sl.col_idx, sl.w)
    a2 = (sl.row_ptr, sl.col_idx, sl.w, "max", hs.eta_p, hs.eta_q, hs.V, hs.num, hs.den)
    assert oracle.certificate(*a2, np.array([2], np.int32))[0] == 0
    assert oracle.certificate(*a2, np.array([2, 2], np.int32))[0] == 4     # not simple


# ------------------------------------------------------------- error handling
def test_oracle_rejects_bad_input():
    g = synth.from_edges(3, [(0, 1, 1), (1, 0, 1), (2, 0, 1)])
    with pytest.raises(oracle.OracleError):
        oracle.howard(g.row_ptr, g.col_idx, np.array([1, 1, -2**31], np.int32))
    rp = np.array([0, 1, 1, 2], np.int32)   # vertex 1 has no out-edge
    with pytest.raises(oracle.OracleError) as ei:
        oracle.howard(rp, np.array([1, 0], np.int32), np.array([1, 1], np.int32))
    assert ei.value.code == -3
    with pytest.raises(oracle.OracleError):
        oracle.howard(np.array([0, 1], np.int32), np.array([5], np.int32),
                      np.array([1], np.int32))


def test_iteration_cap_reports_not_converged():
    g = synth.ring10k()
    with pytest.raises(oracle.OracleError) as ei:
        oracle.howard(g.row_ptr, g.col_idx, g.w, "max", max_iter=1)
    assert ei.value.code == -5


# ------------------------------------------------------------- workload sizes
@pytest.mark.slow
def test_karp_equals_howard_on_ring10k():
    g = synth.ring10k()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert oracle.karp(g.row_ptr, g.col_idx, g.w, g.mode) == h.value
    rc, _ = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, h.eta_p, h.eta_q, h.V,
                               h.num, h.den, h.cycle)
    assert rc == 0


def test_karp_equals_howard_on_small_batch_members():
    graphs = synth.batch_graphs(G=12, nmin=100, nmax=600)
    for g in graphs:
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        assert oracle.karp(g.row_ptr, g.col_idx, g.w, g.mode) == h.value


def test_gradient_is_one_over_cycle_length():
    cf = {c.name: c for c in closed_forms()}["ring5"]
    g = cf.graph
    h = oracle.howard(g.row_ptr, g.col_idx, g.w)
    grad = oracle.gradient(g.m, h.cycle)
    assert np.allclose(grad, 1 / 5)
    # finite difference on the closed form: +1 on any ring edge adds 1/5
    for e in range(g.m):
        w2 = g.w.copy()
        w2[e] += 1
        assert oracle.howard(g.row_ptr, g.col_idx, w2).value - h.value == Fraction(1, 5)


# Gradient pins on closed forms with edges OFF the critical cycle (ring5 has
# none).  The expected gradient comes from the fixture alone: 1/|C*| on the
# fixture's hand-derived cycle and exactly 0 on every other edge (ratio:
# 1/t(C*)).  The weights are scaled by K first (lambda(K w) = K lambda(w), same
# critical cycle), so that +1 on any single edge cannot change which cycle is
# optimal: the finite difference of the oracle's exact value must then equal
# the gradient exactly, edge by edge.
_K = 1000
_GRAD_FORMS = ["ring5", "selfloop", "tworings_max", "tworings_min", "k3", "k3_min"]


def _exact_fd(g, w, mode, base, transit=None):
    out = []
    for e in range(g.m):
        w2 = w.copy()
        w2[e] += 1
        out.append(oracle.howard(g.row_ptr, g.col_idx, w2, mode, transit=transit).value - base)
    return out


def _hand_gradient(m, cycle, denom):
    g = np.zeros(m, np.float64)
    g[list(cycle)] = 1.0 / denom
    return g


@pytest.mark.parametrize("name", _GRAD_FORMS)
def test_gradient_pinned_by_exact_finite_differences(name):
    cf = {c.name: c for c in closed_forms()}[name]
    g = cf.graph
    wk = (g.w.astype(np.int64) * _K).astype(np.int32)
    base = oracle.howard(g.row_ptr, g.col_idx, wk, g.mode)
    assert base.value == Fraction(cf.num * _K, cf.den)
    L = len(cf.cycle)
    expected = _hand_gradient(g.m, cf.cycle, L)
    assert np.array_equal(oracle.gradient(g.m, base.cycle), expected)
    fd = _exact_fd(g, wk, g.mode, base.value)
    for e in range(g.m):
        assert fd[e] == (Fraction(1, L) if e in cf.cycle else 0), (name, e)
        assert float(fd[e]) == expected[e]


def test_gradient_pin_rejects_planted_mistakes():
    """The finite-difference pin above tells a right gradient from plausible
    wrong ones: 1/|C*| on every edge, 1/m everywhere, 1/(|C*|+1) on C*, and the
    right value on all but one edge of C*."""
    cf = {c.name: c for c in closed_forms()}["tworings_max"]
    g = cf.graph
    wk = (g.w.astype(np.int64) * _K).astype(np.int32)
    base = oracle.howard(g.row_ptr, g.col_idx, wk, g.mode)
    fd = np.array([float(x) for x in _exact_fd(g, wk, g.mode, base.value)])
    L = len(cf.cycle)
    assert np.array_equal(oracle.gradient(g.m, base.cycle), fd)
    dropped = _hand_gradient(g.m, cf.cycle, L)
    dropped[cf.cycle[0]] = 0.0
    for bad in (np.full(g.m, 1.0 / L), np.full(g.m, 1.0 / g.m),
                _hand_gradient(g.m, cf.cycle, L + 1), dropped):
        assert not np.array_equal(bad, fd)


_RATIO_GRAD_FORMS = ["ring3", "mean_vs_ratio_max", "mean_vs_ratio_min", "ring5_t4",
                     "negative_max", "negative_min"]


@pytest.mark.parametrize("name", _RATIO_GRAD_FORMS)
def test_gradient_ratio_pinned_by_exact_finite_differences(name):
    rf = {r.name: r for r in ratio_closed_forms()}[name]
    g = rf.graph
    wk = (g.w.astype(np.int64) * _K).astype(np.int32)
    base = oracle.howard(g.row_ptr, g.col_idx, wk, g.mode, transit=rf.transit)
    assert base.value == Fraction(rf.num * _K, rf.den)
    tC = int(sum(int(rf.transit[e]) for e in rf.cycle))
    expected = _hand_gradient(g.m, rf.cycle, tC)
    assert np.array_equal(oracle.gradient_ratio(g.m, base.cycle, rf.transit), expected)
    fd = _exact_fd(g, wk, g.mode, base.value, transit=rf.transit)
    for e in range(g.m):
        assert fd[e] == (Fraction(1, tC) if e in rf.cycle else 0), (name, e)
        assert float(fd[e]) == expected[e]
    # a gradient that ignored the times (1/|C*|) is told apart wherever t != 1
    if tC != len(rf.cycle):
        assert not np.array_equal(oracle.gradient(g.m, base.cycle), expected)


# ----------------------------------------------------------------- warm start
# Policy iteration reaches an optimal policy from any start (Sec. 2.4): the
# value from a random start policy must still be the brute-force optimum and
# carry a valid certificate, and a start from the final policy must stop at
# once with the same answer.
@pytest.mark.parametrize("mode", ["max", "min"])
def test_warm_start_from_random_policies_reaches_the_optimum(mode):
    rng = np.random.default_rng(1111062750 + (mode == "min"))
    for trial in range(600):
        n = int(rng.integers(1, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=bool(trial % 2), mode=mode)
        init = synth.random_policy(rng, g.row_ptr)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, mode, init_policy=init)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode)
        assert h.value == b.value, (trial, n)
        assert tuple(int(e) for e in h.cycle) in b.optimal, trial
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, mode, h.eta_p, h.eta_q, h.V,
                                     h.num, h.den, h.cycle)
        assert rc == 0, (trial, rc, bad)


def test_warm_start_from_the_final_policy_stops_at_once():
    rng = np.random.default_rng(1111062752)
    graphs = [synth.tiny_random(rng, int(rng.integers(1, 9)), max_extra=3) for _ in range(200)]
    graphs.append(synth.ring10k())
    for g in graphs:
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        h2 = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, init_policy=h.policy)
        assert h2.iterations == 0
        assert (h2.num, h2.den) == (h.num, h.den)
        assert h2.cycle.tolist() == h.cycle.tolist()
        assert h2.policy.tolist() == h.policy.tolist()


def test_warm_start_after_a_weight_change_matches_a_cold_solve_in_value():
    # the use the option exists for: re-solve after perturbing some weights,
    # starting from the previous optimal policy
    g = synth.ring10k()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    rng = np.random.default_rng(1111062753)
    w2 = g.w.copy()
    idx = rng.integers(0, g.m, size=50)
    w2[idx] += rng.integers(-20, 21, size=50).astype(np.int32)
    cold = oracle.howard(g.row_ptr, g.col_idx, w2, g.mode)
    warm = oracle.howard(g.row_ptr, g.col_idx, w2, g.mode, init_policy=h.policy)
    assert warm.value == cold.value == oracle.karp(g.row_ptr, g.col_idx, w2, g.mode)
    rc, _ = oracle.certificate(g.row_ptr, g.col_idx, w2, g.mode, warm.eta_p, warm.eta_q, warm.V,
                               warm.num, warm.den, warm.cycle)
    assert rc == 0


def test_warm_start_rejects_an_edge_of_another_vertex():
    g = synth.from_edges(3, [(0, 1, 1), (1, 2, 1), (2, 0, 1), (2, 2, 5)])
    with pytest.raises(oracle.OracleError) as e:
        oracle.howard(g.row_ptr, g.col_idx, g.w, init_policy=np.array([0, 0, 2], np.int32))
    assert e.value.code == -1
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, init_policy=np.array([0, 1, 2], np.int32))
    assert h.value == 5


# ---------------------------------------------------------- optimal cycle ratio
# The cost/time labels of Sec. 2.2 give the optimal cycle ratio w(C)/t(C).
# Pins: unit times reproduce the mean oracle bit for bit; brute-force
# enumeration of every simple cycle on thousands of tiny graphs; hand-derived
# closed forms (tests/golden/ratio_closed_forms.txt); scaling of w and t.
def test_ratio_with_unit_times_is_the_mean():
    rng = np.random.default_rng(1111062770)
    graphs = [synth.tiny_random(rng, int(rng.integers(1, 12)), max_extra=3, wlo=-20, whi=20)
              for _ in range(300)] + [synth.ring10k()]
    for g in graphs:
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        r = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=np.ones(g.m, np.int32))
        assert (r.num, r.den, r.iterations) == (h.num, h.den, h.iterations)
        assert r.cycle.tolist() == h.cycle.tolist()
        assert (r.V == h.V).all() and (r.eta_p == h.eta_p).all() and (r.eta_q == h.eta_q).all()


@pytest.mark.parametrize("mode", ["max", "min"])
def test_ratio_matches_brute_force_on_tiny_graphs(mode):
    rng = np.random.default_rng(1111062771 + (mode == "min"))
    for trial in range(1200):
        n = int(rng.integers(1, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=bool(trial % 3 == 0),
                              mode=mode)
        t = rng.integers(1, 6, size=g.m).astype(np.int32)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, mode, transit=t)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode, transit=t)
        assert h.value == b.value, (trial, n)
        assert tuple(int(e) for e in h.cycle) in b.optimal, trial
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, mode, h.eta_p, h.eta_q, h.V,
                                     h.num, h.den, h.cycle, transit=t)
        assert rc == 0, (trial, rc, bad)


@pytest.mark.parametrize("rf", ratio_closed_forms(), ids=lambda r: r.name)
def test_ratio_closed_forms(rf):
    g = rf.graph
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=rf.transit)
    assert (h.num, h.den) == (rf.num, rf.den)
    assert tuple(int(e) for e in h.cycle) == rf.cycle
    b = oracle.brute(g.row_ptr, g.col_idx, g.w, g.mode, transit=rf.transit)
    assert b.value == Fraction(rf.num, rf.den)


def test_ratio_scaling_and_duality():
    rng = np.random.default_rng(1111062773)
    for trial in range(200):
        g = synth.tiny_random(rng, int(rng.integers(2, 10)), max_extra=3, wlo=-30, whi=30)
        t = rng.integers(1, 8, size=g.m).astype(np.int32)
        base = oracle.howard(g.row_ptr, g.col_idx, g.w, "max", transit=t).value
        k = int(rng.integers(2, 5))
        assert oracle.howard(g.row_ptr, g.col_idx, g.w * k, "max", transit=t).value == k * base
        assert oracle.howard(g.row_ptr, g.col_idx, g.w, "max", transit=t * k).value == base / k
        lo = oracle.howard(g.row_ptr, g.col_idx, -g.w, "min", transit=t).value
        assert lo == -base


def test_ratio_rejects_nonpositive_times():
    g = synth.from_edges(2, [(0, 1, 1), (1, 0, 1)])
    with pytest.raises(oracle.OracleError):
        oracle.howard(g.row_ptr, g.col_idx, g.w, transit=np.array([1, 0], np.int32))


# ------------------------------------------- strongly connected components
# Tarjan's decomposition (the front-end of Sec. 3.3) against its definition:
# u and v share a component iff each reaches the other (brute-force closure);
# the per-component optimum against brute-force cycle enumeration (Prop. 2.2:
# the graph's optimum is the best component's).
def _reach(g):
    n = g.n
    R = np.eye(n, dtype=bool)
    for v in range(n):
        for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
            R[v, g.col_idx[e]] = True
    for k in range(n):
        R |= R[:, [k]] & R[[k], :]
    return R


def test_tarjan_matches_mutual_reachability():
    from scc_helpers import canonical_labels
    rng = np.random.default_rng(1111062790)
    for trial in range(400):
        n = int(rng.integers(1, 14))
        g = synth.random_digraph(rng, n, avg_deg=float(rng.uniform(0.3, 2.5)), sink_frac=0.2)
        R = _reach(g)
        lab = canonical_labels(g.row_ptr, g.col_idx)
        same = R & R.T
        for u in range(n):
            expect = int(np.nonzero(same[u])[0].min())
            assert lab[u] == expect, (trial, u)


def test_per_component_optima_match_brute_force():
    from scc_helpers import components
    rng = np.random.default_rng(1111062791)
    for trial in range(300):
        n = int(rng.integers(1, 10))
        g = synth.random_digraph(rng, n, avg_deg=float(rng.uniform(0.5, 2.5)), sink_frac=0.15)
        comps = components(g)
        has_cycle = any(True for _ in comps)
        if not has_cycle:
            continue
        best = max(Fraction(num, den) for _, num, den, _ in comps)
        assert best == oracle.brute(g.row_ptr, g.col_idx, g.w, "max").value, trial


# ------------------------------------------------- the paper's single-lambda form
# Alg. 1 as written: one lambda, every other policy cycle broken each iteration
# so that all vertices reach the chosen one.  Pins: brute-force enumeration and
# Karp on thousands of strongly connected tiny graphs (a ring through all
# vertices makes them so), the LP-dual certificate of the final values with
# every vertex at lambda* (it also pins the values and the single-cycle
# policy), the ratio form against brute force, and the error on a vertex that
# cannot reach the chosen cycle.
def _single_cycle_policy(g, policy):
    succ = g.col_idx[policy]
    roots = set()
    for v in range(g.n):
        seen, x = set(), v
        while x not in seen:
            seen.add(x)
            x = int(succ[x])
        # x is on v's cycle; name the cycle by its smallest vertex
        cyc, y = [x], int(succ[x])
        while y != x:
            cyc.append(y)
            y = int(succ[y])
        roots.add(min(cyc))
    return len(roots) == 1


@pytest.mark.parametrize("mode", ["max", "min"])
def test_single_lambda_matches_brute_force_on_strongly_connected_graphs(mode):
    rng = np.random.default_rng(1111062800 + (mode == "min"))
    for trial in range(1200):
        n = int(rng.integers(1, 9))
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=True, mode=mode)
        s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, mode)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode)
        assert s.value == b.value == oracle.karp(g.row_ptr, g.col_idx, g.w, mode), trial
        assert tuple(int(e) for e in s.cycle) in b.optimal, (trial, s.cycle, b.optimal)
        assert _single_cycle_policy(g, s.policy), trial
        # every vertex reaches the one cycle: eta = lambda* (max sense) everywhere
        p = s.num if mode == "max" else -s.num
        ep = np.full(n, p, np.int64)
        eq = np.full(n, s.den, np.int64)
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, mode, ep, eq, s.V, s.num, s.den,
                                     s.cycle)
        assert rc == 0, (trial, rc, bad)


def test_single_lambda_ratio_matches_brute_force():
    rng = np.random.default_rng(1111062802)
    for trial in range(800):
        n = int(rng.integers(1, 9))
        mode = "max" if trial % 2 == 0 else "min"
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=True, mode=mode)
        t = rng.integers(1, 6, size=g.m).astype(np.int32)
        s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, mode, transit=t)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode, transit=t)
        assert s.value == b.value, trial
        assert tuple(int(e) for e in s.cycle) in b.optimal, trial
        p = s.num if mode == "max" else -s.num
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, mode, np.full(n, p, np.int64),
                                     np.full(n, s.den, np.int64), s.V, s.num, s.den, s.cycle,
                                     transit=t)
        assert rc == 0, (trial, rc, bad)


def test_single_lambda_agrees_with_multichain_in_value_on_larger_graphs():
    g = synth.ring10k()
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (s.num, s.den) == (h.num, h.den)
    assert s.value == oracle.karp(g.row_ptr, g.col_idx, g.w, g.mode)


def test_single_lambda_needs_every_vertex_to_reach_the_chosen_cycle():
    # two separate 2-cycles of means 5 and 1: the second cannot reach the first
    g = synth.from_edges(4, [(0, 1, 5), (1, 0, 5), (2, 3, 1), (3, 2, 1)])
    with pytest.raises(oracle.OracleError) as ex:
        oracle.howard_single(g.row_ptr, g.col_idx, g.w)
    assert ex.value.code == -8
    # the same with a bridge 2 -> 0: not strongly connected, but every vertex
    # reaches the best cycle, and the answer is the optimum
    g = synth.from_edges(4, [(0, 1, 5), (1, 0, 5), (2, 3, 1), (2, 0, 0), (3, 2, 1)])
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w)
    assert (s.num, s.den) == (5, 1)


@pytest.mark.parametrize("tr", single_lambda_traces(), ids=lambda t: t.name)
def test_single_lambda_hand_traces(tr):
    g = tr.graph
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (s.num, s.den, s.iterations) == (tr.num, tr.den, tr.single_iters)
    assert tuple(int(e) for e in s.cycle) == tr.cycle
    assert s.policy.tolist() == tr.policy.tolist()
    assert s.V.tolist() == tr.values.tolist()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (h.num, h.den, h.iterations) == (tr.num, tr.den, tr.multichain_iters)
    assert tuple(int(e) for e in h.cycle) == tr.cycle


def test_single_lambda_warm_start_reaches_the_optimum():
    rng = np.random.default_rng(1111062804)
    for trial in range(400):
        n = int(rng.integers(1, 9))
        mode = "max" if trial % 2 == 0 else "min"
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-9, whi=9, ring=True, mode=mode)
        init = synth.random_policy(rng, g.row_ptr)
        s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, mode, init_policy=init)
        b = oracle.brute(g.row_ptr, g.col_idx, g.w, mode)
        assert s.value == b.value, trial
        assert tuple(int(e) for e in s.cycle) in b.optimal, trial
        # resuming from the final policy stops at once with the same answer
        r = oracle.howard_single(g.row_ptr, g.col_idx, g.w, mode, init_policy=s.policy)
        assert (r.num, r.den, r.iterations) == (s.num, s.den, 0), trial
        assert r.cycle.tolist() == s.cycle.tolist() and r.V.tolist() == s.V.tolist()


@pytest.mark.parametrize("args", [(2000, 3000, (2600, 1500)), (3, 1100, (7,)),
                                  (1, 2048, (1024, 1023, 2047))])
def test_single_lambda_rebuild_closed_form_heavy_sources(args):
    """Alg. 1's rebuild re-points every vertex to its smallest-index edge into
    the levels below it (reading: smallest index).  On the chain graph of
    hub_graphs the result is known edge by edge: the ring keeps lambda* = 100,
    each heavy vertex takes its first edge to c_L (wherever it lies among
    its 1,024-edge chunks), and V(v) = w(pi(v)) + V(succ(v)) - 100."""
    L, deg, hits = args
    g = hub_graphs.chain_hub_graph(L, deg, list(hits))
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
    pi, V = hub_graphs.chain_hub_expected(g, L, deg, list(hits))
    assert (s.num, s.den, s.iterations) == (100, 1, 0)
    assert s.cycle.tolist() == [0, 1, 2, 3, 4]
    assert s.policy.tolist() == pi.tolist()
    assert s.V.tolist() == V.tolist()


@pytest.mark.parametrize("args", [(5, 300, 10000), (2000, 0, 70000), (1, 0, 5), (3, 2, 1)])
def test_single_lambda_rebuild_closed_form_many_in_edges(args):
    """The same rule on a vertex whose level pushes over all its in-edges at
    once (after a chain, or straight from the ring; also a one-vertex ring,
    i.e. a self-loop, as the chosen cycle)."""
    ring, chain, leaves = args
    g = hub_graphs.in_hub_graph(ring, chain, leaves)
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
    pi, V = hub_graphs.in_hub_expected(g, ring, chain, leaves)
    assert (s.num, s.den, s.iterations) == (100, 1, 0)
    assert s.cycle.tolist() == list(range(ring))
    assert s.policy.tolist() == pi.tolist()
    assert s.V.tolist() == V.tolist()


def test_stored_batch_answers_match_a_fresh_oracle_run():
    """tests/golden/batch4096_values.txt (written by make_batch_values.py) holds
    the oracle's answer for each member of the batched workload; a seeded
    sample of the small members is re-solved here and must match line by line
    (value, cycle length, iterations, cycle digest, first edge)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "batch4096_values.txt")
    rows = [tuple(int(x) for x in l.split()) for l in open(path) if not l.startswith("#")]
    assert [r[0] for r in rows] == list(range(4096))
    sizes = synth.loguniform_sizes(4096, 100, 200000, synth.SEED_BASE + 3)
    assert [r[1] for r in rows] == [int(s) for s in sizes]
    small = [g for g in range(4096) if sizes[g] <= 3000]
    pick = np.random.default_rng(1111062704).choice(small, 12, replace=False)
    for g in sorted(int(x) for x in pick):
        gr = synth.ring_extra(int(sizes[g]), 0, 7, 1, 10000, 1, seed=synth.SEED_BASE + 3,
                              tag=1000 + g, mode="max")
        h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
        cyc = np.asarray(h.cycle, np.int32)
        assert rows[g] == (g, gr.n, gr.m, h.num, h.den, len(cyc), h.iterations,
                           synth.digest(cyc), int(cyc[0])), g
