"""Parity of the CUDA path with the CPU oracle (needs a GB300).

Every comparison is exact: the reduced mean num/den, the critical cycle as a
list of CSR edge indices, and the iteration count, because both sides follow
the same deterministic iteration with exact integers.  The per-vertex means
and potentials returned by the GPU must also satisfy the LP-dual certificate
(Eq. 1, Prop. 2.1), checked by the oracle's certificate routine."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from golden_io import GOLDEN, closed_forms, fig1

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _dev(g):
    d = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
            torch.from_numpy(g.w).to(d))


def gpu_solve(g, **kw):
    rp, col, w = _dev(g)
    return ocm.solve(rp, col, w, g.mode, **kw)


def assert_parity(g, sol, h=None, check_iters=True):
    if h is None:
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (sol.num, sol.den) == (h.num, h.den), g.name
    assert sol.cycle.cpu().numpy().tolist() == [int(x) for x in h.cycle], g.name
    if check_iters:
        assert sol.stats["iterations"] == h.iterations, g.name
    return h


def assert_certificate(g, sol):
    rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode,
                                 sol.eta_num.cpu().numpy(), sol.eta_den.cpu().numpy(),
                                 sol.potential.cpu().numpy(), sol.num, sol.den,
                                 sol.cycle.cpu().numpy())
    assert rc == 0, (g.name, rc, bad)


def golden_values():
    rows = {}
    with open(os.path.join(GOLDEN, "oracle_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, rest = line.split(" ", 1)
            if name.endswith("_cycle"):
                rows[name] = [int(x) for x in rest.split()]
                continue
            kv = {}
            head = rest.split(" head=")
            for tok in head[0].split():
                k, v = tok.split("=")
                kv[k] = v
            kv["head"] = [int(x) for x in head[1].split()] if len(head) > 1 else []
            rows[name] = kv
    return rows


# ------------------------------------------------------------- tiny graphs
@pytest.mark.parametrize("mode", ["max", "min"])
def test_tiny_random_graphs_exact(mode):
    rng = np.random.default_rng(20240 + (mode == "min"))
    for trial in range(250):
        n = int(rng.integers(1, 48))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-30, whi=30, ring=bool(trial % 2),
                              mode=mode)
        sol = gpu_solve(g, certificate=True)
        assert_parity(g, sol)
        assert_certificate(g, sol)


@pytest.mark.parametrize("cf", closed_forms(), ids=lambda c: c.name)
def test_closed_forms_gpu(cf):
    sol = gpu_solve(cf.graph)
    assert (sol.num, sol.den) == (cf.num, cf.den)
    if cf.cycle is not None:
        assert tuple(sol.cycle.cpu().numpy().tolist()) == cf.cycle


def test_fig1_gpu():
    f = fig1()
    for g, val, cyc in ((f.graph_max, f.max_value, f.max_cycle),
                        (f.graph_min, f.min_value, f.min_cycle)):
        sol = gpu_solve(g)
        assert (sol.num, sol.den) == val
        assert tuple(sol.cycle.cpu().numpy().tolist()) == cyc


# ----------------------------------------------------------- edge cases
def test_single_vertex_self_loop():
    g = synth.from_edges(1, [(0, 0, -7)])
    sol = gpu_solve(g, certificate=True)
    assert (sol.num, sol.den) == (-7, 1) and sol.cycle.cpu().tolist() == [0]


def test_all_self_loops_many_cycles():
    """n cycles in the first policy: exercises the exact ranking of many means."""
    rng = np.random.default_rng(4)
    n = 20000
    edges = []
    for v in range(n):
        edges.append((v, v, int(rng.integers(-1000, 1000))))
        edges.append((v, (v + 1) % n, int(rng.integers(-1000, 1000))))
    g = synth.from_edges(n, edges)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


@pytest.mark.parametrize("wrange", [(-1000, 1000), (-3, 3)], ids=["distinct", "duplicates"])
def test_rank_many_cycles_spread_over_blocks(wrange):
    """4,096 to 65,536 cycles in the first policy: the all-pairs rank count is
    split into pieces over every block and summed; duplicate keys (weights in
    -3..3) must still get equal ranks."""
    rng = np.random.default_rng(43 + wrange[1])
    n = 40000
    lo, hi = wrange
    edges = []
    for v in range(n):
        edges.append((v, v, int(rng.integers(lo, hi + 1)) + 2 * hi))
        edges.append((v, (v + 1) % n, int(rng.integers(lo, hi + 1))))
    g = synth.from_edges(n, edges)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


@pytest.mark.parametrize("wrange", [(-1000, 1000), (-3, 3)], ids=["distinct", "duplicates"])
def test_rank_many_cycles_by_radix(wrange):
    """More than 65,536 cycles in the first policy (heavy self-loops): the
    exact ranks come from the radix-sort path; with weights in -3..3 most of
    the 200,000 cycle means are equal (duplicate keys, negative keys)."""
    rng = np.random.default_rng(41 + wrange[1])
    n = 200000
    lo, hi = wrange
    edges = []
    for v in range(n):
        edges.append((v, v, int(rng.integers(lo, hi + 1)) + 2 * hi))
        edges.append((v, (v + 1) % n, int(rng.integers(lo, hi + 1))))
        edges.append((v, int(rng.integers(0, n)), int(rng.integers(lo, hi + 1))))
    g = synth.from_edges(n, edges)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


def test_long_single_ring_extraction():
    """A critical cycle with 2^17 + 3 edges (many lifting bits in extraction)."""
    n = (1 << 17) + 3
    rng = np.random.default_rng(5)
    w = rng.integers(-5, 6, size=n)
    g = synth.from_edges(n, [(i, (i + 1) % n, int(w[i])) for i in range(n)])
    sol = gpu_solve(g)
    from fractions import Fraction
    assert sol.value == Fraction(int(w.sum()), n)
    assert sol.cycle.cpu().numpy().tolist() == list(range(n))


def test_heavy_vertex_spans_many_chunks():
    """One vertex with 50,000 out-edges (more than a shared-memory chunk)."""
    rng = np.random.default_rng(6)
    n = 3000
    edges = [(0, int(t), int(x)) for t, x in zip(rng.integers(0, n, 50000),
                                                 rng.integers(-100, 100, 50000))]
    for v in range(1, n):
        edges.append((v, (v + 1) % n, int(rng.integers(-100, 100))))
        edges.append((v, int(rng.integers(0, n)), int(rng.integers(-100, 100))))
    g = synth.from_edges(n, edges)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


def test_non_strongly_connected_and_negative_weights():
    rng = np.random.default_rng(8)
    for trial in range(20):
        n = int(rng.integers(50, 400))
        g = synth.tiny_random(rng, n, max_extra=2, wlo=-10**6, whi=10**6, mode="min")
        sol = gpu_solve(g, certificate=True)
        assert_parity(g, sol)
        assert_certificate(g, sol)


def test_extreme_weights_within_bound():
    # 2 n^2 max|w| < 2^62 with max|w| = 2^31 - 1 allows n up to 2^15
    rng = np.random.default_rng(9)
    g = synth.tiny_random(rng, 1000, max_extra=3, wlo=-2**31 + 1, whi=2**31 - 1)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


def test_unaligned_input_slices():
    """col_idx / w / row_ptr starting at odd int32 offsets (tensor slices)."""
    g = synth.ring10k()
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    d = torch.device("cuda")
    for off in (1, 2, 3):
        def sl(a):
            buf = torch.zeros(a.shape[0] + off, dtype=torch.int32, device=d)
            buf[off:] = torch.from_numpy(a).to(d)
            return buf[off:]
        sol = ocm.solve(sl(g.row_ptr), sl(g.col_idx), sl(g.w), g.mode)
        assert (sol.num, sol.den) == (h.num, h.den)
        assert sol.cycle.cpu().numpy().tolist() == [int(x) for x in h.cycle]


def test_launch_parameters_do_not_change_results(tmp_path, monkeypatch):
    """Every sweep launch configuration gives the same bits; the autotuner
    picks one of them and records it for the graph's signature."""
    monkeypatch.setenv("OCM_TUNE_FILE", str(tmp_path / "tune.json"))
    g = synth.locality32m(1 << 16)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    rp, col, w = _dev(g)
    for kind, epls in ((ocm.ocm.OCM_SWEEP_CLASSES, (1, 2, 4, 8, 16, 64)),
                       (ocm.ocm.OCM_SWEEP_TILES, (4, 8, 16))):
        for epl in epls:
            for thr in (64, 128, 256, 512):
                sol = ocm.solve(rp, col, w, g.mode, edges_per_lane=epl, sweep_threads=thr,
                                sweep_kind=kind)
                assert (sol.num, sol.den) == (h.num, h.den)
                assert sol.cycle.cpu().numpy().tolist() == [int(x) for x in h.cycle]
                assert sol.stats["iterations"] == h.iterations
    cands = [(1, 2, 256), (2, 8, 128), (2, 4, 256)]
    res = ocm.autotune.tune(rp, col, w, g.mode, candidates=cands)
    picked = (res["sweep_kind"], res["edges_per_lane"], res["sweep_threads"])
    assert picked in cands
    assert ocm.autotune.lookup(rp) == picked
    sol = ocm.solve(rp, col, w, g.mode, tune=True)
    assert (sol.num, sol.den) == (h.num, h.den)


@pytest.mark.parametrize("epl", [4, 8])
def test_edge_tiles_against_degree_classes(epl):
    """The two sweep layouts make the same choices at every step: random
    graphs whose degrees straddle the tile and lane sizes (vertices inside a
    lane, across lanes, across tiles, and exactly filling them), compared
    with the oracle and with each other, including the iteration count and
    the number of switches."""
    rng = np.random.default_rng(4400 + epl)
    et = 32 * epl
    for trial in range(12):
        n = int(rng.integers(50, 1500))
        choices = np.array([1, 2, epl - 1, epl, epl + 1, et - 1, et, et + 1, 3 * et + 5])
        choices = choices[choices >= 1]
        deg = rng.choice(choices, size=n, p=None)
        edges = []
        for v in range(n):
            edges.append((v, (v + 1) % n, int(rng.integers(-50, 50))))
            for _ in range(int(deg[v]) - 1):
                edges.append((v, int(rng.integers(0, n)), int(rng.integers(-50, 50))))
        g = synth.from_edges(n, edges, mode="max" if trial % 2 else "min")
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        rp, col, w = _dev(g)
        a = ocm.solve(rp, col, w, g.mode, sweep_kind=ocm.ocm.OCM_SWEEP_TILES, edges_per_lane=epl)
        b = ocm.solve(rp, col, w, g.mode, sweep_kind=ocm.ocm.OCM_SWEEP_CLASSES)
        for s in (a, b):
            assert (s.num, s.den) == (h.num, h.den), trial
            assert s.cycle.cpu().numpy().tolist() == [int(x) for x in h.cycle], trial
            assert s.stats["iterations"] == h.iterations, trial
        assert a.stats["switched"] == b.stats["switched"], trial


def test_determinism_bitwise():
    g = synth.ring10k()
    a = gpu_solve(g, certificate=True)
    b = gpu_solve(g, certificate=True)
    assert (a.num, a.den) == (b.num, b.den)
    assert torch.equal(a.cycle, b.cycle)
    assert torch.equal(a.potential, b.potential) and torch.equal(a.eta_num, b.eta_num)
    assert torch.equal(a.policy, b.policy)


# -------------------------------------------------------------- errors
def _status(fn):
    with pytest.raises(ocm.OCMError) as ei:
        fn()
    return ei.value.status


def test_error_codes():
    d = torch.device("cuda")
    rp = torch.tensor([0, 1, 1, 2], dtype=torch.int32, device=d)   # vertex 1 has no out-edge
    col = torch.tensor([1, 0], dtype=torch.int32, device=d)
    w = torch.tensor([1, 1], dtype=torch.int32, device=d)
    assert _status(lambda: ocm.solve(rp, col, w)) == -3
    rp2 = torch.tensor([0, 2, 1, 2], dtype=torch.int32, device=d)  # not monotone
    assert _status(lambda: ocm.solve(rp2, col, w)) == -2
    rp3 = torch.tensor([0, 1, 2], dtype=torch.int32, device=d)
    col3 = torch.tensor([1, 5], dtype=torch.int32, device=d)       # target out of range
    assert _status(lambda: ocm.solve(rp3, col3, w)) == -2
    w3 = torch.tensor([1, -2**31], dtype=torch.int32, device=d)    # INT32_MIN
    col4 = torch.tensor([1, 0], dtype=torch.int32, device=d)
    assert _status(lambda: ocm.solve(rp3, col4, w3)) == -4
    # exactness bound 2 n^2 max|w| >= 2^62
    n = 1 << 16
    g = synth.from_edges(n, [(i, (i + 1) % n, 2**31 - 1) for i in range(n)])
    assert _status(lambda: gpu_solve(g)) == -4
    # iteration cap
    assert _status(lambda: gpu_solve(synth.ring10k(), max_iters=1)) == -5


def test_bounded_wait_expires_cleanly():
    """A grid barrier waits for an arrival that never comes (test flag): the
    bounded wait must expire, the solve must report OCM_ERR_TIMEOUT, and the
    device must stay usable for the next solve."""
    g = synth.ring10k()
    rp, col, w = _dev(g)
    out = torch.full((g.n,), 77, dtype=torch.int32, device="cuda")
    with pytest.raises(ocm.OCMError) as ei:
        ocm.solve(rp, col, w, g.mode, flags=ocm.ocm.OCM_FLAG_TEST_STALL, cycle_out=out)
    assert ei.value.status == -6
    assert int(out[0]) == 77
    sol = ocm.solve(rp, col, w, g.mode)
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    assert (sol.num, sol.den) == (h.num, h.den)


def test_errors_leave_outputs_untouched():
    d = torch.device("cuda")
    rp = torch.tensor([0, 1, 1, 2], dtype=torch.int32, device=d)
    col = torch.tensor([1, 0], dtype=torch.int32, device=d)
    w = torch.tensor([1, 1], dtype=torch.int32, device=d)
    out = torch.full((3,), 77, dtype=torch.int32, device=d)
    with pytest.raises(ocm.OCMError):
        ocm.solve(rp, col, w, cycle_out=out)
    assert out.cpu().tolist() == [77, 77, 77]


# ------------------------------------------------------------ workloads
def test_ring10k_exact_and_certified():
    g = synth.ring10k()
    sol = gpu_solve(g, certificate=True)
    h = assert_parity(g, sol)
    assert oracle.karp(g.row_ptr, g.col_idx, g.w, g.mode) == h.value
    assert_certificate(g, sol)


def test_product4_exact_and_certified():
    g = synth.product4()
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


def test_diff1m_exact_and_certified():
    gv = golden_values()
    base = synth.diff1m_base()
    sol = gpu_solve(base, certificate=True)
    assert_parity(base, sol)
    assert_certificate(base, sol)
    assert sol.cycle.cpu().numpy().tolist() == gv["diff1m_base_cycle"]


def test_locality_2_20_exact_and_certified():
    g = synth.locality32m(1 << 20)
    sol = gpu_solve(g, certificate=True)
    assert_parity(g, sol)
    assert_certificate(g, sol)


def test_locality32m_full_size_against_stored_oracle():
    """2^25 vertices, 2^28 edges: the oracle's answer is stored (it takes
    minutes on the CPU); the GPU's potentials are certified here in full."""
    gv = golden_values()["locality32m"]
    g = synth.locality32m()
    sol = gpu_solve(g, certificate=True)
    assert (sol.num, sol.den) == (int(gv["num"]), int(gv["den"]))
    cyc = sol.cycle.cpu().numpy()
    assert cyc.shape[0] == int(gv["len"])
    assert synth.digest(cyc) == int(gv["cycle_digest"])
    assert cyc[:16].tolist() == gv["head"]
    assert sol.stats["iterations"] == int(gv["iters"])
    assert_certificate(g, sol)


def test_batch_members_exact():
    graphs = synth.batch_graphs(G=24, nmin=100, nmax=20000)
    for g in graphs:
        sol = gpu_solve(g)
        assert_parity(g, sol)
