"""The paper's single-lambda form of the iteration (needs a GB300).

With OCM_FLAG_SINGLE_LAMBDA the CUDA path rebuilds the policy graph around the
chosen cycle after every evaluation (Alg. 1's "break all other cycles",
Alg. 2's markMinComponent / connectGpi / valuePropagate) and must follow the
oracle's single-lambda iteration exactly: value, critical cycle, iteration
count, final policy and final values (the oracle's, element by element).  At
full size the stored oracle answers stand in where the oracle takes minutes,
and the final values pass the LP-dual certificate in full."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from golden_io import GOLDEN, single_lambda_traces
from hub_graphs import in_hub_graph

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_STALL, OCM_SWEEP_TILES


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def _solve(g, t=None, **kw):
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    tt = _dev(t)[0] if t is not None else None
    return ocm.solve(rp, col, w, g.mode, single_lambda=True, transit=tt, **kw)


def _check(g, sol, t=None, s=None):
    if s is None:
        s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode, transit=t)
    assert (sol.num, sol.den) == (s.num, s.den), g.name
    assert sol.cycle.cpu().tolist() == s.cycle.tolist(), g.name
    assert sol.stats["iterations"] == s.iterations, g.name
    assert sol.stats["cycles"] == 1, g.name
    if sol.policy is not None:
        assert sol.policy.cpu().numpy().tolist() == s.policy.tolist(), g.name
        assert sol.potential.cpu().numpy().tolist() == s.V.tolist(), g.name
        p = s.num if g.mode == "max" else -s.num
        assert bool((sol.eta_num == p).all()) and bool((sol.eta_den == s.den).all()), g.name
    return s


def _stored():
    rows = {}
    with open(os.path.join(GOLDEN, "single_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, rest = line.split(" ", 1)
            body, head = rest.split(" head=")
            kv = dict(tok.split("=") for tok in body.split())
            kv["head"] = [int(x) for x in head.split()]
            rows[name] = kv
    return rows


@pytest.mark.parametrize("mode", ["max", "min"])
def test_tiny_strongly_connected_graphs_follow_the_oracle(mode):
    rng = np.random.default_rng(1111062810 + (mode == "min"))
    for trial in range(200):
        n = int(rng.integers(1, 60))
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-60, whi=60, ring=True, mode=mode)
        _check(g, _solve(g, certificate=trial % 3 == 0))


@pytest.mark.parametrize("tr", single_lambda_traces(), ids=lambda t: t.name)
def test_hand_traced_runs(tr):
    g = tr.graph
    sol = _solve(g, certificate=True)
    assert (sol.num, sol.den, sol.stats["iterations"]) == (tr.num, tr.den, tr.single_iters)
    assert tuple(sol.cycle.cpu().tolist()) == tr.cycle
    assert sol.policy.cpu().tolist() == tr.policy.tolist()
    assert sol.potential.cpu().tolist() == tr.values.tolist()


@pytest.mark.parametrize("name", ["ring10k", "diff1m_base"])
def test_workloads_against_the_oracle(name):
    g = getattr(synth, name)()
    _check(g, _solve(g, certificate=True))


def test_ratio_form():
    rng = np.random.default_rng(1111062812)
    for trial in range(120):
        n = int(rng.integers(1, 40))
        mode = "max" if trial % 2 == 0 else "min"
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-60, whi=60, ring=True, mode=mode)
        t = rng.integers(1, 9, size=g.m).astype(np.int32)
        _check(g, _solve(g, t, certificate=trial % 3 == 0), t=t)
    g = synth.ring10k()
    t = rng.integers(1, 101, size=g.m).astype(np.int32)
    _check(g, _solve(g, t, certificate=True), t=t)


def test_host_loop_and_graph_loop_agree():
    g = synth.ring10k()
    a = _solve(g, certificate=True)
    b = _solve(g, certificate=True, flags=OCM_FLAG_HOST_LOOP)
    assert a.stats["graph_loop"] == 1 and b.stats["graph_loop"] == 0
    assert (a.num, a.den, a.stats["iterations"], a.stats["rebuild_levels"]) == \
           (b.num, b.den, b.stats["iterations"], b.stats["rebuild_levels"])
    assert torch.equal(a.cycle, b.cycle) and torch.equal(a.potential, b.potential)
    assert torch.equal(a.policy, b.policy)


def test_a_vertex_that_cannot_reach_the_chosen_cycle_is_an_argument_error():
    g = synth.from_edges(4, [(0, 1, 5), (1, 0, 5), (2, 3, 1), (3, 2, 1)])
    with pytest.raises(ocm.OCMError) as ex:
        _solve(g)
    assert ex.value.status == -1
    # not strongly connected, but every vertex reaches the best cycle
    g = synth.from_edges(4, [(0, 1, 5), (1, 0, 5), (2, 3, 1), (2, 0, 0), (3, 2, 1)])
    _check(g, _solve(g, certificate=True))


def test_same_lambda_as_the_multichain_form():
    rng = np.random.default_rng(1111062813)
    for trial in range(40):
        g = synth.ring_extra(int(rng.integers(50, 5000)), 0, 5, -1000, 1000, 1,
                             seed=1111062813, tag=trial, mode="max" if trial % 2 else "min")
        rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
        a = ocm.solve(rp, col, w, g.mode)
        b = ocm.solve(rp, col, w, g.mode, single_lambda=True)
        assert (a.num, a.den) == (b.num, b.den), trial


@pytest.mark.parametrize("name", ["product4", "locality_2^20", "locality32m"])
def test_full_size_against_stored_oracle(name):
    """The oracle's single-lambda answers on the full workloads are stored
    (tests/golden/make_single_values.py); the GPU must match them exactly and
    its final values must certify lambda* in full."""
    sv = _stored()[name]
    g = synth.product4() if name == "product4" else \
        synth.locality32m(1 << 20) if name == "locality_2^20" else synth.locality32m()
    sol = _solve(g, certificate=True)
    assert (sol.num, sol.den) == (int(sv["num"]), int(sv["den"]))
    cyc = sol.cycle.cpu().numpy()
    assert cyc.shape[0] == int(sv["len"])
    assert synth.digest(cyc) == int(sv["cycle_digest"])
    assert cyc[:16].tolist() == sv["head"]
    assert sol.stats["iterations"] == int(sv["iters"])
    assert synth.digest(sol.policy.cpu().numpy()) == int(sv["policy_digest"])
    rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, sol.eta_num.cpu().numpy(),
                                 sol.eta_den.cpu().numpy(), sol.potential.cpu().numpy(), sol.num,
                                 sol.den, cyc)
    assert rc == 0, (name, rc, bad)


def test_warm_start_follows_the_oracle():
    rng = np.random.default_rng(1111062814)
    for trial in range(60):
        n = int(rng.integers(1, 300))
        mode = "max" if trial % 2 == 0 else "min"
        g = synth.tiny_random(rng, n, max_extra=4, wlo=-60, whi=60, ring=True, mode=mode)
        init = synth.random_policy(rng, g.row_ptr)
        s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, mode, init_policy=init)
        _check(g, _solve(g, init_policy=_dev(init)[0], certificate=True), s=s)
    g = synth.ring10k()
    first = _solve(g, certificate=True)
    again = _solve(g, init_policy=first.policy, certificate=True)
    assert (again.num, again.den, again.stats["iterations"]) == (first.num, first.den, 0)
    assert torch.equal(again.cycle, first.cycle) and torch.equal(again.potential, first.potential)


def test_edge_tiled_sweep_gives_the_same_iteration():
    for g in (synth.ring10k(), synth.locality32m(1 << 16)):
        a = _solve(g, certificate=True)
        b = _solve(g, certificate=True, sweep_kind=OCM_SWEEP_TILES)
        assert (a.num, a.den, a.stats["iterations"]) == (b.num, b.den, b.stats["iterations"])
        assert torch.equal(a.cycle, b.cycle) and torch.equal(a.policy, b.policy)
        assert torch.equal(a.potential, b.potential)


def test_bounded_wait_expires_cleanly_in_the_single_lambda_form():
    """The test flag makes the evaluation's first barrier wait for an arrival
    that never comes; the rebuild that follows must not wait either, and the
    device stays usable."""
    g = synth.ring10k()
    for flags in (OCM_FLAG_TEST_STALL, OCM_FLAG_TEST_STALL | OCM_FLAG_HOST_LOOP):
        with pytest.raises(ocm.OCMError) as ex:
            _solve(g, flags=flags)
        assert ex.value.status == -6
    _check(g, _solve(g))


@pytest.mark.parametrize("ring,chain,leaves", [(5, 300, 10000), (5, 300, 70000),
                                               (2000, 0, 10000), (2000, 0, 70000)])
def test_pushing_vertex_with_many_in_edges(ring, chain, leaves):
    """10,000 in-edges: spread over one block; 70,000: over the whole grid;
    after a chain the push runs through the frontier lists, from a large ring
    as a pass over all vertices.  The rebuild must equal the oracle's."""
    g = in_hub_graph(ring, chain, leaves)
    _check(g, _solve(g, certificate=True))


@pytest.mark.parametrize("sinks,wlo,whi", [(1, -1000, 1000), (1, -1000, -900), (12, -1000, 1000)])
def test_sinks_with_many_in_edges(sinks, wlo, whi):
    """A ring, three random edges per vertex and one edge to one of a few sink
    vertices (in-degrees up to about 100,000)."""
    rng = np.random.default_rng(1111062815 + sinks + wlo)
    n = 100_000
    rp = np.arange(n + 1, dtype=np.int64) * 5
    col = rng.integers(0, n, 5 * n).astype(np.int32)
    col[rp[:-1]] = (np.arange(n) + 1) % n
    col[rp[1:] - 1] = rng.integers(0, sinks, n)
    w = rng.integers(-1000, 1001, 5 * n).astype(np.int32)
    w[rp[1:] - 1] = rng.integers(wlo, whi + 1, n)
    g = synth.Graph(rp.astype(np.int32), col, w, "max", f"sinks({sinks},{wlo}..{whi})")
    _check(g, _solve(g, certificate=True))


def test_random_hubs_in_both_directions():
    """Random graphs mixing vertices with many out-edges (chunk scans) and
    sinks with many in-edges (block- and grid-spread pushes), both senses:
    the single-lambda iteration must equal the oracle's exactly."""
    rng = np.random.default_rng(1111062816)
    for trial in range(16):
        n = int(rng.integers(3000, 30000))
        extra = int(rng.integers(1, 4))
        out_hubs = rng.choice(n, int(rng.integers(0, 4)), replace=False)
        sinks = rng.choice(n, int(rng.integers(1, 4)), replace=False)
        to_sink = int(rng.integers(0, 6))     # parallel edges from every vertex to a sink
        deg = np.full(n, 1 + extra + to_sink, np.int64)
        deg[out_hubs] += rng.integers(1025, 20000, size=out_hubs.size)
        rp = np.zeros(n + 1, np.int64)
        np.cumsum(deg, out=rp[1:])
        m = int(rp[-1])
        col = rng.integers(0, n, m).astype(np.int32)
        col[rp[:-1]] = (np.arange(n) + 1) % n
        for j in range(to_sink):
            col[rp[1:] - 1 - j] = rng.choice(sinks, n)
        w = rng.integers(-1000, 1001, m).astype(np.int32)
        mode = "max" if trial % 2 == 0 else "min"
        g = synth.Graph(rp.astype(np.int32), col, w, mode, f"random_hubs#{trial}")
        _check(g, _solve(g, certificate=trial % 4 == 0))
