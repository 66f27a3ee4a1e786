"""Vertices with more than 1,024 out-edges (needs a GB300).

Such a vertex leaves the lane-group classes of the improvement sweep: the
edges of all heavy vertices form one sequence cut into chunks of 1,024, each
chunk's block keeps the best candidate of the (at most two) heavy vertices it
meets, and one block per heavy vertex combines them; the initial policy and
the input checks of heavy vertices run the same way.  Results must equal the
oracle's exactly (value, critical cycle, iteration count, certificate) in
every form -- mean and ratio, both senses, warm start, batch, single-lambda
(whose rebuild scans heavy vertices' edges grid-wide) -- and errors on heavy
edges must be reported as on any other edge."""
import numpy as np
import pytest
import torch

import oracle
import synth
from hub_graphs import chain_hub_graph

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def hub_graph(rng, n, hubs, lo, hi, wlo=-1000, whi=1000, mode="max", extra=3):
    """A ring plus `extra` random out-edges per vertex; `hubs` vertices get
    U[lo, hi] more (random targets, duplicates allowed)."""
    deg = np.full(n, 1 + extra, np.int64)
    hv = rng.choice(n, hubs, replace=False)
    deg[hv] += rng.integers(lo, hi + 1, size=hubs)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    m = int(rp[-1])
    col = rng.integers(0, n, m).astype(np.int32)
    col[rp[:-1]] = (np.arange(n) + 1) % n
    w = rng.integers(wlo, whi + 1, m).astype(np.int32)
    return synth.Graph(rp.astype(np.int32), col, w, mode, f"hub(n={n},hubs={hubs},{lo}..{hi})")


def _check(g, sol, t=None, init=None):
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode, transit=t, init_policy=init)
    assert (sol.num, sol.den) == (h.num, h.den), g.name
    assert sol.cycle.cpu().tolist() == h.cycle.tolist(), g.name
    assert sol.stats["iterations"] == h.iterations, g.name
    if sol.eta_num is not None:
        rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, sol.eta_num.cpu().numpy(),
                                     sol.eta_den.cpu().numpy(), sol.potential.cpu().numpy(),
                                     sol.num, sol.den, sol.cycle.cpu().numpy(), transit=t)
        assert rc == 0, (g.name, rc, bad)


CASES = [(20000, 1, 60000, 60000), (20000, 7, 1025, 5000), (5000, 40, 1000, 3000),
         (3000, 3000, 1025, 1100)]   # the last: every vertex is heavy


@pytest.mark.parametrize("n,hubs,lo,hi", CASES)
@pytest.mark.parametrize("mode", ["max", "min"])
def test_heavy_vertices_follow_the_oracle(n, hubs, lo, hi, mode):
    rng = np.random.default_rng(1111062820 + n + hubs + (mode == "min"))
    g = hub_graph(rng, n, hubs, lo, hi, mode=mode)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    _check(g, ocm.solve(rp, col, w, mode, certificate=True))


def test_heavy_edge_tiled_layout_and_tuning_agree():
    rng = np.random.default_rng(1111062821)
    g = hub_graph(rng, 20000, 5, 2000, 30000)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    a = ocm.solve(rp, col, w, g.mode, certificate=True)
    for kw in (dict(sweep_kind=ocm.ocm.OCM_SWEEP_TILES), dict(edges_per_lane=64),
               dict(edges_per_lane=1, sweep_threads=128)):
        b = ocm.solve(rp, col, w, g.mode, certificate=True, **kw)
        assert (a.num, a.den, a.stats["iterations"]) == (b.num, b.den, b.stats["iterations"])
        assert torch.equal(a.cycle, b.cycle) and torch.equal(a.policy, b.policy)
        assert torch.equal(a.potential, b.potential)


def test_heavy_ratio_and_warm_start():
    rng = np.random.default_rng(1111062822)
    g = hub_graph(rng, 8000, 6, 1100, 20000)
    t = rng.integers(1, 50, size=g.m).astype(np.int32)
    rp, col, w, tt = _dev(g.row_ptr, g.col_idx, g.w, t)
    _check(g, ocm.solve(rp, col, w, g.mode, transit=tt, certificate=True), t=t)
    init = synth.random_policy(rng, g.row_ptr)
    _check(g, ocm.solve(rp, col, w, g.mode, init_policy=_dev(init)[0], certificate=True), init=init)


def test_heavy_vertices_in_a_batch():
    rng = np.random.default_rng(1111062823)
    members = [hub_graph(rng, 3000, 2, 1025, 9000), synth.ring10k(),
               hub_graph(rng, 1500, 1500, 1025, 1030)]
    b = synth.concat(members)
    sol = ocm.solve_batch(*_dev(b.graph_vptr, b.row_ptr, b.col_idx, b.w), b.mode)
    for k, g in enumerate(members):
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        assert (int(sol.num[k]), int(sol.den[k])) == (h.num, h.den), k
        assert sol.cycle(k).cpu().tolist() == [int(x) + int(b.row_ptr[b.graph_vptr[k]])
                                               for x in h.cycle], k


def _check_single(g, sol, t=None):
    s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode, transit=t)
    assert (sol.num, sol.den, sol.stats["iterations"]) == (s.num, s.den, s.iterations), g.name
    assert sol.cycle.cpu().tolist() == s.cycle.tolist(), g.name
    assert sol.policy.cpu().tolist() == s.policy.tolist(), g.name
    assert sol.potential.cpu().tolist() == s.V.tolist(), g.name


@pytest.mark.parametrize("n,hubs,lo,hi", CASES + [(6000, 4, 2000, 12000)])
@pytest.mark.parametrize("mode", ["max", "min"])
def test_heavy_vertices_in_the_single_lambda_form(n, hubs, lo, hi, mode):
    """The rebuild scans a heavy vertex's out-edges grid-wide, in chunks; the
    edge it takes must still be its smallest-index edge into the connected
    levels, as in the oracle."""
    rng = np.random.default_rng(1111062824 + n + hubs + (mode == "min"))
    g = hub_graph(rng, n, hubs, lo, hi, mode=mode)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    _check_single(g, ocm.solve(rp, col, w, mode, single_lambda=True, certificate=True))


def test_heavy_vertices_join_a_listed_level_in_the_single_lambda_form():
    g = chain_hub_graph(2000, 3000, [2600, 1500])
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    sol = ocm.solve(rp, col, w, g.mode, single_lambda=True, certificate=True)
    assert sol.stats["rebuild_levels"] >= 2001
    _check_single(g, sol)
    rng = np.random.default_rng(1111062826)
    t = rng.integers(1, 9, size=g.m).astype(np.int32)
    _check_single(g, ocm.solve(rp, col, w, g.mode, single_lambda=True, transit=_dev(t)[0],
                               certificate=True), t=t)


def test_heavy_vertices_in_the_single_lambda_ratio_form():
    rng = np.random.default_rng(1111062827)
    g = hub_graph(rng, 8000, 6, 1100, 20000)
    t = rng.integers(1, 50, size=g.m).astype(np.int32)
    rp, col, w, tt = _dev(g.row_ptr, g.col_idx, g.w, t)
    _check_single(g, ocm.solve(rp, col, w, g.mode, single_lambda=True, transit=tt,
                               certificate=True), t=t)


def test_errors_on_heavy_edges():
    rng = np.random.default_rng(1111062825)
    g = hub_graph(rng, 4000, 2, 3000, 3000)
    heavy = int(np.argmax(np.diff(g.row_ptr)))
    e = int(g.row_ptr[heavy]) + 2500          # an edge deep inside a heavy vertex
    col = g.col_idx.copy()
    col[e] = g.n + 5
    with pytest.raises(ocm.OCMError) as ex:
        ocm.solve(*_dev(g.row_ptr, col, g.w), g.mode)
    assert ex.value.status == -2
    w = g.w.copy()
    w[e] = np.iinfo(np.int32).min
    with pytest.raises(ocm.OCMError) as ex:
        ocm.solve(*_dev(g.row_ptr, g.col_idx, w), g.mode)
    assert ex.value.status == -4
    t = np.ones(g.m, np.int32)
    t[e] = 0
    rp, c2, w2, tt = _dev(g.row_ptr, g.col_idx, g.w, t)
    with pytest.raises(ocm.OCMError) as ex:
        ocm.solve(rp, c2, w2, g.mode, transit=tt)
    assert ex.value.status == -1
    init = g.row_ptr[:-1].copy()
    init[heavy] = g.row_ptr[heavy + 1]         # the next vertex's first edge
    with pytest.raises(ocm.OCMError) as ex:
        ocm.solve(rp, c2, w2, g.mode, init_policy=_dev(init)[0])
    assert ex.value.status == -1
    # the device stays usable
    _check(g, ocm.solve(rp, c2, w2, g.mode))


def test_heavy_graph_loop_equals_host_loop():
    from paper_1111_0627_gb300.ocm import OCM_FLAG_HOST_LOOP
    rng = np.random.default_rng(1111062826)
    g = hub_graph(rng, 20000, 5, 1500, 40000)
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    a = ocm.solve(rp, col, w, g.mode, certificate=True)
    b = ocm.solve(rp, col, w, g.mode, certificate=True, flags=OCM_FLAG_HOST_LOOP)
    assert a.stats["graph_loop"] == 1 and b.stats["graph_loop"] == 0
    for k in ("iterations", "cycles", "detect_rounds", "value_rounds", "switched", "detect_items",
              "value_items"):
        assert a.stats[k] == b.stats[k], k
    assert torch.equal(a.cycle, b.cycle) and torch.equal(a.potential, b.potential)
    assert torch.equal(a.policy, b.policy)
