"""SCC front-end (needs a GB300): the GPU decomposition gives every vertex
the smallest vertex of its strongly connected component, exactly as Tarjan's
algorithm in the oracle does, on graphs with vertices without out-edges and
many components; the per-component solve gives each component with a cycle
the oracle's value and critical cycle for its induced subgraph, and the best
component is the whole graph's optimum (Prop. 2.2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from golden_io import fig1
from scc_helpers import canonical_labels, components

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm


def _dev(*arrays):
    d = torch.device("cuda")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in arrays]


def _check_labels(g):
    rp, col = _dev(g.row_ptr, g.col_idx)
    labels, count = ocm.scc(rp, col)
    expect = canonical_labels(g.row_ptr, g.col_idx)
    assert labels.cpu().numpy().tolist() == expect.tolist(), g.name
    assert count == len(np.unique(expect))


def _check_solve(g):
    rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
    sol = ocm.solve_scc(rp, col, w, g.mode)
    expect = components(g)
    assert sol.labels.cpu().numpy().tolist() == canonical_labels(g.row_ptr, g.col_idx).tolist()
    assert len(expect) == sol.root.numel(), g.name
    roots = sol.root.cpu().tolist()
    nums, dens = sol.num.cpu().tolist(), sol.den.cpu().tolist()
    for c, (root, num, den, cyc) in enumerate(expect):
        assert roots[c] == root, (g.name, c)
        assert (nums[c], dens[c]) == (num, den), (g.name, c)
        assert sol.cycle(c).cpu().tolist() == cyc, (g.name, c)
    return sol


@pytest.mark.parametrize("mode", ["max", "min"])
def test_tiny_digraphs_labels_and_components(mode):
    rng = np.random.default_rng(1111062792 + (mode == "min"))
    for trial in range(120):
        n = int(rng.integers(1, 40))
        g = synth.random_digraph(rng, n, avg_deg=float(rng.uniform(0.3, 3.0)), sink_frac=0.15,
                                 mode=mode)
        _check_labels(g)
        _check_solve(g)


def test_fig1_components():
    f = fig1()
    _check_labels(f.graph_max)
    sol = _check_solve(f.graph_max)
    best = max(range(sol.root.numel()),
               key=lambda c: (int(sol.num[c]) / int(sol.den[c])))
    assert (int(sol.num[best]), int(sol.den[best])) == f.max_value


@pytest.mark.parametrize("avg_deg", [0.9, 1.3, 2.0])
def test_sparse_digraph_with_many_components(avg_deg):
    rng = np.random.default_rng(int(avg_deg * 100) + 1111062794)
    g = synth.random_digraph(rng, 30000, avg_deg=avg_deg, sink_frac=0.05)
    _check_labels(g)
    _check_solve(g)


def test_chain_of_rings_and_sinks():
    # 300 rings of random lengths joined one way, with tails into sink vertices
    rng = np.random.default_rng(1111062797)
    edges, v = [], 0
    starts = []
    for k in range(300):
        L = int(rng.integers(1, 40))
        starts.append(v)
        for i in range(L):
            edges.append((v + i, v + (i + 1) % L, int(rng.integers(-100, 100))))
        v += L
    for k in range(299):
        edges.append((starts[k], starts[k + 1], 5))
    n = v + 100
    for k in range(100):
        edges.append((int(rng.integers(0, v)), v + k, 1))   # into sinks
    g = synth.from_edges(n, edges)
    _check_labels(g)
    sol = _check_solve(g)
    assert sol.root.numel() == 300


def test_strongly_connected_workloads_have_one_component():
    for g in (synth.ring10k(), synth.locality32m(1 << 18)):
        rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
        labels, count = ocm.scc(rp, col)
        assert count == 1 and int(labels.max()) == 0
        whole = ocm.solve(rp, col, w, g.mode)
        sol = ocm.solve_scc(rp, col, w, g.mode)
        assert sol.root.tolist() == [0]
        assert (int(sol.num[0]), int(sol.den[0])) == (whole.num, whole.den)
        assert sol.cycle(0).cpu().tolist() == whole.cycle.cpu().tolist()


def test_best_component_is_the_whole_graph_optimum():
    rng = np.random.default_rng(1111062798)
    for trial in range(60):
        g = synth.tiny_random(rng, int(rng.integers(2, 60)), max_extra=2, wlo=-30, whi=30)
        rp, col, w = _dev(g.row_ptr, g.col_idx, g.w)
        whole = ocm.solve(rp, col, w, g.mode)
        sol = ocm.solve_scc(rp, col, w, g.mode)
        vals = [(int(a), int(b)) for a, b in zip(sol.num.cpu(), sol.den.cpu())]
        from fractions import Fraction
        assert max(Fraction(a, b) for a, b in vals) == whole.value, trial


def test_edge_cases():
    # no edges at all: n singleton components, none with a cycle
    d = torch.device("cuda")
    rp = torch.zeros(6, dtype=torch.int32, device=d)
    col = torch.zeros(0, dtype=torch.int32, device=d)
    labels, count = ocm.scc(rp, col)
    assert count == 5 and labels.cpu().tolist() == [0, 1, 2, 3, 4]
    sol = ocm.solve_scc(rp, col, torch.zeros(0, dtype=torch.int32, device=d))
    assert sol.root.numel() == 0
    # a lone self-loop is a component with a cycle
    g = synth.from_edges(3, [(0, 1, 4), (1, 1, -2)])
    sol = _check_solve(g)
    assert sol.root.tolist() == [1] and int(sol.num[0]) == -2
    # malformed CSR
    bad = torch.tensor([0, 2, 1], dtype=torch.int32, device=d)
    with pytest.raises(ocm.OCMError) as e:
        ocm.scc(bad, torch.zeros(1, dtype=torch.int32, device=d))
    assert e.value.status == -2


def test_hubs_with_sinks():
    """Vertices with thousands of out-edges (the transposed graph is built
    edge-parallel) next to vertices without out-edges."""
    rng = np.random.default_rng(1111062796)
    n = 20000
    deg = rng.poisson(1.2, size=n).astype(np.int64)
    deg[rng.random(n) < 0.1] = 0
    hubs = rng.choice(n, 6, replace=False)
    deg[hubs] = rng.integers(2000, 60000, size=6)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    col = rng.integers(0, n, int(rp[-1])).astype(np.int32)
    w = rng.integers(-50, 51, int(rp[-1])).astype(np.int32)
    g = synth.Graph(rp.astype(np.int32), col, w, "max", "hubs_with_sinks")
    _check_labels(g)
    _check_solve(g)
