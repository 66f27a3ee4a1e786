"""The chunked local phase of the two-level evaluation (needs a GB300): each
block takes its vertex range in chunks of 4,096 vertices from the top down,
a vertex whose successor lies in a chunk done before starting from that
vertex's state, the paths inside a chunk resolved by jumping in shared memory
and the paths that go back to a lower chunk finished by jumping over the
range at the end.  Forced on and off, on graphs whose edges go forward (no
path goes back), on the same graphs with the vertex order reversed (every
path goes back: the last step does all the work), with many short cycles and
self-loops inside chunks (the two-pass phase takes over), with ranges of
several chunks, and by default (on until a range leaves more than an eighth
of its vertices pending): every solve must equal the oracle, and the other
local form and the one-level evaluation bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import (OCM_FLAG_EVAL_GLOBAL, OCM_FLAG_EVAL_LOCAL,
                                           OCM_FLAG_HOST_LOOP, OCM_FLAG_TEST_LOCAL_CHUNKS,
                                           OCM_FLAG_TEST_NO_LOCAL_CHUNKS)

FORMS = ("chunks", "no_chunks", "default")


def _flags(form):
    return OCM_FLAG_EVAL_LOCAL | {"chunks": OCM_FLAG_TEST_LOCAL_CHUNKS,
                                  "no_chunks": OCM_FLAG_TEST_NO_LOCAL_CHUNKS,
                                  "default": 0}[form]


def _reversed(g):
    """g with vertex v renamed n-1-v (rows in the new order, edges in their
    old order within a row): forward edges become backward ones."""
    n = g.row_ptr.size - 1
    deg = np.diff(g.row_ptr.astype(np.int64))
    order = np.arange(n - 1, -1, -1)
    nd = deg[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nd, out=rp[1:])
    idx = np.repeat(g.row_ptr[order].astype(np.int64) - rp[:-1], nd) + np.arange(rp[-1])
    col = (n - 1 - g.col_idx[idx]).astype(np.int32)
    return synth.Graph(rp.astype(np.int32), col, g.w[idx].copy(), g.mode,
                       g.name + " reversed")


def _dev(g):
    d = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(d), torch.from_numpy(g.col_idx).to(d),
            torch.from_numpy(g.w).to(d))


def _check_oracle(g, flags, h):
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode, flags=flags, certificate=True)
    assert (s.num, s.den) == (h.num, h.den), g.name
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle], g.name
    assert s.stats["iterations"] == h.iterations, g.name
    assert (s.eta_num.cpu().numpy() == h.eta_p).all(), g.name
    assert (s.eta_den.cpu().numpy() == h.eta_q).all(), g.name
    assert (s.potential.cpu().numpy() == h.V).all(), g.name
    return s


def _same(a, b, name):
    assert (a.num, a.den) == (b.num, b.den), name
    assert torch.equal(a.cycle, b.cycle), name
    assert torch.equal(a.policy, b.policy) and torch.equal(a.potential, b.potential), name
    assert a.stats["iterations"] == b.stats["iterations"], name


@pytest.mark.parametrize("mode", ["max", "min"])
def test_chunks_against_the_oracle_on_small_graphs(mode):
    """Ranges of a few hundred to a few thousand vertices (one chunk each)."""
    rng = np.random.default_rng(1111063200 + (mode == "min"))
    cases = []
    for trial in range(3):
        n = int(rng.integers(3000, 50000))
        loc = synth.locality(n, int(rng.integers(2, 600)), -1000, 1000,
                             seed=1111063210 + trial, mode=mode)
        cases += [loc, _reversed(loc)]
    cases.append(synth.tiny_random(rng, 30000, max_extra=3, wlo=-9, whi=9, mode=mode))
    cases.append(synth.ring_extra(20000, 0, 4, -50, 50, 1, seed=1111063219, mode=mode))
    for g in cases:
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        for form in FORMS:
            _check_oracle(g, _flags(form), h)


def test_chunks_on_tiny_graphs():
    """Self-loops and cycles of every length inside one chunk."""
    rng = np.random.default_rng(1111063230)
    for trial in range(80):
        n = int(rng.integers(1, 300))
        mode = "max" if trial % 2 else "min"
        g = synth.tiny_random(rng, n, max_extra=3, wlo=-20, whi=20, ring=bool(trial % 3 == 0),
                              mode=mode)
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        for form in ("chunks", "no_chunks"):
            _check_oracle(g, _flags(form), h)


@pytest.mark.parametrize("reverse", [False, True])
def test_chunks_with_ranges_of_several_chunks(reverse):
    """n = 2^20: ranges of about 6,900 vertices (two chunks), forward edges or
    (reversed) every path going back; equal to the one-level evaluation bit
    for bit in both loop forms, and certified by the oracle."""
    g = synth.locality32m(1 << 20)
    if reverse:
        g = _reversed(g)
    rp, col, w = _dev(g)
    ref = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_GLOBAL, certificate=True)
    for flags in (_flags("chunks"), _flags("default"), _flags("chunks") | OCM_FLAG_HOST_LOOP):
        s = ocm.solve(rp, col, w, g.mode, flags=flags, certificate=True)
        _same(s, ref, g.name)
    rc, bad = oracle.certificate(g.row_ptr, g.col_idx, g.w, g.mode, s.eta_num.cpu().numpy(),
                                 s.eta_den.cpu().numpy(), s.potential.cpu().numpy(),
                                 s.num, s.den, s.cycle.cpu().numpy())
    assert rc == 0, bad


def test_chunks_with_cycles_inside_large_ranges():
    """Short cycles and self-loops in ranges of several chunks: a chunk finds a
    cycle, the two-pass phase takes the range over."""
    rng = np.random.default_rng(1111063240)
    n = 1 << 20
    src = np.repeat(np.arange(n, dtype=np.int64), 2)
    col = ((src + rng.integers(-6, 7, 2 * n)) % n).astype(np.int32)   # self-loops included
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    g = synth.Graph(rp, col, rng.integers(-9, 10, 2 * n).astype(np.int32), "max",
                    "short cycles 2^20")
    rp, col, w = _dev(g)
    ref = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_GLOBAL, certificate=True)
    for form in FORMS:
        s = ocm.solve(rp, col, w, g.mode, flags=_flags(form), certificate=True)
        _same(s, ref, (g.name, form))


def test_default_chunks_on_the_2p20_locality_graph():
    """The stored oracle answer (value, cycle, iterations) by default."""
    from test_gpu_parity import golden_values
    kv = golden_values()["locality_2^20"]
    g = synth.locality32m(1 << 20)
    rp, col, w = _dev(g)
    s = ocm.solve(rp, col, w, g.mode)
    assert (s.num, s.den) == (int(kv["num"]), int(kv["den"]))
    assert synth.digest(s.cycle.cpu().numpy().astype(np.int32)) == int(kv["cycle_digest"])
    assert s.stats["iterations"] == int(kv["iters"])
