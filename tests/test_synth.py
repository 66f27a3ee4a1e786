"""Generator checks (no GPU): determinism across machines (digests written by
tests/golden/make_synth_digests.py), and the structure each workload recipe
promises."""
import os

import numpy as np
import pytest

import synth
from golden_io import GOLDEN


def _digests():
    rows = {}
    with open(os.path.join(GOLDEN, "synth_digests.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows[t[0]] = tuple(int(x) for x in t[1:])
    return rows


_MAKERS = {
    "ring10k": lambda: synth.ring10k(),
    "product4": lambda: synth.product4(),
    "locality_2^20": lambda: synth.locality32m(1 << 20),
    "diff1m_base": lambda: synth.diff1m_base(),
    "batch64": lambda: synth.batch4096(G=64, nmax=5000),
}


@pytest.mark.parametrize("name", list(_MAKERS))
def test_generator_bytes_are_pinned(name):
    g = _MAKERS[name]()
    want = _digests()[name]
    got = (g.row_ptr.shape[0] - 1, g.col_idx.shape[0], synth.digest(g.row_ptr),
           synth.digest(g.col_idx), synth.digest(g.w))
    assert got == want


def test_batch_sizes_pinned_and_log_uniform():
    s = synth.loguniform_sizes(4096, 100, 200000, synth.SEED_BASE + 3)
    want = _digests()["batch_sizes_4096"]
    assert (s.shape[0], int(s.sum()), synth.digest(s)) == want[:3]
    assert s.min() >= 100 and s.max() <= 200000
    # log-uniform: log(n) roughly uniform over [log 100, log 200000]
    u = np.log(s / 100) / np.log(2000)
    hist = np.histogram(u, bins=10, range=(0, 1))[0]
    assert hist.min() > 330 and hist.max() < 490


def _check_csr(g):
    assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.m
    assert (np.diff(g.row_ptr) >= 1).all()
    assert g.col_idx.min() >= 0 and g.col_idx.max() < g.n


def test_ring10k_structure():
    g = synth.ring10k()
    _check_csr(g)
    assert g.n == 10_000 and g.mode == "max"
    deg = np.diff(g.row_ptr)
    assert deg.min() == 1 and deg.max() == 5
    assert (g.col_idx[g.row_ptr[:-1]] == (np.arange(g.n) + 1) % g.n).all()   # ring first
    assert g.w.min() >= 1 and g.w.max() <= 100


def test_product4_structure():
    g = synth.product4()
    _check_csr(g)
    assert g.n == 38 ** 4
    deg = np.diff(g.row_ptr)
    assert deg.min() >= 4 and deg.max() <= 12
    src = np.repeat(np.arange(g.n), deg)
    assert (g.col_idx != src).all()            # no self-loops
    key = src.astype(np.int64) * g.n + g.col_idx
    assert np.unique(key).shape[0] == g.m      # no parallel edges
    # BFS numbering from state 0: every vertex but 0 has a predecessor with a smaller id
    first_pred = np.full(g.n, g.n, dtype=np.int64)
    np.minimum.at(first_pred, g.col_idx, src)
    assert (first_pred[1:] < np.arange(1, g.n)).all()
    assert g.w.min() >= 0 and g.w.max() <= 1000


def test_locality_structure():
    g = synth.locality32m(1 << 18)
    _check_csr(g)
    deg = np.diff(g.row_ptr)
    assert set(np.unique(deg)) == {4, 16, 64}
    assert abs(deg.mean() - 8.0) < 0.1
    src = np.repeat(np.arange(g.n), deg)
    off = (g.col_idx.astype(np.int64) - src) % g.n
    assert off.min() >= 1 and (off[g.row_ptr[:-1]] == 1).all()
    extra = np.ones(g.m, bool)
    extra[g.row_ptr[:-1]] = False
    # 1 + floor|N(0, 4096)|: E|X| = 4096*sqrt(2/pi) ~ 3268
    assert abs(off[extra].mean() - 1 - 4096 * np.sqrt(2 / np.pi)) < 60
    assert g.w.min() >= -1000 and g.w.max() <= 1000 and g.mode == "min"


def test_batch_concat_roundtrip():
    graphs = synth.batch_graphs(G=8, nmin=100, nmax=400)
    b = synth.concat(graphs)
    for i, g in enumerate(graphs):
        h = b.member(i)
        assert (h.row_ptr == g.row_ptr).all() and (h.col_idx == g.col_idx).all()
        assert (h.w == g.w).all()
