"""The extraction's segment walk (needs a GB300).  After the two-level
evaluation the critical cycle is walked from its root exit by exit, each
segment inside a block range by its own thread; with more than 1,024 segments
or a segment of more than 4,096 vertices it gives up and the binary lifting
over the candidates runs instead.  Cycles on each side of both limits, forced
through the two-level evaluation: the cycle (edge list from the root), the
value and the iteration count must equal the oracle's, and the one-level
evaluation's bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1111_0627_gb300 as ocm
    from paper_1111_0627_gb300.ocm import OCM_FLAG_EVAL_GLOBAL, OCM_FLAG_EVAL_LOCAL


def _permutation_graph(n, step, extra, seed, mode):
    """Vertex i -> (i + step) mod n, plus `extra` random out-edges per vertex
    that are much worse (so the permutation's cycles are the optimum)."""
    rng = np.random.default_rng(seed)
    deg = 1 + extra
    col = np.empty(n * deg, dtype=np.int64)
    col[0::deg] = (np.arange(n) + step) % n
    w = np.empty(n * deg, dtype=np.int64)
    w[0::deg] = rng.integers(0, 10, n)
    for j in range(1, deg):
        col[j::deg] = rng.integers(0, n, n)
        w[j::deg] = -1000 if mode == "max" else 1000
    rp = np.arange(0, n * deg + 1, deg, dtype=np.int32)
    return synth.Graph(rp, col.astype(np.int32), w.astype(np.int32), mode,
                       f"perm(n={n}, step={step})")


def _check(g):
    h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
    d = torch.device("cuda")
    rp, col, w = (torch.from_numpy(x).to(d) for x in (g.row_ptr, g.col_idx, g.w))
    s = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_LOCAL)
    ref = ocm.solve(rp, col, w, g.mode, flags=OCM_FLAG_EVAL_GLOBAL)
    assert (s.num, s.den) == (h.num, h.den), g.name
    assert s.cycle.cpu().tolist() == [int(x) for x in h.cycle], g.name
    assert s.stats["iterations"] == h.iterations, g.name
    assert torch.equal(s.cycle, ref.cycle), g.name
    return s


@pytest.mark.parametrize("mode", ["max", "min"])
def test_walk_with_many_segments(mode):
    # ranges of about 1,000 vertices; every step of a cycle changes range:
    # six cycles of 500 segments (walked), one of 4,001 (more than 1,024:
    # lifting)
    _check(_permutation_graph(3000, 1002, 2, 1111063401, mode))
    _check(_permutation_graph(4001, 2001, 2, 1111063402, mode))


@pytest.mark.parametrize("mode", ["max", "min"])
def test_walk_with_long_segments(mode):
    # a ring through 2^20 vertices as the only cycle (ranges of about 6,900:
    # segments longer than 4,096, lifting), one through 2^19 (about 3,450:
    # walked), and a ring with worse shortcuts (Howard iterates to a cycle of
    # tens of thousands of vertices, walked)
    _check(_permutation_graph(1 << 20, 1, 0, 1111063403, mode))
    _check(_permutation_graph(1 << 19, 1, 0, 1111063404, mode))
    _check(_permutation_graph(1 << 19, 1, 1, 1111063407, mode))


def test_walk_on_locality_graphs():
    # forward locality (segments of a few dozen vertices, one per range) and
    # short cycles inside ranges (one segment back to the root)
    _check(synth.locality(300000, 4096, -1000, 1000, seed=1111063405, mode="min"))
    rng = np.random.default_rng(1111063406)
    _check(synth.tiny_random(rng, 20000, max_extra=3, wlo=-9, whi=9, mode="max"))
