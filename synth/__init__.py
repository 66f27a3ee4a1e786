"""Seeded synthetic inputs for the optimal-cycle-mean solver and its oracle.

This package only constructs graphs (CSR: ``row_ptr`` int32[n+1], ``col_idx``
int32[m], ``w`` int32[m]); it holds none of the cycle-mean arithmetic, so the
CPU oracle and the CUDA path can both be fed from it.  The large families are
generated by ``synth.c`` (counter-based SplitMix64 + Lemire bounded integers,
no floating point), so a seed gives the same bytes on every platform.

Workloads (the paper's DiVinE state spaces and its road/random/DIMACS graphs
are not available; these synthetic families stand in for them, Sec. 4):

========  ===============================================================
name      recipe
========  ===============================================================
ring10k   ring + U{0..4} extra uniform edges, n = 10,000, w in U[1,100], max
product4  4 processes x 38-state ring + 2 chords/state, BFS-numbered product
          state space (38^4 = 2,085,136 states), w in U[0,1000], max
locality  n = 2^25, out-degree 4/16/64 (p = .8/.1667/.0333, mean 8),
          targets i + 1 + floor|N(0, 4096)|, w in U[-1000,1000], min
batch     4096 graphs, n_g log-uniform in [100, 200000], ring + U{0..7}
          extras, w in U[1,10000], max
diff1m    n = 2^20, ring + U{0..7} extras, w = 1024 * U[0,1000], max
          (the critical cycle is made unique afterwards, see tests)
========  ===============================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 1111062700


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library (gcc, no OpenMP, no -march)."""
    src = os.path.join(_HERE, "synth.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-strict-aliasing",
                           "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64, i32 = ctypes.c_uint64, ctypes.c_int32
            lib.synth_ring_extra_degrees.argtypes = [u64, u64, i32, i32, i32, i32p]
            lib.synth_ring_extra_fill.argtypes = [u64, u64, i32, i32, i32, i32, i32, i32,
                                                  i32p, i32p, i32p]
            lib.synth_locality_degrees.argtypes = [u64, u64, i32, i32p]
            lib.synth_locality_fill.argtypes = [u64, u64, i32, i32, i32, i32, i32p, i32p, i32p]
            lib.synth_product_num_states.argtypes = [i32, i32]
            lib.synth_product_num_states.restype = ctypes.c_int64
            lib.synth_product_structure.argtypes = [u64, u64, i32, i32, i32, i32p, i32p]
            lib.synth_product_fill.argtypes = [u64, u64, i32, i32, i32, i32, i32, i32p, i32p,
                                               i32p, i32p]
            lib.synth_loguniform_sizes.argtypes = [u64, u64, i32, i32, i32, i32p]
            lib.synth_digest_i32.argtypes = [i32p, ctypes.c_int64]
            lib.synth_digest_i32.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"synth: {what} failed with code {rc}")


@dataclass
class Graph:
    """A CSR digraph with int32 weights and the optimisation sense."""
    row_ptr: np.ndarray
    col_idx: np.ndarray
    w: np.ndarray
    mode: str = "max"          # "max" or "min"
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col_idx.shape[0])


def _row_ptr_from_degrees(deg: np.ndarray) -> np.ndarray:
    rp = np.zeros(deg.shape[0] + 1, dtype=np.int64)
    np.cumsum(deg, out=rp[1:])
    if rp[-1] >= 2**31:
        raise ValueError("graph too large for int32 edge indices")
    return rp.astype(np.int32)


def ring_extra(n: int, xlo: int, xhi: int, wlo: int, whi: int, wscale: int = 1,
               seed: int = SEED_BASE, tag: int = 0, mode: str = "max", name: str = "") -> Graph:
    lib = _load()
    deg = np.empty(n, dtype=np.int32)
    _check(lib.synth_ring_extra_degrees(seed, tag, n, xlo, xhi, _p(deg)), "ring_extra degrees")
    rp = _row_ptr_from_degrees(deg)
    m = int(rp[-1])
    col = np.empty(m, dtype=np.int32)
    w = np.empty(m, dtype=np.int32)
    _check(lib.synth_ring_extra_fill(seed, tag, n, xlo, xhi, wlo, whi, wscale, _p(rp), _p(col),
                                     _p(w)), "ring_extra fill")
    return Graph(rp, col, w, mode, name or f"ring_extra(n={n})")


def locality(n: int = 1 << 25, sigma: int = 4096, wlo: int = -1000, whi: int = 1000,
             seed: int = SEED_BASE + 2, tag: int = 0, mode: str = "min", name: str = "") -> Graph:
    lib = _load()
    deg = np.empty(n, dtype=np.int32)
    _check(lib.synth_locality_degrees(seed, tag, n, _p(deg)), "locality degrees")
    rp = _row_ptr_from_degrees(deg)
    m = int(rp[-1])
    col = np.empty(m, dtype=np.int32)
    w = np.empty(m, dtype=np.int32)
    _check(lib.synth_locality_fill(seed, tag, n, sigma, wlo, whi, _p(rp), _p(col), _p(w)),
           "locality fill")
    return Graph(rp, col, w, mode, name or f"locality(n={n})")


def product(P: int = 4, S: int = 38, C: int = 2, wlo: int = 0, whi: int = 1000,
            seed: int = SEED_BASE + 1, tag: int = 0, mode: str = "max", name: str = "") -> Graph:
    lib = _load()
    N = int(lib.synth_product_num_states(P, S))
    if N < 0:
        raise ValueError("product state space out of range")
    deg = np.empty(N, dtype=np.int32)
    code = np.empty(N, dtype=np.int32)
    _check(lib.synth_product_structure(seed, tag, P, S, C, _p(deg), _p(code)), "product structure")
    rp = _row_ptr_from_degrees(deg)
    m = int(rp[-1])
    col = np.empty(m, dtype=np.int32)
    w = np.empty(m, dtype=np.int32)
    _check(lib.synth_product_fill(seed, tag, P, S, C, wlo, whi, _p(code), _p(rp), _p(col), _p(w)),
           "product fill")
    return Graph(rp, col, w, mode, name or f"product(P={P},S={S},C={C})")


def loguniform_sizes(G: int, nmin: int, nmax: int, seed: int, tag: int = 0) -> np.ndarray:
    lib = _load()
    out = np.empty(G, dtype=np.int32)
    _check(lib.synth_loguniform_sizes(seed, tag, G, nmin, nmax, _p(out)), "loguniform sizes")
    return out


@dataclass
class Batch:
    """G independent graphs as one disjoint-union CSR (global vertex ids)."""
    graph_vptr: np.ndarray    # int32[G+1] vertex offsets
    row_ptr: np.ndarray       # int32[N+1]
    col_idx: np.ndarray       # int32[M], global ids
    w: np.ndarray             # int32[M]
    mode: str = "max"
    name: str = ""

    @property
    def G(self) -> int:
        return int(self.graph_vptr.shape[0] - 1)

    @property
    def N(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def M(self) -> int:
        return int(self.col_idx.shape[0])

    def member(self, g: int) -> Graph:
        v0, v1 = int(self.graph_vptr[g]), int(self.graph_vptr[g + 1])
        e0, e1 = int(self.row_ptr[v0]), int(self.row_ptr[v1])
        return Graph((self.row_ptr[v0:v1 + 1] - e0).astype(np.int32),
                     (self.col_idx[e0:e1] - v0).astype(np.int32),
                     self.w[e0:e1].copy(), self.mode, f"{self.name}[{g}]")


def concat(graphs: list[Graph], name: str = "") -> Batch:
    """Disjoint union of graphs (all with the same mode)."""
    modes = {g.mode for g in graphs}
    if len(modes) != 1:
        raise ValueError("all batch members must share one mode")
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    ms = np.array([g.m for g in graphs], dtype=np.int64)
    if ns.sum() >= 2**31 or ms.sum() >= 2**31:
        raise ValueError("batch too large for int32 indices")
    vptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=vptr[1:])
    eptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ms, out=eptr[1:])
    rp = np.empty(int(vptr[-1]) + 1, dtype=np.int32)
    col = np.empty(int(eptr[-1]), dtype=np.int32)
    w = np.empty(int(eptr[-1]), dtype=np.int32)
    for i, g in enumerate(graphs):
        v0, e0 = int(vptr[i]), int(eptr[i])
        rp[v0:v0 + g.n] = g.row_ptr[:-1] + e0
        col[e0:e0 + g.m] = g.col_idx + v0
        w[e0:e0 + g.m] = g.w
    rp[-1] = int(eptr[-1])
    return Batch(vptr.astype(np.int32), rp, col, w, modes.pop(), name)


def batch_graphs(G: int = 4096, nmin: int = 100, nmax: int = 200000, xlo: int = 0, xhi: int = 7,
                 wlo: int = 1, whi: int = 10000, seed: int = SEED_BASE + 3) -> list[Graph]:
    sizes = loguniform_sizes(G, nmin, nmax, seed, tag=0)
    return [ring_extra(int(sizes[g]), xlo, xhi, wlo, whi, 1, seed=seed, tag=1000 + g,
                       mode="max", name=f"batch[{g}]") for g in range(G)]


# --------------------------------------------------------------------------
# The five workloads, by name.
# --------------------------------------------------------------------------

def ring10k() -> Graph:
    return ring_extra(10_000, 0, 4, 1, 100, 1, seed=SEED_BASE + 0, mode="max", name="ring10k")


def product4() -> Graph:
    return product(4, 38, 2, 0, 1000, seed=SEED_BASE + 1, mode="max", name="product4")


def locality32m(n: int = 1 << 25) -> Graph:
    return locality(n, 4096, -1000, 1000, seed=SEED_BASE + 2, mode="min",
                    name="locality32m" if n == 1 << 25 else f"locality(n={n})")


def batch4096(G: int = 4096, nmax: int = 200000) -> Batch:
    return concat(batch_graphs(G, 100, nmax), name=f"batch{G}")


def diff1m_base(n: int = 1 << 20) -> Graph:
    """Differentiation workload before its critical cycle is made unique."""
    return ring_extra(n, 0, 7, 0, 1000, 1024, seed=SEED_BASE + 4, mode="max",
                      name="diff1m" if n == 1 << 20 else f"diff(n={n})")


def hub4m(n: int = 1 << 20, hub_deg: int = 4_000_000, seed: int = SEED_BASE + 5) -> Graph:
    """A ring plus 3 uniform extra out-edges per vertex, and one vertex (chosen
    by the seed) with hub_deg more: the skewed-degree workload (numpy PCG64,
    the same bytes on every platform)."""
    rng = np.random.default_rng(seed)
    deg = np.full(n, 4, np.int64)
    hub = int(rng.integers(0, n))
    deg[hub] += hub_deg
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(deg, out=rp[1:])
    m = int(rp[-1])
    col = rng.integers(0, n, m).astype(np.int32)
    col[rp[:-1]] = (np.arange(n) + 1) % n
    w = rng.integers(-1000, 1001, m).astype(np.int32)
    return Graph(rp.astype(np.int32), col, w, "max", "hub4m" if (n, hub_deg) == (1 << 20, 4_000_000)
                 else f"hub(n={n},deg={hub_deg})")


def digest(a: np.ndarray) -> int:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return int(_load().synth_digest_i32(_p(a), a.shape[0]))


# --------------------------------------------------------------------------
# Small random graphs for exhaustive tests (numpy Generator, seeded).
# --------------------------------------------------------------------------

def tiny_random(rng: np.random.Generator, n: int, max_extra: int = 3, wlo: int = -9,
                whi: int = 9, ring: bool = False, mode: str = "max") -> Graph:
    """n vertices, every out-degree >= 1; self-loops and parallel edges allowed."""
    rows = []
    for v in range(n):
        k = int(rng.integers(1, max_extra + 1))
        tg = list(rng.integers(0, n, size=k))
        if ring:
            tg = [(v + 1) % n] + tg
        rows.append(tg)
    deg = np.array([len(r) for r in rows], dtype=np.int32)
    rp = _row_ptr_from_degrees(deg)
    col = np.array([t for r in rows for t in r], dtype=np.int32)
    w = rng.integers(wlo, whi + 1, size=col.shape[0]).astype(np.int32)
    return Graph(rp, col, w, mode, f"tiny(n={n})")


def from_edges(n: int, edges: list[tuple[int, int, int]], mode: str = "max", name: str = "") -> Graph:
    """CSR from (src, dst, w) triples; row order = order of appearance per source."""
    rows: list[list[tuple[int, int]]] = [[] for _ in range(n)]
    for s, t, wt in edges:
        rows[s].append((t, wt))
    deg = np.array([len(r) for r in rows], dtype=np.int32)
    rp = _row_ptr_from_degrees(deg)
    col = np.array([t for r in rows for (t, _) in r], dtype=np.int32)
    w = np.array([wt for r in rows for (_, wt) in r], dtype=np.int32)
    return Graph(rp, col, w, mode, name)


def random_policy(rng: np.random.Generator, row_ptr: np.ndarray) -> np.ndarray:
    """One uniformly drawn out-edge index per vertex (a start policy for warm
    starts): row_ptr[v] + U{0 .. deg(v)-1}."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    deg = rp[1:] - rp[:-1]
    return (rp[:-1] + rng.integers(0, 1 << 62, size=deg.shape[0]) % deg).astype(np.int32)


def random_digraph(rng: np.random.Generator, n: int, avg_deg: float, wlo: int = -50,
                   whi: int = 50, sink_frac: float = 0.1, mode: str = "max") -> Graph:
    """Sparse random digraph with vertices that have no out-edges (a fraction
    sink_frac of them) and, at low average degree, many strongly connected
    components: out-degree ~ Poisson(avg_deg) elsewhere, targets uniform,
    self-loops and parallel edges allowed."""
    deg = rng.poisson(avg_deg, size=n).astype(np.int64)
    deg[rng.random(n) < sink_frac] = 0
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rp[1:])
    m = int(rp[-1])
    col = rng.integers(0, n, size=m).astype(np.int32)
    w = rng.integers(wlo, whi + 1, size=m).astype(np.int32)
    return Graph(rp.astype(np.int32), col, w, mode, f"digraph(n={n})")
