"""CPU oracle for the optimal cycle mean -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA solver never imports, links
or calls it, and it shares no code with the solver: its C source
(``ocm_oracle.c``) is compiled here with gcc into its own library.

Every function works on a CSR graph (row_ptr, col_idx, w: int32 numpy arrays)
and returns exact integers.  See ``ocm_oracle.c`` for the paper passages each
routine follows:

* :func:`howard`      -- Howard policy iteration (Alg. 1, multichain reading),
                          the parity target for the CUDA path;
* :func:`karp`        -- Karp's recurrence, independent exact value;
* :func:`brute`       -- every simple cycle, tiny graphs only;
* :func:`tarjan_scc`  -- strongly connected components;
* :func:`certificate` -- LP-dual optimality check of an answer (Eq. 1,
                          Prop. 2.1);
* :func:`gradient`    -- d lambda*/dw = 1/|C*| on the critical cycle, else 0.

:func:`howard`, :func:`brute` and :func:`certificate` take an optional
``transit`` array (int32 transit times t(e) >= 1, Sec. 2.2): they then work on
the optimal cycle ratio w(C)/t(C); ``transit`` of all ones gives the mean.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libocm_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -1: "invalid argument", -2: "bad CSR", -3: "vertex without out-edge",
          -4: "weight out of range", -5: "not converged", -6: "out of memory",
          -7: "too many optimal cycles", -8: "not strongly connected"}

MAX, MIN = 0, 1


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "ocm_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(src)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, src])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32, i64, c_int = ctypes.c_int32, ctypes.c_int64, ctypes.c_int
            lib.oracle_howard.argtypes = [i32, i32, i32p, i32p, i32p, c_int, i64, i64p, i64p,
                                          i32p, i32p, i64p, i64p, i64p, i32p, i64p, i64p, i64,
                                          i32p]
            lib.oracle_karp.argtypes = [i32, i32, i32p, i32p, i32p, c_int, i64p, i64p]
            lib.oracle_brute.argtypes = [i32, i32, i32p, i32p, i32p, c_int, i64p, i64p, i64p,
                                         i32p, i64, i64p, i64, i64p]
            lib.oracle_tarjan_scc.argtypes = [i32, i32p, i32p, i32p]
            lib.oracle_tarjan_scc.restype = i32
            lib.oracle_certificate.argtypes = [i32, i32, i32p, i32p, i32p, c_int, i64p, i64p,
                                               i64p, i64, i64, i32p, i32, i64p]
            lib.oracle_howard_single.argtypes = [i32, i32, i32p, i32p, i32p, i32p, c_int, i64,
                                                 i64p, i64p, i32p, i32p, i64p, i32p, i64p, i32p]
            lib.oracle_howard_ratio.argtypes = [i32, i32, i32p, i32p, i32p, i32p, c_int, i64,
                                                i64p, i64p, i32p, i32p, i64p, i64p, i64p, i32p,
                                                i64p, i32p]
            lib.oracle_brute_ratio.argtypes = [i32, i32, i32p, i32p, i32p, i32p, c_int, i64p,
                                               i64p, i64p, i32p, i64, i64p, i64, i64p]
            lib.oracle_certificate_ratio.argtypes = [i32, i32, i32p, i32p, i32p, i32p, c_int,
                                                     i64p, i64p, i64p, i64, i64, i32p, i32, i64p]
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _mode(mode) -> int:
    if mode in (0, "max"):
        return MAX
    if mode in (1, "min"):
        return MIN
    raise ValueError(f"mode must be 'max' or 'min', got {mode!r}")


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {STATUS.get(code, code)} ({code})")
        self.code = code


@dataclass
class HowardResult:
    num: int
    den: int
    cycle: np.ndarray        # critical cycle, CSR edge indices
    eta_p: np.ndarray        # per-vertex mean numerator (max sense)
    eta_q: np.ndarray        # per-vertex mean denominator
    V: np.ndarray            # per-vertex value, scaled by eta_q (max sense)
    policy: np.ndarray       # final policy edge per vertex
    iterations: int
    trace: np.ndarray        # per iteration: (#cycles, #switched, iteration)

    @property
    def value(self) -> Fraction:
        return Fraction(self.num, self.den)


def howard(row_ptr, col_idx, w, mode="max", max_iter: int = 0, trace_cap: int = 4096,
           init_policy=None, transit=None) -> HowardResult:
    """Howard policy iteration; ``init_policy`` (an out-edge index per vertex)
    replaces the initial policy of Alg. 1's first pass (warm start);
    ``transit`` switches to the optimal cycle ratio (no trace is kept then)."""
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    ww, wp = _i32(w)
    n, m = rp.shape[0] - 1, col.shape[0]
    num = np.zeros(1, np.int64)
    den = np.zeros(1, np.int64)
    cyc = np.zeros(max(n, 1), np.int32)
    clen = np.zeros(1, np.int32)
    ep = np.zeros(n, np.int64)
    eq = np.zeros(n, np.int64)
    V = np.zeros(n, np.int64)
    pol = np.zeros(n, np.int32)
    its = np.zeros(1, np.int64)
    tr = np.zeros(3 * trace_cap, np.int64)
    init, initp = _i32(init_policy) if init_policy is not None else (None, None)
    if init is not None and init.shape[0] != n:
        raise ValueError("init_policy must have one entry per vertex")
    if transit is not None:
        tt, ttp = _i32(transit)
        if tt.shape[0] != m:
            raise ValueError("transit needs one entry per edge")
        rc = lib.oracle_howard_ratio(n, m, rpp, colp, wp, ttp, _mode(mode), max_iter,
                                     _i64p(num), _i64p(den),
                                     cyc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     clen.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     _i64p(ep), _i64p(eq), _i64p(V),
                                     pol.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     _i64p(its), initp)
    else:
        rc = lib.oracle_howard(n, m, rpp, colp, wp, _mode(mode), max_iter, _i64p(num), _i64p(den),
                               cyc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               clen.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               _i64p(ep), _i64p(eq), _i64p(V),
                               pol.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _i64p(its),
                               _i64p(tr), trace_cap, initp)
    if rc != 0:
        raise OracleError(rc, "howard")
    it = int(its[0])
    ntr = min(it + 1, trace_cap)
    return HowardResult(int(num[0]), int(den[0]), cyc[:int(clen[0])].copy(), ep, eq, V, pol, it,
                        tr[:3 * ntr].reshape(ntr, 3))


@dataclass
class SingleResult:
    num: int
    den: int
    cycle: np.ndarray
    V: np.ndarray
    policy: np.ndarray
    iterations: int

    @property
    def value(self) -> Fraction:
        return Fraction(self.num, self.den)


def howard_single(row_ptr, col_idx, w, mode="max", max_iter: int = 0,
                  transit=None, init_policy=None) -> SingleResult:
    """The paper's form of Howard's iteration (Alg. 1 as written): one lambda,
    every other policy cycle broken each iteration by a backward search from
    the chosen cycle's component; every vertex must reach that cycle.
    ``init_policy`` replaces the first pass (warm start)."""
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    ww, wp = _i32(w)
    n, m = rp.shape[0] - 1, col.shape[0]
    num = np.zeros(1, np.int64)
    den = np.zeros(1, np.int64)
    cyc = np.zeros(max(n, 1), np.int32)
    clen = np.zeros(1, np.int32)
    V = np.zeros(n, np.int64)
    pol = np.zeros(n, np.int32)
    its = np.zeros(1, np.int64)
    ttp = None
    if transit is not None:
        tt, ttp = _i32(transit)
        if tt.shape[0] != m:
            raise ValueError("transit needs one entry per edge")
    init, initp = _i32(init_policy) if init_policy is not None else (None, None)
    if init is not None and init.shape[0] != n:
        raise ValueError("init_policy must have one entry per vertex")
    i32p = ctypes.POINTER(ctypes.c_int32)
    rc = lib.oracle_howard_single(n, m, rpp, colp, wp, ttp, _mode(mode), max_iter, _i64p(num),
                                  _i64p(den), cyc.ctypes.data_as(i32p),
                                  clen.ctypes.data_as(i32p), _i64p(V), pol.ctypes.data_as(i32p),
                                  _i64p(its), initp)
    if rc != 0:
        raise OracleError(rc, "howard_single")
    return SingleResult(int(num[0]), int(den[0]), cyc[:int(clen[0])].copy(), V, pol,
                        int(its[0]))


def karp(row_ptr, col_idx, w, mode="max") -> Fraction:
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    ww, wp = _i32(w)
    num = np.zeros(1, np.int64)
    den = np.zeros(1, np.int64)
    rc = lib.oracle_karp(rp.shape[0] - 1, col.shape[0], rpp, colp, wp, _mode(mode), _i64p(num),
                         _i64p(den))
    if rc != 0:
        raise OracleError(rc, "karp")
    return Fraction(int(num[0]), int(den[0]))


@dataclass
class BruteResult:
    value: Fraction
    ncycles: int
    optimal: list            # each optimal cycle as a tuple of edge indices, from its min vertex


def brute(row_ptr, col_idx, w, mode="max", cap: int = 100000, transit=None) -> BruteResult:
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    ww, wp = _i32(w)
    n = rp.shape[0] - 1
    num = np.zeros(1, np.int64)
    den = np.zeros(1, np.int64)
    nc = np.zeros(1, np.int64)
    nopt = np.zeros(1, np.int64)
    edges = np.zeros(cap * min(n, 16), np.int32)
    ptr = np.zeros(cap + 1, np.int64)
    if transit is not None:
        tt, ttp = _i32(transit)
        rc = lib.oracle_brute_ratio(n, col.shape[0], rpp, colp, wp, ttp, _mode(mode), _i64p(num),
                                    _i64p(den), _i64p(nc),
                                    edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    edges.shape[0], _i64p(ptr), cap, _i64p(nopt))
    else:
        rc = lib.oracle_brute(n, col.shape[0], rpp, colp, wp, _mode(mode), _i64p(num),
                              _i64p(den), _i64p(nc),
                              edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              edges.shape[0], _i64p(ptr), cap, _i64p(nopt))
    if rc != 0:
        raise OracleError(rc, "brute")
    k = int(nopt[0])
    opt = [tuple(int(x) for x in edges[ptr[i]:ptr[i + 1]]) for i in range(k)]
    return BruteResult(Fraction(int(num[0]), int(den[0])), int(nc[0]), opt)


def tarjan_scc(row_ptr, col_idx) -> tuple[int, np.ndarray]:
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    n = rp.shape[0] - 1
    comp = np.zeros(n, np.int32)
    k = lib.oracle_tarjan_scc(n, rpp, colp, comp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if k < 0:
        raise OracleError(k, "tarjan")
    return int(k), comp


def certificate(row_ptr, col_idx, w, mode, eta_p, eta_q, V, num: int, den: int, cycle,
                transit=None) -> tuple[int, int]:
    """0 if (eta, V, num/den, cycle) proves optimality, else a failure code (1-6) and index."""
    lib = _load()
    rp, rpp = _i32(row_ptr)
    col, colp = _i32(col_idx)
    ww, wp = _i32(w)
    ep = np.ascontiguousarray(eta_p, dtype=np.int64)
    eq = np.ascontiguousarray(eta_q, dtype=np.int64)
    vv = np.ascontiguousarray(V, dtype=np.int64)
    cy, cyp = _i32(cycle if len(cycle) else np.zeros(1, np.int32))
    bad = np.zeros(1, np.int64)
    if transit is not None:
        tt, ttp = _i32(transit)
        rc = lib.oracle_certificate_ratio(rp.shape[0] - 1, col.shape[0], rpp, colp, wp, ttp,
                                          _mode(mode), _i64p(ep), _i64p(eq), _i64p(vv), int(num),
                                          int(den), cyp, len(cycle), _i64p(bad))
    else:
        rc = lib.oracle_certificate(rp.shape[0] - 1, col.shape[0], rpp, colp, wp, _mode(mode),
                                    _i64p(ep), _i64p(eq), _i64p(vv), int(num), int(den), cyp,
                                    len(cycle), _i64p(bad))
    return int(rc), int(bad[0])


def gradient_ratio(m: int, cycle, transit) -> np.ndarray:
    """d lambda*/dw for the optimal cycle ratio: lambda* = w(C*)/t(C*) is linear
    in the weights of C* with slope 1/t(C*), so each critical-cycle edge gets
    1/t(C*) and every other edge 0."""
    g = np.zeros(m, np.float64)
    cyc = np.asarray(cycle, dtype=np.int64)
    g[cyc] += 1.0 / float(np.asarray(transit, dtype=np.int64)[cyc].sum())
    return g


def gradient(m: int, cycle) -> np.ndarray:
    """d lambda*/dw in float64: 1/|C*| on each critical-cycle edge, 0 elsewhere.

    lambda* = w(C*)/|C*| is linear in the weights of C* while C* stays optimal,
    so each of its edges has partial derivative 1/|C*| (the same in min mode)."""
    g = np.zeros(m, np.float64)
    cyc = np.asarray(cycle, dtype=np.int64)
    g[cyc] += 1.0 / len(cyc)
    return g
