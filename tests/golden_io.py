"""Readers for the text fixtures under tests/golden/ (no solver arithmetic)."""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class ClosedForm:
    name: str
    graph: synth.Graph
    num: int
    den: int
    cycle: tuple | None


def closed_forms() -> list[ClosedForm]:
    out: list[ClosedForm] = []
    cur = None
    edges: list[tuple[int, int, int]] = []

    def flush():
        if cur is not None:
            name, n, mode, num, den, cyc = cur
            out.append(ClosedForm(name, synth.from_edges(n, edges, mode, name), num, den, cyc))

    with open(os.path.join(GOLDEN, "closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                flush()
                cyc = None if tok[6] == "-" else tuple(int(x) for x in tok[6:])
                cur = (tok[1], int(tok[2]), tok[3], int(tok[4]), int(tok[5]), cyc)
                edges = []
            else:
                edges.append((int(tok[0]), int(tok[1]), int(tok[2])))
    flush()
    return out


@dataclass
class RatioForm:
    name: str
    graph: synth.Graph
    transit: np.ndarray
    num: int
    den: int
    cycle: tuple


def ratio_closed_forms() -> list[RatioForm]:
    out: list[RatioForm] = []
    cur = None
    edges: list[tuple[int, int, int]] = []
    times: list[int] = []

    def flush():
        if cur is not None:
            name, n, mode, num, den, cyc = cur
            g = synth.from_edges(n, edges, mode, name)
            # from_edges keeps the order of appearance per source, and the
            # fixture lists edges in CSR order, so times line up with edges
            out.append(RatioForm(name, g, np.array(times, np.int32), num, den, cyc))

    with open(os.path.join(GOLDEN, "ratio_closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                flush()
                cur = (tok[1], int(tok[2]), tok[3], int(tok[4]), int(tok[5]),
                       tuple(int(x) for x in tok[6:]))
                edges, times = [], []
            else:
                edges.append((int(tok[0]), int(tok[1]), int(tok[2])))
                times.append(int(tok[3]))
    flush()
    return out


@dataclass
class Fig1:
    graph_max: synth.Graph
    graph_min: synth.Graph
    names: list
    sccs: list
    max_value: tuple
    max_cycle: tuple
    min_value: tuple
    min_cycle: tuple


def fig1() -> Fig1:
    names: list[str] = []
    sccs: list[set] = []
    edges: list[tuple[int, int, int]] = []
    res = {}
    with open(os.path.join(GOLDEN, "fig1_scc.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "vertices":
                names = tok[1:]
            elif tok[0] == "scc":
                sccs = [set(s.strip("{}").split(",")) for s in tok[1:]]
            elif tok[0] == "edge":
                edges.append((names.index(tok[1]), names.index(tok[2]), int(tok[3])))
            elif tok[0] in ("max", "min"):
                res[tok[0]] = ((int(tok[1]), int(tok[2])), [t.split("->") for t in tok[3:]])
    n = len(names)
    gmax = synth.from_edges(n, edges, "max", "fig1")
    gmin = synth.from_edges(n, edges, "min", "fig1")

    def to_edges(g, pairs):
        ids = []
        for s, t in pairs:
            si, ti = names.index(s), names.index(t)
            cand = [e for e in range(g.row_ptr[si], g.row_ptr[si + 1]) if g.col_idx[e] == ti]
            assert len(cand) == 1
            ids.append(int(cand[0]))
        return tuple(ids)

    return Fig1(gmax, gmin, names, sccs, res["max"][0], to_edges(gmax, res["max"][1]),
                res["min"][0], to_edges(gmax, res["min"][1]))


def read_kv(path: str) -> dict:
    """'key value...' lines, '#' comments; values kept as strings."""
    d = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, _, v = line.partition(" ")
            d[k] = v.strip()
    return d


def relabel(g: synth.Graph, perm: np.ndarray) -> synth.Graph:
    """Graph with vertex v renamed perm[v]; each row keeps its edge order."""
    n = g.n
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    edges = []
    for new_v in range(n):
        old_v = int(inv[new_v])
        for e in range(g.row_ptr[old_v], g.row_ptr[old_v + 1]):
            edges.append((new_v, int(perm[g.col_idx[e]]), int(g.w[e])))
    return synth.from_edges(n, edges, g.mode, g.name + "-relabelled")


@dataclass
class SingleTrace:
    name: str
    graph: synth.Graph
    num: int
    den: int
    single_iters: int
    multichain_iters: int
    cycle: tuple
    policy: np.ndarray
    values: np.ndarray


def single_lambda_traces() -> list[SingleTrace]:
    out: list[SingleTrace] = []
    cur = None
    edges: list[tuple[int, int, int]] = []

    def flush():
        if cur is not None:
            name, n, mode, num, den, si, mi, cyc, pol, val = cur
            out.append(SingleTrace(name, synth.from_edges(n, edges, mode, name), num, den, si, mi,
                                   cyc, np.array(pol, np.int32), np.array(val, np.int64)))

    with open(os.path.join(GOLDEN, "single_lambda_traces.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                flush()
                cur = [tok[1], int(tok[2]), tok[3], int(tok[4]), int(tok[5]), int(tok[6]),
                       int(tok[7]), tuple(int(x) for x in tok[8:]), None, None]
                edges = []
            elif tok[0] == "policy":
                cur[8] = [int(x) for x in tok[1:]]
            elif tok[0] == "values":
                cur[9] = [int(x) for x in tok[1:]]
            else:
                edges.append((int(tok[0]), int(tok[1]), int(tok[2])))
    flush()
    return out
