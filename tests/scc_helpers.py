"""Per-component answers from the CPU oracle, for the SCC tests (no solver
arithmetic here beyond calling the oracle): Tarjan's components labelled by
their smallest vertex, and for every component that holds a cycle the
oracle's Howard iteration on its induced subgraph, with the component's
vertices in increasing order and each row's edges in CSR order."""
from __future__ import annotations

import numpy as np

import oracle
import synth


def canonical_labels(row_ptr, col_idx) -> np.ndarray:
    """Tarjan's components, each labelled by its smallest vertex."""
    _, comp = oracle.tarjan_scc(row_ptr, col_idx)
    n = comp.shape[0]
    smallest = np.full(int(comp.max()) + 1 if n else 0, np.iinfo(np.int32).max, np.int64)
    np.minimum.at(smallest, comp, np.arange(n))
    return smallest[comp].astype(np.int32)


def components(g: synth.Graph, transit=None):
    """[(root, num, den, cycle as original edge indices)] for every component
    with a cycle, in increasing order of root."""
    labels = canonical_labels(g.row_ptr, g.col_idx)
    out = []
    for root in np.unique(labels):
        verts = np.nonzero(labels == root)[0]
        local = {int(v): i for i, v in enumerate(verts)}
        rows, edges = [], []
        for v in verts:
            keep = [e for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1]))
                    if labels[g.col_idx[e]] == root]
            rows.append(len(keep))
            edges.extend(keep)
        if not edges:
            continue                      # a single vertex without a self-loop
        rp = np.zeros(len(verts) + 1, np.int32)
        np.cumsum(rows, out=rp[1:])
        emap = np.array(edges, np.int64)
        col = np.array([local[int(g.col_idx[e])] for e in emap], np.int32)
        w = g.w[emap].astype(np.int32)
        h = oracle.howard(rp, col, w, g.mode)
        out.append((int(root), h.num, h.den, [int(emap[e]) for e in h.cycle]))
    return out
