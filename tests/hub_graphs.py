"""Graphs built so that heavy vertices meet the single-lambda rebuild in a
chosen way, with the rebuild's outcome known in closed form.

Both have one best cycle, a ring of weight-100 edges (lambda* = 100), reached
from everything else only through a chain c_1..c_L of one-vertex levels
(c_i -> c_{i-1}, weight 0; c_0 is ring vertex 0).  Every other vertex starts
on a worse cycle S (a self-loop of weight 10) and reaches the chain only
through chosen edges.  The first rebuild re-points each vertex to its
smallest-index edge into the levels below it, after which no edge improves,
so the final policy and potentials are those of the rebuild:
V(v) = w(pi(v)) + V(succ(v)) - 100, V(ring) = 0 (the ring's root is vertex 0).
"""
import numpy as np

import synth


def chain_hub_graph(L, hub_deg, hits):
    """A 5-ring, the chain, S leaving through c_L (weight -100), and two heavy
    vertices h1, h2 whose first edge goes to S (weight 60) and whose other
    hub_deg edges go to S (weight 0) except at positions `hits` (shifted by
    333 for h2), which go to c_L.  S, h1 and h2 form rebuild level L + 1, a
    level of three reached through the frontier lists."""
    c = lambda i: 0 if i == 0 else 4 + i
    S = 5 + L
    rows = [[((i + 1) % 5, 100)] for i in range(5)]
    rows += [[(S, 50), (c(i - 1), 0)] for i in range(1, L + 1)]
    rows.append([(S, 10), (c(L), -100)])
    for shift in (0, 333):
        row = [(S, 60)] + [(S, 0)] * hub_deg
        for p in hits:
            row[1 + (p + shift) % hub_deg] = (c(L), 0)
        rows.append(row)
    edges = [(v, t, wt) for v, row in enumerate(rows) for t, wt in row]
    return synth.from_edges(len(rows), edges, name=f"chain_hub({L},{hub_deg})")


def chain_hub_expected(g, L, hub_deg, hits):
    """(policy, V) after the solve, in closed form."""
    rp = g.row_ptr
    S = 5 + L
    pi = np.zeros(g.n, np.int64)
    V = np.zeros(g.n, np.int64)
    pi[:5] = rp[:5]
    for i in range(1, L + 1):
        pi[4 + i] = rp[4 + i] + 1
        V[4 + i] = -100 * i
    pi[S] = rp[S] + 1
    V[S] = -100 * (L + 2)
    for k, shift in enumerate((0, 333)):
        h = S + 1 + k
        pi[h] = rp[h] + 1 + min((p + shift) % hub_deg for p in hits)
        V[h] = -100 * (L + 1)
    return pi, V


def in_hub_graph(ring, chain, leaves):
    """A ring of `ring` vertices, the chain (chain = 0: none, c_0 = vertex 0),
    S leaving through c_chain (weight -100), and `leaves` vertices whose first
    edge goes to S (weight 60) and whose second goes to c_chain (weight 0):
    c_chain then has leaves + 1 (+1 for the ring's closing edge when
    chain = 0) in-edges and pushes over all of them at once."""
    c = lambda i: 0 if i == 0 else ring - 1 + i
    S = ring + chain
    rows = [[((i + 1) % ring, 100)] for i in range(ring)]
    rows += [[(S, 50), (c(i - 1), 0)] for i in range(1, chain + 1)]
    rows.append([(S, 10), (c(chain), -100)])
    rows += [[(S, 60), (c(chain), 0)] for _ in range(leaves)]
    edges = [(v, t, wt) for v, row in enumerate(rows) for t, wt in row]
    return synth.from_edges(len(rows), edges, name=f"in_hub({ring},{chain},{leaves})")


def in_hub_expected(g, ring, chain, leaves):
    """(policy, V) after the solve, in closed form."""
    rp = g.row_ptr
    S = ring + chain
    pi = np.zeros(g.n, np.int64)
    V = np.zeros(g.n, np.int64)
    pi[:ring] = rp[:ring]
    for i in range(1, chain + 1):
        pi[ring - 1 + i] = rp[ring - 1 + i] + 1
        V[ring - 1 + i] = -100 * i
    pi[S:] = rp[S:-1] + 1
    V[S] = -100 * (chain + 2)
    V[S + 1:] = -100 * (chain + 1)
    return pi, V
