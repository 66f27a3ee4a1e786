"""Writes oracle_values.txt: the CPU oracle's answers on the full-size workloads.

Calls only oracle/ (and synth/ for the inputs).  The GPU parity tests compare
the CUDA path with these values where re-running the oracle inside a test
would take minutes (the 2^25-vertex locality graph), and they rebuild the
differentiation workload from the critical cycle recorded here.

Run from the repository root (takes a few minutes, mostly the 32M graph):
    python tests/golden/make_golden.py [--skip-large]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.txt")


def diff1m_unique(base: synth.Graph, cycle: np.ndarray) -> synth.Graph:
    """+1 on every edge of the base graph's critical cycle: with weights that
    are multiples of 1024 that cycle becomes the unique optimum (any other
    simple cycle shares at most |C|-1 of its edges)."""
    w = base.w.copy()
    w[cycle] += 1
    return synth.Graph(base.row_ptr, base.col_idx, w, base.mode, "diff1m")


def record(f, name, g, h, seconds):
    cyc = np.asarray(h.cycle, dtype=np.int32)
    head = " ".join(str(int(x)) for x in cyc[:16])
    f.write(f"{name} n={g.n} m={g.m} mode={g.mode} num={h.num} den={h.den} len={cyc.shape[0]} "
            f"iters={h.iterations} cycle_digest={synth.digest(cyc)} oracle_s={seconds:.1f} "
            f"head={head}\n")
    f.flush()


def main(skip_large: bool):
    with open(OUT, "w") as f:
        f.write("# Oracle (CPU, exact) answers on the synthetic workloads; written by make_golden.py.\n")
        f.write("# name n m mode num den len iters cycle_digest oracle_seconds head(first 16 edges)\n")
        work = [("ring10k", synth.ring10k), ("product4", synth.product4),
                ("locality_2^20", lambda: synth.locality32m(1 << 20))]
        for name, make in work:
            g = make()
            t = time.time()
            h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
            record(f, name, g, h, time.time() - t)
        base = synth.diff1m_base()
        t = time.time()
        hb = oracle.howard(base.row_ptr, base.col_idx, base.w, base.mode)
        record(f, "diff1m_base", base, hb, time.time() - t)
        f.write("diff1m_base_cycle " + " ".join(str(int(x)) for x in hb.cycle) + "\n")
        g = diff1m_unique(base, hb.cycle)
        t = time.time()
        h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
        record(f, "diff1m", g, h, time.time() - t)
        if not skip_large:
            g = synth.locality32m()
            t = time.time()
            h = oracle.howard(g.row_ptr, g.col_idx, g.w, g.mode)
            record(f, "locality32m", g, h, time.time() - t)
    print("wrote", OUT)


if __name__ == "__main__":
    main("--skip-large" in sys.argv)
