"""Writes single_values.txt: the CPU oracle's answers in the paper's
single-lambda form of the iteration (Alg. 1 with the rebuild) on the
full-size workloads.

Calls only oracle/ (and synth/ for the inputs).  The GPU tests compare the
CUDA path's single-lambda solve with these values where re-running the oracle
inside a test would take minutes.

Run from the repository root (a few minutes, mostly the 2^25-vertex graph):
    python tests/golden/make_single_values.py [--skip-large]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_values.txt")


def record(f, name, g, s, seconds):
    cyc = np.asarray(s.cycle, dtype=np.int32)
    head = " ".join(str(int(x)) for x in cyc[:16])
    f.write(f"{name} n={g.n} m={g.m} mode={g.mode} num={s.num} den={s.den} len={cyc.shape[0]} "
            f"iters={s.iterations} cycle_digest={synth.digest(cyc)} "
            f"policy_digest={synth.digest(s.policy)} oracle_s={seconds:.1f} head={head}\n")
    f.flush()


def main(skip_large: bool):
    work = [("ring10k", synth.ring10k), ("product4", synth.product4),
            ("locality_2^20", lambda: synth.locality32m(1 << 20)),
            ("diff1m_base", synth.diff1m_base)]
    if not skip_large:
        work.append(("locality32m", synth.locality32m))
    with open(OUT, "w") as f:
        f.write("# Oracle (CPU, exact) answers of the single-lambda iteration; written by "
                "make_single_values.py.\n")
        f.write("# name n m mode num den len iters cycle_digest policy_digest oracle_seconds "
                "head(first 16 edges)\n")
        for name, make in work:
            g = make()
            t = time.time()
            s = oracle.howard_single(g.row_ptr, g.col_idx, g.w, g.mode)
            record(f, name, g, s, time.time() - t)
    print("wrote", OUT)


if __name__ == "__main__":
    main("--skip-large" in sys.argv)
