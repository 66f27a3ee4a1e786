"""Writes batch4096_values.txt: the CPU oracle's answer for every member of the
full batched workload (4096 graphs, sizes log-uniform in [100, 200000], each a
ring plus U{0..7} extra edges, w in U[1,10000], max).

Calls only oracle/ and synth/.  The GPU test of the batched form compares each
of the 4096 members (value, cycle length, cycle digest) with these lines.  The
graphs are independent, so they are solved by a process pool (spawned, so no
parent state is inherited); the oracle itself stays single-threaded.

Run from the repository root (a few minutes on 8 cores):
    python tests/golden/make_batch_values.py [--jobs J]
"""
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch4096_values.txt")
G, NMIN, NMAX = 4096, 100, 200000


def _solve(g):
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import synth
    sizes = synth.loguniform_sizes(G, NMIN, NMAX, synth.SEED_BASE + 3, tag=0)
    gr = synth.ring_extra(int(sizes[g]), 0, 7, 1, 10000, 1, seed=synth.SEED_BASE + 3,
                          tag=1000 + g, mode="max")
    h = oracle.howard(gr.row_ptr, gr.col_idx, gr.w, gr.mode)
    cyc = np.asarray(h.cycle, dtype=np.int32)
    return (g, gr.n, gr.m, h.num, h.den, int(cyc.shape[0]), h.iterations, synth.digest(cyc),
            int(cyc[0]))


def main():
    jobs = os.cpu_count() or 1
    if "--jobs" in sys.argv:
        jobs = int(sys.argv[sys.argv.index("--jobs") + 1])
    t = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(jobs) as pool:
        rows = sorted(pool.imap_unordered(_solve, range(G), chunksize=4))
    with open(OUT, "w") as f:
        f.write("# Oracle (CPU, exact) answer for every member of the batched workload batch4096;\n")
        f.write("# written by make_batch_values.py.  Edge ids are local to the member graph.\n")
        f.write("# g n m num den len iters cycle_digest first_edge\n")
        for r in rows:
            f.write(" ".join(str(int(x)) for x in r) + "\n")
    print(f"wrote {OUT} ({time.time() - t:.0f} s, {jobs} processes)")


if __name__ == "__main__":
    main()
