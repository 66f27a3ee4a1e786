"""Writes synth_digests.txt: fingerprints of the generated inputs.

These are input fingerprints, not expected results: they let the test suite
check that a seed produces the same bytes on every machine (x86_64 here,
aarch64 next to the GPU).  Run from the repository root:
    python tests/golden/make_synth_digests.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import synth  # noqa: E402

CASES = {
    "ring10k": lambda: synth.ring10k(),
    "product4": lambda: synth.product4(),
    "locality_2^20": lambda: synth.locality32m(1 << 20),
    "diff1m_base": lambda: synth.diff1m_base(),
    "batch64": lambda: synth.batch4096(G=64, nmax=5000),
}

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_digests.txt")
    with open(out, "w") as f:
        f.write("# name n m digest(row_ptr) digest(col_idx) digest(w)\n")
        for name, make in CASES.items():
            g = make()
            f.write(f"{name} {g.row_ptr.shape[0]-1} {g.col_idx.shape[0]} {synth.digest(g.row_ptr)} "
                    f"{synth.digest(g.col_idx)} {synth.digest(g.w)}\n")
        sizes = synth.loguniform_sizes(4096, 100, 200000, synth.SEED_BASE + 3)
        f.write(f"batch_sizes_4096 {sizes.shape[0]} {int(sizes.sum())} {synth.digest(sizes)} 0 0\n")
    print("wrote", out)
