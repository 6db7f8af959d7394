"""Writes tests/golden/oracle_values.json from the CPU oracle alone.

Every stored value below is computed by ``oracle`` on inputs from
``graphgen``; nothing here runs the CUDA library.  Re-run after a change to
the oracle's arithmetic that a cited reading of the paper justifies:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402

CASES = {
    "complete9": lambda: gg.complete(9),
    "gnp40": lambda: gg.gnp(40, 0.3, 12),
    "chung_lu_2000": lambda: gg.chung_lu(2000, 12.0, 2.4, 150.0, 21),
}


def main():
    out = {}
    for name, make in CASES.items():
        g = make()
        og = O.prepare(g.off, g.col)
        N, C = O.exact_counts(g.off, g.col)
        k = 50000
        h6 = O.sample_3paths(og, k, 7)
        h4 = O.sample_centered(og, k, 7)
        st, est, lo, hi = O.estimate(og.W, og.Lambda, og.N1, h6, k, h4, k, 0.01)
        out[name] = {
            "n": g.n, "m": og.m, "W": og.W, "Lambda": og.Lambda, "N1": og.N1,
            "exact_C": [int(x) for x in C], "k": k, "seed": 7,
            "hist6": [int(x) for x in h6], "hist4": [int(x) for x in h4],
            "estimate": [float(x) for x in est],
        }
    with open(os.path.join(HERE, "oracle_values.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
