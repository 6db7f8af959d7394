"""Writes tests/golden/exact_counts_rmat20.json from the CPU oracle alone.

The exact non-induced counts N (Eq. (1)'s right-hand side) and induced
counts C of the R-MAT scale-20 graph (seed 11), from ``oracle`` on the graph
``graphgen.rmat20()`` builds; nothing here runs the CUDA library.  The
oracle's plain enumeration took 7,979 s (about 2.2 hours) on one core for the
stored file:

    python tests/golden/make_exact_rmat20.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402


def main():
    g = gg.rmat20()
    t = time.time()
    N, C = O.exact_counts(g.off, g.col)
    out = {
        "graph": "R-MAT scale 20, edge factor 16, seed 11 (graphgen.rmat20)",
        "N": [int(x) for x in N],
        "C": [int(x) for x in C],
        "oracle_seconds": round(time.time() - t, 1),
    }
    path = os.path.join(HERE, "exact_counts_rmat20.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
