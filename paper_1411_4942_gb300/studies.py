"""Accuracy studies through the batched path: synthetic counterparts of the
paper's Section 6 experiments on convergence with k, on the 3-path sampler
against the centred sampler for the cycle-based motifs, and on the Corollary
5.3 error bars against the actual error.

Every sampling run of a study (all graphs, seeds, sample sizes and both
samplers) is one request of one batched launch; the exact counts come from
the library's exact counter and the estimates from its estimator.

    python -m paper_1411_4942_gb300.studies --graphs chung_lu_5k rmat20 --seeds 32
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import batch as B
from . import pathsample as ps

MOTIFS = ["3-star", "3-path", "tailed-tri", "4-cycle", "chordal", "4-clique"]


def run(graphs: dict, seeds, ks, delta: float = 0.01, cfg: B.LaunchConfig | None = None) -> dict:
    """graphs: name -> ps.Graph.  Returns per graph the exact counts and, for
    each k and motif, the mean relative error over the seeds of the final
    estimates and of the 3-path sampler's own C4..C6, the fraction of runs
    whose bars hold the exact count, and the mean relative bar half-width."""
    names = list(graphs)
    gset = B.GraphSet([graphs[n] for n in names])
    reqs, key = [], {}
    for gi, _ in enumerate(names):
        for s in seeds:
            for k in ks:
                for sampler in (0, 1):
                    key[(gi, s, k, sampler)] = len(reqs)
                    reqs.append(B.Request(gi, sampler, int(k), int(s), slot=len(reqs)))
    runner = B.BatchRunner(gset, reqs, cfg or B.LaunchConfig())
    runner.launch()
    hist = runner.histograms()
    out = {}
    for gi, name in enumerate(names):
        G = graphs[name]
        _, C, _ = G.count_exact()
        C = C.astype(np.float64)
        rows = []
        for k in ks:
            rel_final, rel_basic, cover, width = [], [], [], []
            for s in seeds:
                h6 = hist[key[(gi, s, k, 0)]]
                h4 = hist[key[(gi, s, k, 1)]][:4]
                rc, est, lo, hi = ps.ps_estimate_ex(G.stats, h6, k, h4, k, delta, 0)
                _, best, _, _ = ps.ps_estimate_ex(G.stats, h6, k, h4, k, delta, ps.PS_EST_3PATH_ONLY)
                with np.errstate(divide="ignore", invalid="ignore"):
                    rel_final.append(np.abs(est - C) / C)
                    rel_basic.append(np.abs(best - C) / C)
                    width.append(np.maximum(hi - est, est - lo) / C)
                cover.append((lo <= C) & (C <= hi))
            rows.append({
                "k": int(k),
                "rel_err": np.mean(rel_final, axis=0).tolist(),
                "rel_err_3path_only": np.mean(rel_basic, axis=0).tolist(),
                "coverage": np.mean(cover, axis=0).tolist(),
                "rel_halfwidth": np.mean(width, axis=0).tolist(),
            })
        out[name] = {"exact": C.astype(np.int64).tolist(), "seeds": len(seeds), "delta": delta,
                     "by_k": rows}
    return out


def table(result: dict) -> str:
    """Markdown summary: relative error of the final estimate (and of the
    3-path sampler alone for C4..C6), bar coverage, per k."""
    lines = []
    for name, r in result.items():
        lines.append(f"**{name}** (exact C1..C6 = {r['exact']}, {r['seeds']} seeds, delta {r['delta']})")
        lines.append("")
        lines.append("| k | " + " | ".join(MOTIFS) + " | 4-cycle / chordal / clique, 3-path sampler only | coverage (min) |")
        lines.append("|---|" + "---|" * 8)
        for row in r["by_k"]:
            fe = " | ".join(f"{x:.2e}" for x in row["rel_err"])
            be = " / ".join(f"{x:.2e}" for x in row["rel_err_3path_only"][3:])
            lines.append(f"| 2^{int(np.log2(row['k']))} | {fe} | {be} | {min(row['coverage']):.2f} |")
        lines.append("")
    return "\n".join(lines)


def main(argv=None):
    import graphgen as gg
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--graphs", nargs="+", default=["chung_lu_5k", "rmat20"])
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--log2k", type=int, nargs=2, default=[12, 22])
    ap.add_argument("--delta", type=float, default=0.01)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    makers = {"chung_lu_5k": gg.chung_lu_5k, "rmat20": gg.rmat20, "social3m": gg.social_chung_lu_3m}
    graphs = {}
    for name in a.graphs:
        g = makers[name]()
        graphs[name] = ps.Graph(g.off, g.col)
    ks = [1 << e for e in range(a.log2k[0], a.log2k[1] + 1)]
    res = run(graphs, list(range(1, a.seeds + 1)), ks, a.delta)
    print(table(res))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
