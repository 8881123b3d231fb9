"""Run one named workload through the library a few times (for profilers and demos).

  python -m paper_2011_03135_b300.cases --case clique-rmat20 [--reps N]

Cases build their seeded input, upload it once, then repeat the counting
path (orientation included) `reps` times and print the counts.
"""
from __future__ import annotations

import argparse
import json
import time

CASES = {
    # name: (generator, patterns)
    "clique-rmat20": ("rmat20", "clique45"),
    "clique-rmat21": ("rmat21", "clique45"),
    "clique6-rmat20": ("rmat20", "clique6"),
    "clique789-cl1m": ("chunglu1m", "clique789"),
    "clique7-rmat16": ("rmat16", "clique7"),
    "tc-rmat14": ("rmat14", "tc"),
    "motif4-rmat18": ("rmat18", "motif4"),
    "sl-chunglu1m": ("chunglu1m", "sl"),
    "sl-chunglu4m": ("chunglu4m", "sl"),
}


def _graph(name):
    from paper_2011_03135_b300 import graphgen as gg
    if name == "rmat20":
        return gg.workload_clique6_rmat20()
    if name == "rmat21":
        return gg.workload_clique_rmat21()
    if name == "rmat14":
        return gg.workload_tc_rmat14()
    if name == "rmat16":
        return gg.rmat(16, 16.0, seed=2)
    if name == "rmat18":
        return gg.rmat(18, 16.0, seed=2)
    if name == "chunglu1m":
        return gg.workload_clique789_chung_lu1m()
    if name == "chunglu4m":
        return gg.workload_sl_chung_lu4m()
    raise ValueError(name)


def _patterns(gpm, name):
    import numpy as np
    if name == "clique45":
        return [gpm.Pattern.clique(4), gpm.Pattern.clique(5)]
    if name == "clique6":
        return [gpm.Pattern.clique(6)]
    if name == "clique789":
        return [7, 8, 9]
    if name == "clique7":
        return [7]
    if name == "tc":
        return [gpm.Pattern.clique(3)]
    if name == "motif4":
        return gpm.Pattern.motifs(4)
    if name == "sl":
        d = np.zeros((4, 4), np.uint8)
        for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]:
            d[a, b] = d[b, a] = 1
        c = np.zeros((4, 4), np.uint8)
        for a, b in [(0, 2), (2, 1), (1, 3), (3, 0)]:
            c[a, b] = c[b, a] = 1
        return [gpm.Pattern.spec(d, induced=False), gpm.Pattern.spec(c, induced=False)]
    raise ValueError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=sorted(CASES), required=True)
    ap.add_argument("--reps", type=int, default=1)
    a = ap.parse_args()
    import torch
    from paper_2011_03135_b300 import gpm
    gname, pname = CASES[a.case]
    g = _graph(gname)
    G = gpm.Graph.from_host(g)
    pats = _patterns(gpm, pname)
    out = None
    for _ in range(a.reps):
        G.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = [gpm.count_cliques(G, k) for k in pats] if isinstance(pats[0], int) else gpm.count(G, pats)
        dt = time.perf_counter() - t0
    print(json.dumps({"case": a.case, "n": g.n, "m": g.m, "counts": out, "last_seconds": dt}))
    G.close()


if __name__ == "__main__":
    main()
