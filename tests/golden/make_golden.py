"""Write tests/golden/fullsize_counts.json: oracle counts for the full-size workloads.

Every value comes from ``oracle/`` alone (the seeded generators build the
inputs). Counts restricted to root ranges are exact partitions of the total
(each subgraph has exactly one root vertex under the oracle's root
conventions), so the ranges run in a spawn-started process pool and are
summed; nothing in the arithmetic depends on the split.

Usage:  python tests/golden/make_golden.py [--only NAME ...] [--procs P]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "fullsize_counts.json")

_G = None


def _largest_batch_motif4_rmat():
    """The largest R-MAT graph among the 4-motif queries of the 512-query batch."""
    from paper_2011_03135_b300 import graphgen as gg
    specs = [s for s in gg.batch_query_specs(512) if s["kind"] == "rmat" and s["k"] == 4]
    return max(specs, key=lambda s: (s["n"], s["edge_factor"]))


def _graph(name):
    from paper_2011_03135_b300 import graphgen as gg
    return {
        "tc_rmat14": gg.workload_tc_rmat14,
        "clique_rmat21": gg.workload_clique_rmat21,
        "sl_chunglu4m": gg.workload_sl_chung_lu4m,
        "clique789_chunglu1m": gg.workload_clique789_chung_lu1m,
        "motif4_batch_rmat20": lambda: gg.graph_from_spec(_largest_batch_motif4_rmat()),
    }[name]()


def _init(name):
    global _G
    _G = _graph(name)


def _work(args):
    what, lo, hi = args
    import oracle as O
    if what.startswith("clique"):
        return O.cliques(_G, int(what[6:]), lo, hi)
    if what == "diamond":
        return O.diamonds(_G, lo, hi)
    if what == "cycle4":
        return O.cycles4(_G, lo, hi)
    raise ValueError(what)


def run(name, whats, procs, chunks=512):
    g = _graph(name)
    res = dict(n=g.n, nnz=g.nnz, digest=g.digest())
    if whats == ["motifs4"]:
        # the six induced 4-vertex motif counts are global sums (per-edge
        # triangle terms), computed whole by the single-threaded oracle
        import oracle as O
        t0 = time.time()
        res["motifs4"] = O.motifs(g, 4)
        print(f"{name} motifs4 = {res['motifs4']}  ({time.time() - t0:.1f} s, 1 process)", flush=True)
        return res
    bounds = [g.n * i // chunks for i in range(chunks + 1)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_init, initargs=(name,)) as pool:
        for what in whats:
            t0 = time.time()
            tasks = [(what, bounds[i], bounds[i + 1]) for i in range(chunks)]
            total = sum(pool.map(_work, tasks, chunksize=1))
            res[what] = total
            res[what + "_oracle_core_seconds"] = None
            print(f"{name} {what} = {total}  ({time.time() - t0:.1f} s wall, {procs} procs)", flush=True)
    return res


PLAN = {
    "tc_rmat14": ["clique3", "clique4", "clique5"],
    "clique_rmat21": ["clique3", "clique4", "clique5"],
    "sl_chunglu4m": ["diamond", "cycle4", "clique3"],
    "clique789_chunglu1m": ["clique7", "clique8", "clique9"],
    "motif4_batch_rmat20": ["motifs4"],
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*")
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name, whats in PLAN.items():
        if a.only and name not in a.only:
            continue
        r = run(name, whats, a.procs)
        r = {k: v for k, v in r.items() if not k.endswith("_oracle_core_seconds")}
        data[name] = r
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
