"""Benchmark: exact k-clique counting (k = 4 and 5) on the R-MAT scale-21 graph.

One step = the whole counting path on a device-resident CSR: degree-ordered
orientation, root-task classes, the fused local-graph pass that counts 3-, 4-
and 5-cliques, and the reduction to exact uint64 counts. `value` is the number
of 4- and 5-cliques counted per second of device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

At N = 1 the same line also carries the oracle's CPU baselines (one thread,
and the unchanged oracle over root ranges on every host core) and, under
"legs", the subgraph-listing workload (diamonds and 4-cycles on Chung-Lu 4M,
with the 4-cycle pass's HBM roofline and DRAM traffic) and triangle counting
on R-MAT 14, each checked against the oracle's stored totals.

Under torchrun (N > 1) every rank counts its own replica of the workload
(weak scaling, no collective on the data path); the slowest rank's time sets
the step time. `--impl reference` times the CPU oracle (single-threaded C) on
a bounded root sample of the same workload.

Other legs (one GPU, one JSON line each): `--workload tc`, `sl`, `motif5`
(the 21 five-vertex motifs, Erdos-Renyi 1M), `guided` (general patterns by
the pattern-guided search, Erdos-Renyi 1M), `clique6` (6-cliques, R-MAT 20),
`clique789` (7-, 8-, 9-cliques, Chung-Lu 1M), `batched` and `served` (many
small queries); `--orientation core` runs the headline leg under the
core value based (degeneracy) order, k-core peel included in each step;
`--case NAME --reps N` runs a named workload for a profiler.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4-clique/4-motif counts per sec, HBM GB/s % peak; batched vs plain speedup"
UNIT = "cliques/s (4- and 5-cliques counted)"
WORKLOAD = "k-clique counting k=4,5, R-MAT scale 21 (2,097,152 vertices), edge factor 16, (0.57,0.19,0.19,0.05), seed 2"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"gpm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def out_degrees_np(g):
    """Out-degrees in the orientation (input statistics for the roofline, numpy)."""
    d = np.diff(g.rowptr).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), d)
    dst = g.col.astype(np.int64)
    keep = (d[src] < d[dst]) | ((d[src] == d[dst]) & (src < dst))
    return np.bincount(src[keep], minlength=g.n), src[keep], dst[keep]


def clique_pass_bytes(g, opts):
    """Algorithmic DRAM bytes of the fused clique pass, per class of roots.

    Per root u (out-degree d_u >= 2): its two row offsets and N+(u), plus, for
    every member x of N+(u), its two row offsets and N+(x):
        16 + 4 d_u + sum_{x in N+(u)} (16 + 4 d_x).
    """
    od, s, t = out_degrees_np(g)
    inner = np.bincount(s, weights=(16 + 4 * od[t]).astype(np.float64), minlength=g.n)
    per_root = 16 + 4 * od + inner
    cls = np.full(g.n, -1)
    cls[(od >= 2) & (od <= 32)] = 0
    cls[(od > 32) & (od <= opts["warp_max_degree"])] = 1
    cls[(od > opts["warp_max_degree"]) & (od <= opts["cta_max_degree"])] = 2
    cls[(od > 384) & (od <= opts["cta_max_degree"])] = 4  # CTA roots above the split degree
    cls[od > opts["cta_max_degree"]] = 3
    names = {0: "lg_warp_d32", 1: "lg_warp", 2: "lg_cta_lo", 4: "lg_cta_hi", 3: "lg_cta_global"}
    return {names[c]: float(per_root[cls == c].sum()) for c in names}, int(od.max())


# Per-launch counters of the dominant kernel, per workload, from a one-pass
# `ncu` capture of the same kernel on the same workload
# (profiles/lg_cta_hi_rmat21_counters.md, profiles/lg_cta_hi_k6_rmat20_counters.md,
# profiles/lg_cta_lo_k789_chunglu1m_counters.md):
#   ncu --metrics smsp__inst_executed.sum,gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none -k regex:lg_cta_kernel -c 1
#       python bench.py --case <clique-rmat21 | clique6-rmat20> --reps 1
#   (clique789-cl1m: -c 6, every lg_cta_kernel launch of one step)
# valid only for the kernel sources they were taken on (digest of
# csrc/lg_device.cuh + csrc/clique.cu); a stale entry is ignored.
NCU_COUNTERS = {
    "clique-rmat21": {
        "lg_cta_hi": {"digest": "88c1037f49f64430", "inst_per_launch": 151170055324,
                      "dram_bytes_per_launch": 28273152 + 3584, "ncu_ms": 184.272},
    },
    "clique6-rmat20": {
        "lg_cta_hi": {"digest": "88c1037f49f64430", "inst_per_step": 1638179347992,
                      "dram_bytes_per_step": 13086464, "ncu_ms": 1676.139},
    },
    # every 4-cycle kernel launch of one step (c4_bound x 2, 42 pull passes of
    # c4_pull_mark x 2, c4_pull, c4_pull_tiny, c4_pull_rows; c4_bucket,
    # c4_small; the per-graph tables excluded), summed;
    # profiles/c4_sl_chunglu4m_dram.md; digest of motif.cu + motif_device.cuh + c4_pull.cu
    "sl-chunglu4m": {
        "c4": {"digest": "ae36e12d04121df9", "dram_bytes_per_step": 84845894144},
    },
    # profiles/enum_k5_er1m_counters.md; digest of enumerate.cu
    "motif5-er1m": {
        "enum_kernel_k5": {"digest": "8422a055c7d075f6", "inst_per_launch": 226039644786,
                           "dram_bytes_per_launch": 44991232 + 972544, "ncu_ms": 266.830},
    },
    # three launches per step (6-path, 5-star, 6-cycle), summed;
    # profiles/guided_er1m_counters.md; digest of guided.cu
    "guided-er1m": {
        "guided_kernel": {"digest": "90803c4b5ac813dc",
                          "inst_per_step": 2031750401033 + 116953504346 + 246503983250,
                          "dram_bytes_per_step": 49243136 + 6882816 + 48381184 + 51968 + 48180224 + 465920},
    },
    # three launches per step (k = 7, 8, 9), summed
    "clique789-cl1m": {
        "lg_cta_lo": {"digest": "88c1037f49f64430", "inst_per_step": 18019851342 + 36222280753 + 85370485547,
                      "dram_bytes_per_step": 6813952 + 6629632 + 6719744, "ncu_ms": 27.188 + 64.375 + 179.117},
    },
}


def counters_for(case, name):
    cnt = NCU_COUNTERS.get(case, {}).get(name)
    return cnt if cnt and cnt.get("digest") == kernel_digest() else None


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for f in ("lg_device.cuh", "clique.cu"):
        h.update(open(os.path.join(ROOT, "paper_2011_03135_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def c4_digest():
    import hashlib
    h = hashlib.sha256()
    for f in ("motif.cu", "motif_device.cuh", "c4_pull.cu"):
        h.update(open(os.path.join(ROOT, "paper_2011_03135_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def issue_peak(sm_mhz):
    """Warp-instruction issue peak: 148 SMs x 4 schedulers x 1 instruction per clock."""
    return 148 * 4 * sm_mhz * 1e6 / 1e9  # G warp-instructions / s


def cpu_baseline(g, seconds_target=15.0):
    """The oracle, as it stands, on a bounded root sample of the same workload."""
    import oracle as O
    import multiprocessing  # noqa: F401  (the oracle is single-threaded; nothing is forked)
    # vertex ids are randomly permuted by the generator, so an id range is a random root sample
    lo, hi = 0, 4096
    t0 = time.perf_counter()
    c4 = O.cliques(g, 4, lo, hi)
    c5 = O.cliques(g, 5, lo, hi)
    dt = time.perf_counter() - t0
    if dt < seconds_target / 4:
        hi = min(g.n, int(hi * seconds_target / max(dt, 1e-3)))
        t0 = time.perf_counter()
        c4 = O.cliques(g, 4, lo, hi)
        c5 = O.cliques(g, 5, lo, hi)
        dt = time.perf_counter() - t0
    return {"value": (c4 + c5) / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": _cpu_model(),
            "roots": hi - lo, "seconds": dt,
            "sample": f"roots with id in [{lo}, {hi}) of {g.n} (random sample: ids are permuted); "
                      f"4-CL + 5-CL single-threaded, {dt:.1f} s, counts {c4} + {c5}"}


_CPU_G = None


def _cpu_init(n, rp_path, col_path):
    """Worker set-up of the all-core oracle leg: the CSR, memory-mapped."""
    global _CPU_G
    from paper_2011_03135_b300 import graphgen as gg
    _CPU_G = gg.Graph(n, np.load(rp_path, mmap_mode="r"), np.load(col_path, mmap_mode="r"))


def _cpu_work(task):
    ks, lo, hi = task
    import oracle as O
    return sum(O.cliques(_CPU_G, k, lo, hi) for k in ks)


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline_all_cores(g, ks, unit, single, seconds_target=6.0):
    """The same oracle code, unchanged, over root ranges on every host core
    (a spawn-started process pool: no fork after the GPU is in use). The
    sample is the prefix [0, hi) of the randomly permuted ids, sized from the
    single-threaded rate for about `seconds_target` of wall time, cut into two
    ranges per process (every oracle call orients the whole graph first, so
    few calls per process; the ids are a random permutation, so ranges of
    equal length carry similar work)."""
    import multiprocessing as mp
    import tempfile
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    per_root_s = single["seconds"] / max(single["roots"], 1)
    hi = int(min(g.n, max(single["roots"], cores * seconds_target / max(per_root_s, 1e-9))))
    nchunks = max(1, min(hi, cores * 2))
    bounds = [hi * i // nchunks for i in range(nchunks + 1)]
    tasks = [(tuple(ks), bounds[i], bounds[i + 1]) for i in range(nchunks) if bounds[i + 1] > bounds[i]]
    with tempfile.TemporaryDirectory(prefix="gpm_cpu_") as d:
        rp_path, col_path = os.path.join(d, "rowptr.npy"), os.path.join(d, "col.npy")
        np.save(rp_path, g.rowptr)
        np.save(col_path, g.col)
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_cpu_init, initargs=(g.n, rp_path, col_path)) as pool:
            pool.map(_cpu_work, [tasks[0]])  # workers started before the clock
            t0 = time.perf_counter()
            total = sum(pool.map(_cpu_work, tasks, chunksize=1))
            dt = time.perf_counter() - t0
    return {"value": total / dt, "unit": unit, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
            "sample": f"roots with id in [0, {hi}) of {g.n} (random sample: ids are permuted) in {len(tasks)} chunks "
                      f"over {cores} processes; {'+'.join(str(k) for k in ks)}-cliques, {dt:.1f} s wall, total {total}"}


BATCH_WORKLOAD = ("batched 3-/4-motif counting: 512 queries, each on its own seeded graph, Erdos-Renyi (mean degree "
                  "8-64) or R-MAT (edge factor 4-32), 1K-1M vertices log-uniform")


def run_batched(args, graphs=None):
    """Batched form vs the plain one-query-per-call path on the same resident graphs (same GPU)."""
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    specs = gg.batch_query_specs(args.batch_queries)
    if graphs is None:
        graphs = gg.generate_many(specs)
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    Gs = [gpm.Graph.from_host(g, validate=False) for g in graphs]
    for G in Gs:
        G.prepare()
    setup_s = time.perf_counter() - t0
    kinds = [gpm.QUERY_MOTIF3 if s["k"] == 3 else gpm.QUERY_MOTIF4 for s in specs]
    pats = {k: gpm.plain_patterns(k) for k in set(kinds)}

    def plain():
        return [gpm.count(G, pats[k]) for G, k in zip(Gs, kinds)]

    want = plain()  # warm-up; also builds the lazily created task lists
    torch.cuda.synchronize()
    plain_t = []
    for _ in range(max(1, args.batch_steps)):
        t0 = time.perf_counter()
        got = plain()
        plain_t.append(time.perf_counter() - t0)
        assert got == want
    # per-query wall times of the plain path (each count returns its counts to the host)
    per_q = []
    for G, k in zip(Gs, kinds):
        t0 = time.perf_counter()
        gpm.count(G, pats[k])
        per_q.append(time.perf_counter() - t0)
    per_q = np.array(per_q)
    order = np.argsort(-per_q)
    plain_profile = {"top10pct_share": float(per_q[order[:max(1, len(per_q) // 10)]].sum() / per_q.sum()),
                     "queries_under_1ms": int((per_q < 1e-3).sum()), "seconds_under_1ms": float(per_q[per_q < 1e-3].sum()),
                     "largest_s": [round(float(x), 4) for x in per_q[order[:8]]],
                     "largest_edges": [int(graphs[i].m) for i in order[:8]]}
    B = gpm.Batch(list(zip(Gs, kinds)))
    t0 = time.perf_counter()
    first = B.run()  # autotunes the item schedule
    tune_s = time.perf_counter() - t0
    assert first == want, "batched counts differ from the plain path"
    batch_t = []
    for _ in range(max(1, args.batch_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = B.run()
        batch_t.append(time.perf_counter() - t0)
        assert got == want
    info = B.info()
    B.close()
    nq = len(specs)
    pq = nq / (sum(plain_t) / len(plain_t))
    bq = nq / (sum(batch_t) / len(batch_t))

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    # the queries under 1 ms of plain time alone: batched vs plain
    small = [i for i in range(nq) if per_q[i] < 1e-3]
    subset = None
    if small:
        Bs = gpm.Batch([(Gs[i], kinds[i]) for i in small])
        assert Bs.run() == [want[i] for i in small]
        bs = timed(Bs.run)
        ps = timed(lambda: [gpm.count(Gs[i], pats[kinds[i]]) for i in small])
        Bs.close()
        subset = {"queries": len(small), "plain_queries_per_s": len(small) / ps,
                  "batched_queries_per_s": len(small) / bs, "speedup": ps / bs}
    # the heaviest queries alone: the persistent kernel on all their items
    # (no plain-path fallback) against their plain launch chain
    heavy = []
    old = gpm.get_options()
    try:
        gpm.set_options(batch_direct_us=0xffffffff)
        for i in order[:12]:
            B1 = gpm.Batch([(Gs[i], kinds[i])])
            assert B1.run() == [want[i]]
            t_items = timed(B1.run)
            B1.close()
            t_plain = timed(lambda: gpm.count(Gs[i], pats[kinds[i]]))
            heavy.append({"query": int(i), "kind": "3-motif" if kinds[i] == gpm.QUERY_MOTIF3 else "4-motif",
                          "graph": graphs[i].name, "edges": int(graphs[i].m), "plain_s": t_plain,
                          "persistent_s": t_items, "persistent_over_plain": t_items / t_plain})
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})
    for G in Gs:
        G.close()
    return {"workload": BATCH_WORKLOAD, "queries": nq, "edges_total": int(sum(g.m for g in graphs)),
            "plain_queries_per_s": pq, "batched_queries_per_s": bq, "speedup": bq / pq,
            "plain_s": plain_t, "batched_s": batch_t, "autotune_s": tune_s, "setup_s": setup_s,
            "plain_per_query": plain_profile, "sub_1ms_subset": subset, "heaviest_alone": heavy,
            "schedule": info, "equal_counts": True}


SERVED_WORKLOAD = ("served: 64 resident R-MAT graphs (scale 12+(i mod 11), edge factor 8/16/32 by seeded draw, "
                   "seed 100+i), Poisson arrivals at 2000 queries/s (seed 5), query kind uniform over "
                   "{triangles, 4-cliques, 5-cliques, 4-motifs}, graph uniform over the 64")


def served_specs():
    specs = []
    for i in range(64):
        r = np.random.default_rng(100 + i)
        scale = 12 + (i % 11)
        specs.append(dict(kind="rmat", k=4, scale=scale, n=1 << scale, edge_factor=float([8, 16, 32][r.integers(3)]),
                          seed=100 + i))
    return specs


def served_trace(rate, seconds, ngraphs, seed=5):
    r = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += r.exponential(1.0 / rate)
        if t > seconds:
            return out
        out.append((t, int(r.integers(ngraphs)), int(r.integers(4))))


def _pct(xs, q):
    return float(np.percentile(np.array(xs), q)) if xs else None


def run_served(args):
    """Continuous-batching server vs plain serial serving of the same arrival trace (same GPU)."""
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    specs = served_specs()
    graphs = gg.generate_many(specs)
    torch.cuda.set_device(0)
    Gs = [gpm.Graph.from_host(g, validate=False) for g in graphs]
    kinds = [gpm.QUERY_TC, gpm.QUERY_CLIQUE4, gpm.QUERY_CLIQUE5, gpm.QUERY_MOTIF4]
    trace = served_trace(args.serve_rate, args.serve_seconds, len(Gs))
    horizon = args.serve_seconds + args.serve_grace
    t0 = time.perf_counter()
    S = gpm.Server(Gs, max_inflight=512)
    start_s = time.perf_counter() - t0
    # served
    done, lat = {}, []
    i = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while i < len(trace) and trace[i][0] <= now:
            _, gi, ki = trace[i]
            S.submit(gi, kinds[ki], i)
            i += 1
        for tag, gi, kind, status, counts in S.poll():
            assert status == 0
            done[tag] = counts
            lat.append(time.perf_counter() - t0 - trace[tag][0])
        if (i == len(trace) and len(done) == len(trace)) or now > horizon:
            break
        time.sleep(0.0002)
    served_elapsed = min(time.perf_counter() - t0, horizon)
    S.stop()
    # plain serial serving of the same trace: one query at a time, each after its arrival
    pats = {k: gpm.plain_patterns(k) for k in kinds}
    plain_done, plain_lat = {}, []
    t0 = time.perf_counter()
    for tag, (ta, gi, ki) in enumerate(trace):
        now = time.perf_counter() - t0
        if now > horizon:
            break
        if ta > now:
            time.sleep(ta - now)
        c = gpm.count(Gs[gi], pats[kinds[ki]])
        plain_done[tag] = c
        plain_lat.append(time.perf_counter() - t0 - ta)
    plain_elapsed = min(time.perf_counter() - t0, horizon)
    mismatches = sum(1 for t, c in done.items() if t in plain_done and plain_done[t] != c)
    # sampled oracle check on the smallest graphs
    import oracle as O
    checked = 0
    for tag, counts in sorted(done.items())[:2000]:
        _, gi, ki = trace[tag]
        if graphs[gi].n > (1 << 12) or checked >= 8:
            continue
        g = graphs[gi]
        want = ([O.triangles(g)] if ki == 0 else [O.cliques(g, 4)] if ki == 1 else [O.cliques(g, 5)] if ki == 2
                else O.motifs(g, 4))
        assert counts == want, (tag, gi, ki)
        checked += 1
    for G in Gs:
        G.close()
    return {"workload": SERVED_WORKLOAD, "offered_per_s": args.serve_rate, "window_s": args.serve_seconds,
            "horizon_s": horizon, "offered": len(trace), "server_start_s": start_s,
            "served": {"completed": len(done), "queries_per_s": len(done) / served_elapsed,
                       "p50_s": _pct(lat, 50), "p99_s": _pct(lat, 99), "backlog": len(trace) - len(done)},
            "plain": {"completed": len(plain_done), "queries_per_s": len(plain_done) / plain_elapsed,
                      "p50_s": _pct(plain_lat, 50), "p99_s": _pct(plain_lat, 99),
                      "backlog": len(trace) - len(plain_done)},
            "mismatches_vs_plain": mismatches, "oracle_checked": checked}


SL_WORKLOAD = ("subgraph listing, edge-induced diamond and 4-cycle: Chung-Lu 4,194,304 vertices, mean degree 24, "
               "exponent 2.1, seed 3; exact counts plus the first 10^6 matches of each")


def c4_pass_bytes(g):
    """Algorithmic bytes of the 4-cycle pass: every vertex reads its list and the degrees
    of its neighbours (8 B per entry); every arc x -> v0 of the orientation makes v0 scan
    N(x) with the degrees (16 B of offsets + 8 B per entry)."""
    od, s, t = out_degrees_np(g)
    d = np.diff(g.rowptr).astype(np.float64)
    return 8.0 * g.nnz + float(np.sum(od * (16.0 + 8.0 * d)))


def run_sl(args):
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    import oracle as O
    g = gg.workload_sl_chung_lu4m()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    c4opts = {k: v for k, v in dict(c4_range_bound=args.c4_range_bound, c4_range_width=args.c4_range_width,
                                    c4_hub_bound=args.c4_hub_bound, c4_pull_bound=args.c4_pull_bound).items() if v}
    if c4opts:
        gpm.set_options(**c4opts)
    G = gpm.Graph(torch.from_numpy(g.rowptr.view(np.int64)).to(dev), torch.from_numpy(g.col.view(np.int32)).to(dev),
                  g.n, validate=True, stream=stream)
    D = gpm.Pattern.spec(O.DIAMOND, induced=False)
    C = gpm.Pattern.spec(O.CYCLE4, induced=False)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step():
        G.reset()
        return gpm.count(G, [D, C], stream=stream)

    counts = None
    for _ in range(max(args.warmup, 3)):
        counts = step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpm.profile_reset()
    gpm.profile_enable(True)
    launches0 = gpm.kernel_launches()
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            assert step() == counts
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpm.profile_enable(False)
    launches = gpm.kernel_launches() - launches0
    prof = gpm.profile_report()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    # listing the first 10^6 matches of each pattern
    t0 = time.perf_counter()
    ld, td = gpm.list_embeddings(G, D, cap=1_000_000, stream=stream)
    lc, tc = gpm.list_embeddings(G, C, cap=1_000_000, stream=stream)
    list_s = time.perf_counter() - t0
    assert (td, tc) == tuple(counts) and len(ld) == min(td, 10 ** 6) and len(lc) == min(tc, 10 ** 6)
    peak, peak_kind = _peaks()
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    roof = None
    if top[0].startswith("c4_"):
        c4ms = sum(v["ms"] for k, v in prof.items() if k.startswith("c4_")) / args.steps
        ach = c4_pass_bytes(g) / (c4ms / 1000.0) / 1e9
        c4k = " + ".join(sorted(k for k in prof if k.startswith("c4_") and k.endswith("_kernel")
                                and k not in ("c4_bound_kernel", "c4_edeg_kernel", "c4_hub_units_kernel")))
        alg = c4_pass_bytes(g)
        roof = {"bound": "hbm", "kernel": c4k, "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_kind,
                "algorithmic_bytes_per_step": alg, "ms_per_step_4cycle_kernels": c4ms,
                "kernel_digest": c4_digest()}
        cnt = NCU_COUNTERS.get("sl-chunglu4m", {}).get("c4")
        if cnt and cnt.get("digest") == c4_digest():
            roof.update(traffic=cnt["dram_bytes_per_step"], traffic_over_algorithmic=cnt["dram_bytes_per_step"] / alg,
                        traffic_note="DRAM bytes per step of the 4-cycle kernels (ncu, every launch of one step)")
    G.close()
    return {"workload": SL_WORKLOAD, "c4_options": gpm.get_options(), "counts": {"diamond": counts[0], "4-cycle": counts[1]},
            "ms_per_step": ms, "matches_per_s": (counts[0] + counts[1]) / (ms / 1000.0),
            "listing_s_for_2x10^6": list_s, "gpu_launches": launches, "roofline": roof, "clocks": clk.summary(),
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}


def _golden(name):
    p = os.path.join(ROOT, "tests", "golden", "fullsize_counts.json")
    try:
        return json.load(open(p)).get(name)
    except (OSError, ValueError):
        return None


def compact_sl(d):
    """The SL leg for the headline line: counts (and whether they equal the
    oracle's stored totals), time per step, the 4-cycle pass roofline."""
    gold = _golden("sl_chunglu4m")
    keep = ("workload", "counts", "ms_per_step", "matches_per_s", "listing_s_for_2x10^6", "gpu_launches",
            "roofline", "clocks")
    out = {k: d[k] for k in keep if k in d}
    out["kernels"] = dict(list(d["kernels"].items())[:6])
    if gold:
        out["equal_to_oracle_totals"] = (d["counts"]["diamond"] == gold.get("diamond")
                                         and d["counts"]["4-cycle"] == gold.get("cycle4"))
    return out


CLIQUE6_WORKLOAD = ("6-clique counting, R-MAT scale 20 (1,048,576 vertices), edge factor 16, (0.57,0.19,0.19,0.05), "
                    "seed 2")
CLIQUE789_WORKLOAD = ("k-clique counting k = 7, 8, 9 (one count per k), Chung-Lu 1,048,576 vertices, mean degree 24, "
                      "exponent 2.1, seed 3")


def run_large_k(args, workload, g, ks, case):
    """Counting k-cliques for large k through gpm_count_cliques: k = 6 is the
    fused pass with a fourth bitmap level, k >= 7 the generic search."""
    import torch
    from paper_2011_03135_b300 import gpm
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    G = gpm.Graph(torch.from_numpy(g.rowptr.view(np.int64)).to(dev), torch.from_numpy(g.col.view(np.int32)).to(dev),
                  g.n, validate=True, stream=stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step():
        G.reset()
        return [gpm.count_cliques(G, k, stream=stream) for k in ks]

    counts = None
    for _ in range(max(args.warmup, 3)):
        counts = step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = gpm.kernel_launches()
    gpm.profile_reset()
    gpm.profile_enable(True)
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            assert step() == counts
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpm.profile_enable(False)
    launches = gpm.kernel_launches() - launches0
    prof = gpm.profile_report()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    total = sum(counts)
    rp_h = torch.from_numpy(g.rowptr.view(np.int64)).pin_memory()
    col_h = torch.from_numpy(g.col.view(np.int32)).pin_memory()
    e2e = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = gpm.Graph(rp_h, col_h, g.n, validate=True, stream=stream)
        c = [gpm.count_cliques(H, k, stream=stream) for k in ks]
        H.close()
        if i > 0:
            e2e.append(time.perf_counter() - t0)
        assert c == counts
    e2e_s = sum(e2e) / len(e2e)
    name, st = max(prof.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = st["ms"] / max(st["launches"], 1)
    clk_now = clk.summary()
    ipeak = issue_peak(clk_now["sm_mhz"] or 2032.0)
    cnt = counters_for(case, name)
    roof = {"bound": "alu", "kernel": name, "unit": "G warp-instructions/s", "peak": ipeak,
            "peak_source": "148 SMs x 4 schedulers x 1 issue/clk x median SM clock under load",
            "achieved": None, "frac": None, "traffic": None, "kernel_digest": kernel_digest()}
    if cnt:
        # counters summed over the kernel's launches in one step (one per k)
        kms = prof[name]["ms"] / args.steps
        ach = cnt["inst_per_step"] / (kms / 1000.0) / 1e9
        roof.update(achieved=ach, frac=ach / ipeak, traffic=cnt.get("dram_bytes_per_step"),
                    traffic_note="DRAM bytes per step of this kernel (all its launches)")
    unit = "cliques/s (" + ", ".join(f"{k}-cliques" for k in ks) + ")"
    line = {"workload": workload, "metric": unit.split(" (")[0] + " counted per second", "value": total / (ms / 1000.0),
            "unit": unit, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "step_ms": step_ms, "counts": {f"{k}-clique": c for k, c in zip(ks, counts)}, "dtype": "u64",
            "data": "synthetic", "config": {"l2": "flushed between steps (512 MB write)"},
            "e2e": {"value": total / e2e_s, "unit": unit, "h2d_bytes_per_step": g.rowptr.nbytes + g.col.nbytes,
                    "d2h_bytes_per_step": 8 * len(ks), "seconds": e2e_s},
            "gpu_launches": launches, "roofline": roof, "clocks": clk_now,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_large_k(g, ks, unit)
    G.close()
    return line


def cpu_baseline_large_k(g, ks, unit, seconds_target=15.0):
    """The oracle on a bounded root sample of the same workload (ids are permuted: a random sample)."""
    import oracle as O
    lo, hi = 0, 256
    t0 = time.perf_counter()
    cs = [O.cliques(g, k, lo, hi) for k in ks]
    dt = time.perf_counter() - t0
    if dt < seconds_target / 4:
        hi = min(g.n, int(hi * seconds_target / max(dt, 1e-3)))
        t0 = time.perf_counter()
        cs = [O.cliques(g, k, lo, hi) for k in ks]
        dt = time.perf_counter() - t0
    return {"value": sum(cs) / dt, "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"roots with id in [{lo}, {hi}) of {g.n}; single-threaded, {dt:.1f} s, counts {cs}"}


MOTIF5_WORKLOAD = ("5-vertex motif counting (all 21 connected induced 5-vertex patterns) by pattern-oblivious "
                   "enumeration with connectivity codes: Erdos-Renyi 1,048,576 vertices, mean degree 8, seed 7")


def enum_digest():
    import hashlib
    return hashlib.sha256(open(os.path.join(ROOT, "paper_2011_03135_b300", "csrc", "enumerate.cu"), "rb").read()
                          ).hexdigest()[:16]


def run_motif5(args):
    """All 21 induced 5-vertex motif counts in one call (one enumeration per step)."""
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    g = gg.workload_motif5_er1m()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    G = gpm.Graph(torch.from_numpy(g.rowptr.view(np.int64)).to(dev), torch.from_numpy(g.col.view(np.int32)).to(dev),
                  g.n, validate=True, stream=stream)
    M = gpm.Pattern.motifs(5)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step():
        G.reset()
        return gpm.count(G, M, stream=stream)

    counts = None
    for _ in range(max(args.warmup, 3)):
        counts = step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = gpm.kernel_launches()
    gpm.profile_reset()
    gpm.profile_enable(True)
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            assert step() == counts
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpm.profile_enable(False)
    launches = gpm.kernel_launches() - launches0
    prof = gpm.profile_report()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    total = sum(counts)
    clk_now = clk.summary()
    ipeak = issue_peak(clk_now["sm_mhz"] or 2032.0)
    kname = "enum_kernel_k5"
    kms = prof.get(kname, {"ms": 0.0})["ms"] / args.steps
    roof = {"bound": "alu", "kernel": kname, "unit": "G warp-instructions/s", "peak": ipeak,
            "peak_source": "148 SMs x 4 schedulers x 1 issue/clk x median SM clock under load",
            "achieved": None, "frac": None, "traffic": None, "kernel_digest": enum_digest()}
    cnt = NCU_COUNTERS.get("motif5-er1m", {}).get(kname)
    if cnt and cnt.get("digest") == enum_digest() and kms > 0:
        ach = cnt["inst_per_launch"] / (kms / 1000.0) / 1e9
        roof.update(achieved=ach, frac=ach / ipeak, traffic=cnt.get("dram_bytes_per_launch"))
    line = {"workload": MOTIF5_WORKLOAD, "metric": "connected induced 5-vertex subgraphs counted per second",
            "value": total / (ms / 1000.0), "unit": "5-vertex subgraphs/s", "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "counts": counts, "subgraphs": total, "dtype": "u64",
            "data": "synthetic", "config": {"l2": "flushed between steps (512 MB write)"}, "gpu_launches": launches,
            "roofline": roof, "clocks": clk_now,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}
    if not args.no_cpu_baseline:
        import oracle as O
        hi = 256
        t0 = time.perf_counter()
        c, _ = O.motifs5(g, 0, hi)
        dt = time.perf_counter() - t0
        hi = min(g.n, int(hi * 10.0 / max(dt, 1e-3)))
        t0 = time.perf_counter()
        c, _ = O.motifs5(g, 0, hi)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sum(c) / dt, "unit": "5-vertex subgraphs/s", "cores": 1, "kind": "oracle",
                                "sample": f"roots (smallest vertex) with id in [0, {hi}) of {g.n}; single-threaded, "
                                          f"{dt:.1f} s, {sum(c)} subgraphs"}
    G.close()
    return line


GUIDED_WORKLOAD = ("pattern-guided search (matching order, symmetry-breaking bounds, degree filter): edge-induced "
                   "6-vertex path, 5-star and 6-cycle on Erdos-Renyi 1,048,576 vertices, mean degree 8, seed 7")
GUIDED_PATTERNS = {"6-path": [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)],
                   "5-star": [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5)],
                   "6-cycle": [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0)]}


def guided_digest():
    import hashlib
    return hashlib.sha256(open(os.path.join(ROOT, "paper_2011_03135_b300", "csrc", "guided.cu"), "rb").read()
                          ).hexdigest()[:16]


def run_guided(args):
    """Counts of general patterns by the pattern-guided search, one search per pattern per step."""
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    g = gg.workload_motif5_er1m()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    G = gpm.Graph(torch.from_numpy(g.rowptr.view(np.int64)).to(dev), torch.from_numpy(g.col.view(np.int32)).to(dev),
                  g.n, validate=True, stream=stream)

    def pat(es):
        k = max(max(e) for e in es) + 1
        a = np.zeros((k, k), np.uint8)
        for u, v in es:
            a[u, v] = a[v, u] = 1
        return gpm.Pattern.spec(a, induced=False)

    P = [pat(es) for es in GUIDED_PATTERNS.values()]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def step():
        G.reset()
        return gpm.count_guided(G, P, stream=stream)

    counts = None
    for _ in range(max(args.warmup, 3)):
        counts = step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = gpm.kernel_launches()
    gpm.profile_reset()
    gpm.profile_enable(True)
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[i][0].record(stream)
            assert step() == counts
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    gpm.profile_enable(False)
    launches = gpm.kernel_launches() - launches0
    prof = gpm.profile_report()
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    clk_now = clk.summary()
    ipeak = issue_peak(clk_now["sm_mhz"] or 2032.0)
    kms = prof.get("guided_kernel", {"ms": 0.0})["ms"] / args.steps
    roof = {"bound": "alu", "kernel": "guided_kernel", "unit": "G warp-instructions/s", "peak": ipeak,
            "peak_source": "148 SMs x 4 schedulers x 1 issue/clk x median SM clock under load",
            "achieved": None, "frac": None, "traffic": None, "kernel_digest": guided_digest()}
    cnt = NCU_COUNTERS.get("guided-er1m", {}).get("guided_kernel")
    if cnt and cnt.get("digest") == guided_digest() and kms > 0:
        ach = cnt["inst_per_step"] / (kms / 1000.0) / 1e9
        roof.update(achieved=ach, frac=ach / ipeak, traffic=cnt.get("dram_bytes_per_step"))
    total = sum(counts)
    line = {"workload": GUIDED_WORKLOAD, "metric": "pattern embeddings (distinct subgraphs) counted per second",
            "value": total / (ms / 1000.0), "unit": "subgraphs/s", "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "counts": dict(zip(GUIDED_PATTERNS, counts)), "dtype": "u64", "data": "synthetic",
            "config": {"l2": "flushed between steps (512 MB write)"}, "gpu_launches": launches, "roofline": roof,
            "clocks": clk_now,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}}
    G.close()
    return line


TC_WORKLOAD = "triangle counting, R-MAT scale 14 (16,384 vertices), edge factor 16, (0.57,0.19,0.19,0.05), seed 1"


def run_tc(args):
    """Triangle counting on the small R-MAT: launch- and latency-bound (the graph fits L2)."""
    import torch
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg
    g = gg.workload_tc_rmat14()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    G = gpm.Graph(torch.from_numpy(g.rowptr.view(np.int64)).to(dev), torch.from_numpy(g.col.view(np.int32)).to(dev),
                  g.n, validate=True, stream=stream)
    P = [gpm.Pattern.clique(3)]
    for _ in range(max(args.warmup, 3)):
        G.reset()
        want = gpm.count(G, P, stream=stream)
    # whole path (orientation + count) and count alone on the oriented graph
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    for i in range(args.steps):
        ev[i][0].record(stream)
        G.reset()
        assert gpm.count(G, P, stream=stream) == want
        ev[i][1].record(stream)
        ev2[i][0].record(stream)
        gpm.count_async(G, P, out, stream=stream)
        ev2[i][1].record(stream)
    torch.cuda.synchronize()
    assert int(out.item()) == want[0]
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    ms2 = sum(a.elapsed_time(b) for a, b in ev2) / len(ev2)
    G.close()
    gold = _golden("tc_rmat14")
    return {"workload": TC_WORKLOAD, "triangles": want[0], "equal_to_oracle_total": bool(gold) and gold.get("clique3") == want[0],
            "ms_per_step_with_orientation": ms,
            "ms_count_only": ms2, "triangles_per_s": want[0] / (ms2 / 1000.0),
            "note": "the graph (1.7 MB CSR) is L2-resident; the path is launch/latency-bound"}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_2011_03135_b300 import graphgen as gg
    import oracle as O
    g = gg.workload_clique_rmat21()
    # each step: the oracle on a fixed root sample [0, hi) sized so that the
    # whole run takes about 150 s. Vertex ids are a random permutation, so a
    # prefix of ids is a random sample; hi grows by half until one sample takes at
    # least half a step's share (these trials are the warm-up)
    lo, hi = 0, 256
    step_budget = 150.0 / max(1, args.steps + args.warmup)
    while True:
        t0 = time.perf_counter()
        O.cliques(g, 4, lo, hi)
        O.cliques(g, 5, lo, hi)
        dt = time.perf_counter() - t0
        if dt >= step_budget / 2 or hi >= g.n:
            break
        hi = min(g.n, hi + hi // 2)
    times, total = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        c = O.cliques(g, 4, lo, hi) + O.cliques(g, 5, lo, hi)
        times.append(time.perf_counter() - t0)
        total += c
    value = total / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"roots [{lo}, {hi})"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"roots with id in [{lo}, {hi}) per step, 4-CL + 5-CL"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2011_03135_b300 import gpm
    from paper_2011_03135_b300 import graphgen as gg

    g = gg.workload_clique_rmat21()
    dev = torch.device("cuda", local)
    rp_d = torch.from_numpy(g.rowptr.view(np.int64)).to(dev)
    col_d = torch.from_numpy(g.col.view(np.int32)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    G = gpm.Graph(rp_d, col_d, g.n, validate=True, stream=stream)
    if args.orientation != "degree":
        G.set_orientation(args.orientation)
    pats = [gpm.Pattern.clique(4), gpm.Pattern.clique(5)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (126 MB)

    def step():
        G.reset()
        return gpm.count(G, pats, stream=stream)

    counts = None
    for _ in range(max(args.warmup, 3)):
        counts = step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = gpm.kernel_launches()
    gpm.profile_reset()
    gpm.profile_enable(True)
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict the graph from L2 between steps
                ev[i][0].record(stream)
            c = step()
            ev[i][1].record(stream)
            assert c == counts, "counts changed between steps"
        torch.cuda.synchronize()
    gpm.profile_enable(False)
    launches = gpm.kernel_launches() - launches0
    prof = gpm.profile_report()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    units = (counts[0] + counts[1]) * world
    value = units / (ms / 1000.0)

    # end to end through the C-ABI with host buffers (pinned): upload, validate, orient, count, read back
    rp_h = torch.from_numpy(g.rowptr.view(np.int64)).pin_memory()
    col_h = torch.from_numpy(g.col.view(np.int32)).pin_memory()
    e2e_times = []
    for i in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = gpm.Graph(rp_h, col_h, g.n, validate=True, stream=stream)
        if args.orientation != "degree":
            H.set_orientation(args.orientation)
        c = gpm.count(H, pats, stream=stream)
        H.close()
        dt = time.perf_counter() - t0
        assert c == counts
        if i > 0:
            e2e_times.append(dt)
    e2e_s = sum(e2e_times) / len(e2e_times)
    h2d = g.rowptr.nbytes + g.col.nbytes

    # rooflines of the dominant kernel: instruction issue (the binding resource of the
    # bitmap search) and HBM (algorithmic bytes; the oriented graph is L2-resident)
    opts = gpm.get_options()
    alg_bytes, max_od = clique_pass_bytes(g, opts)
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, st = top
    per_launch_ms = st["ms"] / max(st["launches"], 1)
    peak, peak_kind = _peaks()
    clk_now = clk.summary()
    digest = kernel_digest()
    # the counters and the algorithmic bytes are for the degree order
    cnt = counters_for("clique-rmat21", name) if args.orientation == "degree" else None
    ipeak = issue_peak(clk_now["sm_mhz"] or 2032.0)
    roof = {"bound": "alu", "kernel": name, "unit": "G warp-instructions/s", "peak": ipeak,
            "peak_source": "148 SMs x 4 schedulers x 1 issue/clk x median SM clock under load",
            "achieved": None, "frac": None, "traffic": None, "kernel_digest": digest}
    if cnt:
        ach = cnt["inst_per_launch"] / (per_launch_ms / 1000.0) / 1e9
        roof.update(achieved=ach, frac=ach / ipeak, traffic=cnt.get("dram_bytes_per_launch"))
    roof_hbm = {"bound": "hbm", "kernel": name, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "peak_source": peak_kind}
    if name in alg_bytes and args.orientation == "degree":
        ach = alg_bytes[name] / (per_launch_ms / 1000.0) / 1e9
        roof_hbm.update(achieved=ach, frac=ach / peak)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": world, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas{world}", "counts": {"4-clique": counts[0], "5-clique": counts[1]},
                       "orientation": args.orientation,
                       "max_out_degree": max_od},
            "e2e": {"value": (counts[0] + counts[1]) * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 16, "seconds": e2e_s},
            "gpu_launches": launches, "roofline": roof, "roofline_hbm": roof_hbm, "clocks": clk_now,
            "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / max(v["launches"], 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
            "step_ms": step_ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(g, (4, 5), UNIT, line["cpu_baseline"])
    G.close()
    del rp_d, col_d, flush
    if rank == 0 and world == 1 and not args.no_legs:
        # the other configurations on the same GPU, compact (full lines: --workload sl / tc)
        line["legs"] = {"sl": compact_sl(run_sl(args)), "tc": run_tc(args)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# Named workloads for profilers (`--case NAME --reps N`): build the seeded
# input, upload it once, repeat the counting path (orientation included) `reps`
# times and print the counts. No timing is reported: a profiler measures.
CASES = {
    "clique-rmat20": ("rmat20", "clique45"),
    "clique-rmat21": ("rmat21", "clique45"),
    "clique6-rmat20": ("rmat20", "clique6"),
    "clique789-cl1m": ("chunglu1m", "clique789"),
    "clique7-rmat16": ("rmat16", "clique7"),
    "tc-rmat14": ("rmat14", "tc"),
    "motif4-rmat18": ("rmat18", "motif4"),
    "sl-chunglu1m": ("chunglu1m", "sl"),
    "sl-chunglu2m": ("chunglu2m", "sl"),
    "sl-chunglu4m": ("chunglu4m", "sl"),
    "motif5-er1m": ("er1m", "motif5"),
    "guided-er1m": ("er1m", "guided"),
}


def _case_graph(name):
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
    if name == "chunglu2m":
        return gg.chung_lu(1 << 21, 24.0, 2.1, seed=3)
    if name == "chunglu4m":
        return gg.workload_sl_chung_lu4m()
    if name == "er1m":
        return gg.workload_motif5_er1m()
    raise ValueError(name)


def _case_patterns(gpm, name):
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
    if name == "motif5":
        return gpm.Pattern.motifs(5)
    if name == "guided":
        out = []
        for es in GUIDED_PATTERNS.values():
            k = max(max(e) for e in es) + 1
            a = np.zeros((k, k), np.uint8)
            for u, v in es:
                a[u, v] = a[v, u] = 1
            out.append(gpm.Pattern.spec(a, induced=False))
        return out
    if name == "sl":
        d = np.zeros((4, 4), np.uint8)
        for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]:
            d[a, b] = d[b, a] = 1
        c = np.zeros((4, 4), np.uint8)
        for a, b in [(0, 2), (2, 1), (1, 3), (3, 0)]:
            c[a, b] = c[b, a] = 1
        return [gpm.Pattern.spec(d, induced=False), gpm.Pattern.spec(c, induced=False)]
    raise ValueError(name)


def run_case(args):
    import torch
    from paper_2011_03135_b300 import gpm
    gname, pname = CASES[args.case]
    g = _case_graph(gname)
    G = gpm.Graph.from_host(g)
    pats = _case_patterns(gpm, pname)
    out = None
    for _ in range(args.reps):
        G.reset()
        if isinstance(pats[0], int):
            out = [gpm.count_cliques(G, k) for k in pats]
        elif pname == "guided":
            out = gpm.count_guided(G, pats)
        else:
            out = gpm.count(G, pats)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": g.n, "m": g.m, "counts": out}))
    G.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--orientation", choices=["degree", "core"], default="degree",
                    help="order of the orientation for the k-clique leg (core: k-core peel at prepare time)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="headline leg only (no sl / tc legs in its line)")
    ap.add_argument("--workload", choices=["cliques", "clique6", "clique789", "batched", "served", "sl", "tc", "motif5",
                                           "guided"],
                    default="cliques")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-grace", type=float, default=10.0)
    ap.add_argument("--batch-queries", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--c4-range-bound", type=int, default=0, help="4-cycle tuning for the sl leg (0: library default)")
    ap.add_argument("--c4-range-width", type=int, default=0)
    ap.add_argument("--c4-hub-bound", type=int, default=0)
    ap.add_argument("--c4-pull-bound", type=int, default=0)
    ap.add_argument("--case", choices=sorted(CASES), help="run a named workload for a profiler and exit")
    ap.add_argument("--reps", type=int, default=1)
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        print(json.dumps(run_batched(args)), flush=True)
        return 0
    if args.workload == "served":
        print(json.dumps(run_served(args)), flush=True)
        return 0
    if args.workload == "sl":
        print(json.dumps(run_sl(args)), flush=True)
        return 0
    if args.workload == "tc":
        print(json.dumps(run_tc(args)), flush=True)
        return 0
    if args.workload == "motif5":
        print(json.dumps(run_motif5(args)), flush=True)
        return 0
    if args.workload == "guided":
        print(json.dumps(run_guided(args)), flush=True)
        return 0
    if args.workload == "clique6":
        from paper_2011_03135_b300 import graphgen as gg
        print(json.dumps(run_large_k(args, CLIQUE6_WORKLOAD, gg.workload_clique6_rmat20(), (6,), "clique6-rmat20")),
              flush=True)
        return 0
    if args.workload == "clique789":
        from paper_2011_03135_b300 import graphgen as gg
        print(json.dumps(run_large_k(args, CLIQUE789_WORKLOAD, gg.workload_clique789_chung_lu1m(), (7, 8, 9),
                                     "clique789-cl1m")), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
