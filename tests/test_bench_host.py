"""Host-side measurement logic of bench.py (no GPU): the algorithmic-byte
numerators of the rooflines against plain loops over their definitions, the
issue peak, and the clock-record summary."""
import math

import numpy as np
import pytest

import bench
from paper_2011_03135_b300 import graphgen as gg


def _graphs():
    return [gg.rmat(8, 8.0, seed=3), gg.chung_lu(600, 6.0, 2.1, seed=4), gg.erdos_renyi(300, 0.05, seed=2),
            gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 2)])]


def _lists(g):
    rp = g.rowptr.astype(np.int64)
    return [g.col[rp[v]:rp[v + 1]].astype(np.int64).tolist() for v in range(g.n)]


def _before(d, x, v):
    # appendix "Orientation (Total Order)": x precedes v in the degree order
    return (d[x], x) < (d[v], v)


@pytest.mark.parametrize("gi", range(4))
def test_out_degrees_follow_the_degree_order(gi):
    g = _graphs()[gi]
    N = _lists(g)
    d = [len(a) for a in N]
    od, s, t = bench.out_degrees_np(g)
    arcs = sorted((v, x) for v in range(g.n) for x in N[v] if _before(d, v, x))
    assert sorted(zip(s.tolist(), t.tolist())) == arcs
    assert od.tolist() == [sum(1 for x in N[v] if _before(d, v, x)) for v in range(g.n)]
    assert len(arcs) * 2 == int(g.rowptr[-1])


@pytest.mark.parametrize("gi", range(4))
def test_four_cycle_bytes_are_the_wedge_scan(gi):
    # every vertex reads its list with the degrees (8 B per entry); each root
    # v0 scans, for every x before it in N(v0), x's two offsets and N(x) with
    # the degrees (16 B + 8 B per entry)
    g = _graphs()[gi]
    N = _lists(g)
    d = [len(a) for a in N]
    want = 8 * int(g.rowptr[-1])
    for v0 in range(g.n):
        for x in N[v0]:
            if _before(d, x, v0):
                want += 16 + 8 * d[x]
    assert bench.c4_pass_bytes(g) == want


@pytest.mark.parametrize("gi", range(4))
def test_clique_bytes_are_the_local_graph_reads(gi):
    # a root u of out-degree >= 2 reads its offsets and N+(u), and for every x
    # in N+(u) the offsets and N+(x)
    g = _graphs()[gi]
    N = _lists(g)
    d = [len(a) for a in N]
    out = [[x for x in N[v] if _before(d, v, x)] for v in range(g.n)]
    want = 0
    for u in range(g.n):
        if len(out[u]) >= 2:
            want += 16 + 4 * len(out[u]) + sum(16 + 4 * len(out[x]) for x in out[u])
    per_class, maxod = bench.clique_pass_bytes(g, {"warp_max_degree": 128, "cta_max_degree": 1024})
    assert sum(per_class.values()) == want
    assert maxod == max(len(a) for a in out)


def test_issue_peak():
    # 148 SMs x 4 schedulers x one warp instruction per clock
    assert math.isclose(bench.issue_peak(2032.0), 148 * 4 * 2.032)


def test_clock_summary_reports_throttle_reasons(tmp_path):
    rows = ["0, 2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2032, 2032, 950.3, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2032, 1010.0, 0x8, Active, Not Active, Not Active, Not Active",
            "0, 345, 2032, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    cs.proc = object()  # a sampler that ran
    s = cs.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["sm_max_mhz"] == 2032.0
    assert s["sm_mhz"] == 2032.0  # the idle sample is left out of the median
    assert s["samples"] == 4
