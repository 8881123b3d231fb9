"""GPU path vs the CPU oracle, element by element, through the C-ABI.

All counts are integers, so the bar is bit-exact equality. Small graphs
(n <= 30) cover every pattern class against the oracle's brute force tier;
medium graphs span every root class (warp, CTA, global-memory bitmaps) and a
ragged tail; the full-size workloads are checked on sampled root ranges the
oracle computes one by one, and on totals stored by tests/golden/make_golden.py
(which calls only the oracle).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2011_03135_b300 import graphgen as gg

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_counts.json")


@pytest.fixture(scope="module")
def gpm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_03135_b300 import gpm as m
    return m


def _golden():
    if os.path.exists(GOLDEN):
        return json.load(open(GOLDEN))
    return {}


SMALL = [
    gg.complete(6), gg.complete(9), gg.complete_multipartite([2, 3, 4]), gg.complete_multipartite([3, 3]),
    gg.petersen(), gg.cycle(4), gg.cycle(7), gg.star(6), gg.path(5), gg.empty(4),
    gg.from_edges(2, [(0, 1)]), gg.from_edges(3, [(0, 1), (1, 2)]),
] + [gg.random_small(n, p, s) for s, (n, p) in enumerate(
    [(10, 0.5), (14, 0.4), (18, 0.35), (22, 0.3), (25, 0.25), (28, 0.2), (30, 0.3), (30, 0.5), (16, 0.8),
     (20, 0.6), (24, 0.15), (29, 0.45)])] + [gg.rmat(5, 6.0, seed=s) for s in range(4)]


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_small_graph_every_pattern(gpm, gi):
    g = SMALL[gi]
    G = gpm.Graph.from_host(g)
    cl = [gpm.Pattern.clique(k) for k in (1, 2, 3, 4, 5, 6)]
    assert gpm.count(G, cl) == [g.n, g.m] + [O.cliques(g, k) for k in (3, 4, 5, 6)]
    m4 = gpm.Pattern.motifs(4)
    m3 = gpm.Pattern.motifs(3)
    assert gpm.count(G, m4) == O.motifs(g, 4)
    assert gpm.count(G, m3) == O.motifs(g, 3)
    ni4 = [gpm.Pattern.spec(p, induced=False) for p in O.MOTIF4_PATTERNS]
    ni3 = [gpm.Pattern.spec(p, induced=False) for p in O.MOTIF3_PATTERNS]
    assert gpm.count(G, ni4) == O.noninduced_terms(g, 4)
    assert gpm.count(G, ni3) == O.noninduced_terms(g, 3)
    # every pattern alone gives the same as in a group
    for p, want in zip(m4 + ni4, O.motifs(g, 4) + O.noninduced_terms(g, 4)):
        assert gpm.count(G, [p]) == [want]
    G.close()


def _medium():
    return [gg.rmat(11, 16.0, seed=21), gg.rmat(12, 8.0, seed=22), gg.erdos_renyi(3000, 0.01, seed=23, permute=True),
            gg.chung_lu(5000, 16.0, 2.1, seed=24)]


@pytest.mark.parametrize("opts", [dict(), dict(warp_max_degree=32, cta_max_degree=32),
                                  dict(warp_max_degree=64, cta_max_degree=64),
                                  dict(warp_max_degree=256, cta_max_degree=1024),
                                  dict(warp_max_degree=32, cta_max_degree=96)])
def test_medium_graphs_every_root_class(gpm, opts):
    old = gpm.get_options()
    try:
        if opts:
            gpm.set_options(**opts)
        for g in _medium():
            G = gpm.Graph.from_host(g)
            info = G.prepare().info()
            assert info["dag_arcs"] == g.m
            assert info["max_out_degree"] == int(O.out_degrees(g).max())
            cl = [gpm.Pattern.clique(k) for k in (3, 4, 5, 6)]
            assert gpm.count(G, cl) == [O.cliques(g, k) for k in (3, 4, 5, 6)], g.name
            assert gpm.count(G, gpm.Pattern.motifs(4)) == O.motifs(g, 4), g.name
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def test_root_ranges_match_oracle(gpm):
    g = gg.rmat(12, 16.0, seed=31)
    G = gpm.Graph.from_host(g)
    pats = [gpm.Pattern.clique(3), gpm.Pattern.clique(4), gpm.Pattern.clique(5),
            gpm.Pattern.spec(O.DIAMOND, induced=False), gpm.Pattern.spec(O.CYCLE4, induced=False),
            gpm.Pattern.clique(6)]
    cuts = [0, 1, 777, 2048, 2049, 3333, g.n]
    tot = [0] * 6
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        got = gpm.count_roots(G, pats, lo, hi)
        want = [O.cliques(g, 3, lo, hi), O.cliques(g, 4, lo, hi), O.cliques(g, 5, lo, hi),
                O.diamonds(g, lo, hi), O.cycles4(g, lo, hi), O.cliques(g, 6, lo, hi)]
        assert got == want, (lo, hi)
        tot = [a + b for a, b in zip(tot, got)]
    assert tot == gpm.count(G, pats)
    G.close()


def _multi_hub_graph(hubs=(1500, 2200, 3100), nl=3200, nm=120, per=3, seed=6):
    """Hubs joined to random subsets of a set L, each vertex of L joined to
    `per` random vertices of a set M: the hubs are 4-cycle roots whose lists
    are longer than one 1024-entry chunk, with wedges hub - x - w through L."""
    rng = np.random.default_rng(seed)
    nh = len(hubs)
    L0, M0 = nh, nh + nl
    e = []
    for h, d in enumerate(hubs):
        e += [(h, L0 + int(x)) for x in rng.choice(nl, size=d, replace=False)]
    for x in range(nl):
        e += [(L0 + x, M0 + int(w)) for w in rng.choice(nm, size=per, replace=False)]
    return gg.from_edges(nh + nl + nm, e, name="multihub")


NEVER = 0xffffffff


def _wide_root_graph(nl=2000, per=300, nm=50000, seed=8):
    """One hub joined to nl vertices, each joined to `per` random vertices of
    a set of nm: the hub's wedge bound is about nl (per + 1) = 602,000, above
    the bucketed kernel's narrow-table bound (524,288)."""
    rng = np.random.default_rng(seed)
    L0, M0 = 1, 1 + nl
    e = [(0, L0 + i) for i in range(nl)]
    for i in range(nl):
        e += [(L0 + i, M0 + int(w)) for w in rng.choice(nm, size=per, replace=False)]
    return gg.from_edges(1 + nl + nm, e, name="wide-root")


@pytest.mark.parametrize("width,bound,pull", [(98304, 1048576, 262144), (98304, 512, NEVER), (512, 512, NEVER),
                                              (64, 2000, NEVER), (1000, 4000, NEVER), (98304, 512, 512),
                                              (512, 512, 4000), (98304, 4000, 600), (98304, NEVER, 2000),
                                              (98304, 0xfffffffe, 0xfffffffe)])
def test_cycles4_range_path(gpm, width, bound, pull):
    # large roots counted range by range over vertex ids with a dense
    # shared-memory tally, or 128 at a time by the pull over every list with
    # bit-sliced counters: narrow ranges make many ranges per root, low bounds
    # send most roots there (several pull passes, the last one partial), and
    # the multi-hub graph has roots whose lists span several 1024-entry chunks
    # and vertices of degree > 1024 that precede some roots of a pass and not
    # others; with both bounds at their largest the bucketed class takes roots
    # up to 2^20 (the wide-root graph's hub with wider tables in half of the
    # warps); totals, root ranges (passes with no root in the range skipped)
    # and the motif inversion against the oracle
    old = gpm.get_options()
    try:
        gpm.set_options(c4_range_width=width, c4_range_bound=bound, c4_pull_bound=pull)
        C = gpm.Pattern.spec(O.CYCLE4, induced=False)
        extra = [_wide_root_graph()] if bound == 0xfffffffe else []
        for g in _medium() + [gg.rmat(12, 16.0, seed=31), _multi_hub_graph()] + extra:
            G = gpm.Graph.from_host(g)
            want = O.cycles4(g)
            assert gpm.count(G, [C]) == [want], g.name
            assert gpm.count(G, [C]) == [want], g.name  # the tally was left at zero
            cuts = [0, g.n // 3, g.n // 3 + 1, g.n - 5, g.n]
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                assert gpm.count_roots(G, [C], lo, hi) == [O.cycles4(g, lo, hi)], (g.name, lo, hi)
            assert gpm.count(G, gpm.Pattern.motifs(4)) == O.motifs(g, 4), g.name
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


@pytest.mark.parametrize("hub_bound", [513, 4000, 60000])
def test_cycles4_hub_path(gpm, hub_bound):
    # a low hub threshold sends many roots of medium graphs through the
    # whole-grid tally path (groups of roots per launch, tally reset by the
    # next launch); totals, root ranges and the motif inversion must not change.
    # The plain path takes the hub class only with the range and pull classes switched off.
    old = gpm.get_options()
    try:
        gpm.set_options(c4_hub_bound=hub_bound, c4_range_bound=NEVER, c4_pull_bound=NEVER)
        C = gpm.Pattern.spec(O.CYCLE4, induced=False)
        for g in _medium():
            G = gpm.Graph.from_host(g)
            assert gpm.count(G, [C]) == [O.cycles4(g)], g.name
            assert gpm.count(G, [C]) == [O.cycles4(g)], g.name  # tallies were left at zero
            cuts = [0, g.n // 3, g.n // 3 + 1, g.n - 5, g.n]
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                assert gpm.count_roots(G, [C], lo, hi) == [O.cycles4(g, lo, hi)], (g.name, lo, hi)
            assert gpm.count(G, gpm.Pattern.motifs(4)) == O.motifs(g, 4), g.name
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def _adjacent(g, u, v):
    nb = g.neighbors(int(u))
    i = np.searchsorted(nb, v)
    return i < len(nb) and nb[i] == v


def _edge_keys(g, adj, tuples):
    """Per tuple, the sorted codes of the graph edges its pattern edges land on."""
    k = adj.shape[0]
    t = np.asarray(tuples, dtype=np.int64).reshape(-1, k)
    cols = [np.minimum(t[:, i], t[:, j]) * g.n + np.maximum(t[:, i], t[:, j])
            for i in range(k) for j in range(i + 1, k) if adj[i, j]]
    return np.sort(np.stack(cols, axis=1), axis=1)


def _check_tuples(g, adj, info, tuples):
    """Each tuple is an embedding satisfying the constraints; all are distinct subgraphs."""
    k = adj.shape[0]
    pedges = [(i, j) for i in range(k) for j in range(i + 1, k) if adj[i, j]]
    seen = set()
    for t in np.asarray(tuples).tolist():
        assert len(set(t)) == k
        for i, j in pedges:
            assert _adjacent(g, t[i], t[j]), (t, i, j)
        for a, b in info["sb_pairs"]:
            assert t[a] < t[b], (t, a, b)
        es = frozenset((min(t[i], t[j]), max(t[i], t[j])) for i, j in pedges)
        assert es not in seen
        seen.add(es)
    return seen


def _check_tuples_all(g, adj, info, tuples):
    """Vectorised _check_tuples for large listings: distinct vertices per
    tuple, every pattern edge on a graph edge, the symmetry-breaking
    constraints, and distinct subgraphs (edge sets) over all tuples."""
    k = adj.shape[0]
    t = np.asarray(tuples, dtype=np.int64).reshape(-1, k)
    srt = np.sort(t, axis=1)
    assert (srt[:, 1:] != srt[:, :-1]).all()
    deg = np.diff(g.rowptr.astype(np.int64))
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.col.astype(np.int64)
    codes = src[src < dst] * g.n + dst[src < dst]  # ascending: rows ascending, lists sorted
    for i in range(k):
        for j in range(i + 1, k):
            if adj[i, j]:
                c = np.minimum(t[:, i], t[:, j]) * g.n + np.maximum(t[:, i], t[:, j])
                pos = np.minimum(np.searchsorted(codes, c), len(codes) - 1)
                assert (codes[pos] == c).all(), (i, j)
    for a, b in info["sb_pairs"]:
        assert (t[:, a] < t[:, b]).all(), (a, b)
    assert len(np.unique(_edge_keys(g, adj, t), axis=0)) == len(t)


LIST_PATTERNS = [
    (O.DIAMOND, False),
    (O.CYCLE4, False),
    (O.pattern(4, [(2, 3), (2, 0), (2, 1), (3, 0), (3, 1)]), False),   # diamond, other numbering
    (O.pattern(4, [(0, 1), (1, 2), (2, 3), (3, 0)]), False),           # 4-cycle, other numbering
    (O.clique_pattern(3), True), (O.clique_pattern(4), True), (O.clique_pattern(5), True),
    (O.clique_pattern(6), True), (O.clique_pattern(7), True), (O.clique_pattern(8), True),
]


@pytest.mark.parametrize("pi", range(len(LIST_PATTERNS)))
def test_listing_all_small(gpm, pi):
    adj, induced = LIST_PATTERNS[pi]
    for g in SMALL[:8] + SMALL[12:20]:
        G = gpm.Graph.from_host(g)
        P = gpm.Pattern.spec(adj, induced=induced)
        want = O.bf_subgraph_set(g, adj)
        tuples, total = gpm.list_embeddings(G, P, cap=len(want) + 5)
        assert total == len(want) == len(tuples)
        assert _check_tuples(g, adj, P.info(), tuples) == want
        G.close()


@pytest.mark.parametrize("pi", range(len(LIST_PATTERNS)))
def test_listing_capped(gpm, pi):
    adj, induced = LIST_PATTERNS[pi]
    g = gg.rmat(10, 16.0, seed=41)
    G = gpm.Graph.from_host(g)
    P = gpm.Pattern.spec(adj, induced=induced)
    total_want = gpm.count(G, [P])[0]
    for cap in (1, 1000, 12345):
        tuples, total = gpm.list_embeddings(G, P, cap=cap)
        assert total == total_want
        assert len(tuples) == min(cap, total)
        _check_tuples(g, adj, P.info(), tuples)
    G.close()


def test_listing_into_device_tensor(gpm):
    import torch
    g = gg.rmat(9, 8.0, seed=5)
    G = gpm.Graph.from_host(g)
    P = gpm.Pattern.spec(O.DIAMOND, induced=False)
    out = torch.zeros((500, 4), dtype=torch.int32, device="cuda")
    tuples, total = gpm.list_embeddings(G, P, cap=500, out=out)
    _check_tuples(g, O.DIAMOND, P.info(), tuples.cpu().numpy().astype(np.int64))
    G.close()


def test_count_async_and_device_input(gpm):
    import torch
    g = gg.rmat(10, 8.0, seed=7)
    rp = torch.from_numpy(g.rowptr.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    G = gpm.Graph(rp, col, g.n)
    G.prepare()
    pats = gpm.Pattern.motifs(4)
    out = torch.zeros(6, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    gpm.count(G, pats, stream=s)  # builds lazily-created task lists
    gpm.count_async(G, pats, out, stream=s)
    s.synchronize()
    assert [int(x) for x in out.cpu()] == O.motifs(g, 4)
    G.close()


def _bad(n, rows):
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = []
    for v, r in enumerate(rows):
        col += r
        rp[v + 1] = len(col)
    return rp, np.array(col, dtype=np.uint32)


@pytest.mark.parametrize("rows,code", [
    ([[1, 1], [0, 0]], "DUPLICATE"),
    ([[2, 1], [0], [0]], "NOT_SORTED"),
    ([[0, 1], [0, 1]], "SELF_LOOP"),
    ([[1, 2], [2], [0], []], "ASYMMETRIC"),     # 0 in N(2) is missing its mirror in N(1)
    ([[1], [0, 1]], "ASYMMETRIC"),              # odd nnz: rejected on the host
    ([[5], [0]], "OUT_OF_RANGE"),
])
def test_validation_rejects_malformed_csr(gpm, rows, code):
    rp, col = _bad(len(rows), rows)
    with pytest.raises(gpm.GpmError) as e:
        gpm.Graph(rp, col, len(rp) - 1)
    assert e.value.name == code


def _hub_rows(h):
    # hubs 0 and 1 each joined to leaves 2..h+1: rows of h entries
    return [list(range(2, h + 2)), list(range(2, h + 2))] + [[0, 1] for _ in range(h)]


def _long_row_cases(h=3000):
    swapped = _hub_rows(h)
    swapped[0][100], swapped[0][101] = swapped[0][101], swapped[0][100]
    unmirrored = _hub_rows(h)
    unmirrored[h + 1] = []  # 0 -> h+1 and 1 -> h+1 have no mirror; nnz stays even
    outside = _hub_rows(h)
    outside[0][-1] = outside[1][-1] = h + 2
    outside[h + 1] = []
    doubled = _hub_rows(h)
    doubled[0][50] = doubled[0][49]
    return [(swapped, "NOT_SORTED"), (unmirrored, "ASYMMETRIC"), (outside, "OUT_OF_RANGE"),
            (doubled, "DUPLICATE")]


@pytest.mark.parametrize("case", range(4))
def test_validation_rejects_malformed_long_rows(gpm, case):
    # rows above 2048 entries are checked by their own kernel: every fault
    # planted here lies in the two hub rows only
    rows, code = _long_row_cases()[case]
    rp, col = _bad(len(rows), rows)
    with pytest.raises(gpm.GpmError) as e:
        gpm.Graph(rp, col, len(rp) - 1)
    assert e.value.name == code


def test_validation_accepts_rows_at_and_above_the_split(gpm):
    # hub 0 has 2048 neighbours (warp-per-vertex check), hub 1 2049 (long-row
    # check), the leaves form a path
    edges = [(0, k) for k in range(2, 2050)] + [(1, k) for k in range(2, 2051)] + [(k, k + 1) for k in range(2, 2050)]
    g = gg.from_edges(2051, edges)
    assert np.diff(g.rowptr.astype(np.int64))[:2].tolist() == [2048, 2049]
    G = gpm.Graph.from_host(g)
    assert gpm.count(G, [gpm.Pattern.clique(3), gpm.Pattern.clique(4)]) == [O.triangles(g), O.cliques(g, 4)]
    G.close()


def test_degenerate_graphs(gpm):
    for g in (gg.empty(1), gg.empty(100), gg.from_edges(2, [(0, 1)])):
        G = gpm.Graph.from_host(g)
        assert gpm.count(G, [gpm.Pattern.clique(3), gpm.Pattern.clique(5)]) == [0, 0]
        assert gpm.count(G, gpm.Pattern.motifs(4)) == [0] * 6
        t, total = gpm.list_embeddings(G, gpm.Pattern.spec(O.DIAMOND, induced=False), cap=10)
        assert total == 0 and len(t) == 0
        G.close()


# ---------------- full-size workloads ----------------

def test_fullsize_tc_rmat14(gpm):
    g = gg.workload_tc_rmat14()
    gold = _golden().get("tc_rmat14", {})
    G = gpm.Graph.from_host(g)
    got = gpm.count(G, [gpm.Pattern.clique(k) for k in (3, 4, 5)])
    assert got == [O.triangles(g), O.cliques(g, 4), O.cliques(g, 5)]
    if gold:
        assert gold["digest"] == g.digest()
        assert got == [gold["clique3"], gold["clique4"], gold["clique5"]]
    G.close()


def _sample_ranges(n, seed, count=4, width=1500):
    rng = np.random.default_rng(seed)
    starts = sorted(rng.integers(0, n - width, size=count).tolist())
    return [(s, s + width) for s in starts] + [(n - 7, n)]


def test_fullsize_cliques_rmat21(gpm):
    g = gg.workload_clique_rmat21()
    gold = _golden().get("clique_rmat21", {})
    G = gpm.Graph.from_host(g)
    pats = [gpm.Pattern.clique(k) for k in (3, 4, 5)]
    for lo, hi in _sample_ranges(g.n, 2, count=3, width=600):
        assert gpm.count_roots(G, pats, lo, hi) == [O.cliques(g, k, lo, hi) for k in (3, 4, 5)], (lo, hi)
    # the heaviest roots (largest out-degree, CTA class) are checked one by one
    od = O.out_degrees(g)
    for v in np.argsort(od)[-3:].tolist():
        assert gpm.count_roots(G, pats[:2], v, v + 1) == [O.cliques(g, k, v, v + 1) for k in (3, 4)], v
    v = int(np.argmax(od))
    assert gpm.count_roots(G, pats[2:], v, v + 1) == [O.cliques(g, 5, v, v + 1)], v
    got = gpm.count(G, pats)
    if gold:
        assert gold["digest"] == g.digest()
        for k, c in zip((3, 4, 5), got):
            if f"clique{k}" in gold:
                assert c == gold[f"clique{k}"], k
    G.close()


def test_fullsize_clique6_rmat20(gpm):
    # the 6-clique workload in the launch configuration bench.py times: sampled
    # root ranges and the lightest root of the 1024-thread class against the
    # oracle; the total against a partition of the roots and the 5-clique total
    # against the k <= 5 pass
    g = gg.workload_clique6_rmat20()
    G = gpm.Graph.from_host(g)
    K6 = gpm.Pattern.clique(6)
    for lo, hi in _sample_ranges(g.n, 7, count=3, width=40):
        assert gpm.count_roots(G, [K6], lo, hi) == [O.cliques(g, 6, lo, hi)], (lo, hi)
    od = O.out_degrees(g)
    hi_class = np.nonzero(od > 384)[0]
    v = int(hi_class[np.argmin(od[hi_class])])
    assert gpm.count_roots(G, [K6], v, v + 1) == [O.cliques(g, 6, v, v + 1)], v
    tot = gpm.count(G, [gpm.Pattern.clique(5), K6])
    cuts = [0, 1, g.n // 3, g.n // 3 + 1, g.n - 5, g.n]
    assert sum(gpm.count_roots(G, [K6], lo, hi)[0] for lo, hi in zip(cuts[:-1], cuts[1:])) == tot[1]
    assert gpm.count(G, [gpm.Pattern.clique(4), gpm.Pattern.clique(5)])[1] == tot[0]
    G.close()


def test_fullsize_clique789_chunglu1m(gpm):
    # the k = 7..9 workload as bench.py counts it (gpm_count_cliques): a root
    # range, the ragged tail, the lightest root of the 129..384 out-degree class
    # and the heaviest root against the oracle; the total against a partition
    g = gg.workload_clique789_chung_lu1m()
    G = gpm.Graph.from_host(g)
    od = O.out_degrees(g)
    lo_class = np.nonzero(od > 128)[0]
    v_lo = int(lo_class[np.argmin(od[lo_class])])
    v_max = int(np.argmax(od))
    for lo, hi in [(0, 600), (g.n - 7, g.n), (v_lo, v_lo + 1), (v_max, v_max + 1)]:
        assert [gpm.count_cliques(G, k, lo, hi) for k in (7, 8, 9)] == [O.cliques(g, k, lo, hi) for k in (7, 8, 9)], \
            (lo, hi)
    cuts = [0, g.n // 2, g.n // 2 + 1, g.n]
    for k in (7, 9):
        assert sum(gpm.count_cliques(G, k, a, b) for a, b in zip(cuts[:-1], cuts[1:])) == gpm.count_cliques(G, k)
    # the totals against the oracle's (tests/golden/make_golden.py)
    gold = _golden().get("clique789_chunglu1m", {})
    if gold:
        assert gold["digest"] == g.digest()
        for k in (7, 8, 9):
            if f"clique{k}" in gold:
                assert gpm.count_cliques(G, k) == gold[f"clique{k}"], k
    G.close()


def test_fullsize_sl_chunglu4m(gpm):
    g = gg.workload_sl_chung_lu4m()
    gold = _golden().get("sl_chunglu4m", {})
    G = gpm.Graph.from_host(g)
    D = gpm.Pattern.spec(O.DIAMOND, induced=False)
    C = gpm.Pattern.spec(O.CYCLE4, induced=False)
    for lo, hi in _sample_ranges(g.n, 3, width=4000):
        assert gpm.count_roots(G, [D, C], lo, hi) == [O.diamonds(g, lo, hi), O.cycles4(g, lo, hi)], (lo, hi)
    got = gpm.count(G, [D, C])
    if gold:
        assert gold["digest"] == g.digest()
        if "diamond" in gold:
            assert got[0] == gold["diamond"]
        if "cycle4" in gold:
            assert got[1] == gold["cycle4"]
    for P, adj in ((D, O.DIAMOND), (C, O.CYCLE4)):
        tuples, total = gpm.list_embeddings(G, P, cap=1_000_000)
        assert len(tuples) == min(total, 1_000_000)
        # every written tuple valid, all distinct subgraphs
        _check_tuples_all(g, adj, P.info(), tuples)
    G.close()


def test_fullsize_motif4_batch_rmat20(gpm):
    # the largest R-MAT graph of the batched workload's 4-motif queries
    # (scale 20): all six induced 4-vertex motif counts equal the oracle's,
    # stored by tests/golden/make_golden.py, through local counting and
    # through the batched form's plain-path equivalent
    import importlib.util
    gold = _golden().get("motif4_batch_rmat20")
    if not gold:
        pytest.skip("no stored oracle counts for this graph")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(os.path.dirname(GOLDEN), "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    g = gg.graph_from_spec(mg._largest_batch_motif4_rmat())
    assert gold["digest"] == g.digest()
    G = gpm.Graph.from_host(g)
    assert gpm.count(G, gpm.Pattern.motifs(4)) == gold["motifs4"]
    G.close()


def test_complete_graph_every_class(gpm):
    # K_1100 in degree order (ties by id): out-degrees 0..1099 cover every root
    # class, including the 1024-thread shared-memory class at its largest
    # (out-degree 1024, where the one-warp rows fall back to 64 candidates) and
    # the global-memory class above it. Closed forms C(n, k).
    import math
    n = 1100
    g = gg.complete(n)
    G = gpm.Graph.from_host(g)
    info = G.prepare().info()
    assert info["max_out_degree"] == n - 1
    got = gpm.count(G, [gpm.Pattern.clique(k) for k in (3, 4, 5)])
    assert got == [math.comb(n, 3), math.comb(n, 4), math.comb(n, 5)]
    # root ranges: the roots with out-degree in (384, 1024] alone
    lo, hi = n - 1 - 1024, n - 1 - 384
    got = gpm.count_roots(G, [gpm.Pattern.clique(5)], lo, hi)
    assert got == [sum(math.comb(n - 1 - v, 4) for v in range(lo, hi))]
    G.close()


@pytest.mark.parametrize("opts", [dict(), dict(warp_max_degree=32, cta_max_degree=32),
                                  dict(warp_max_degree=32, cta_max_degree=96)])
def test_six_cliques_every_root_class(gpm, opts):
    # the 6-clique level in every root class: warp rows, CTA nested rows
    # (register, warp, group and CTA-wide paths) and global-memory bitmaps;
    # closed forms on complete and complete multipartite graphs, the oracle elsewhere
    import math
    old = gpm.get_options()
    try:
        if opts:
            gpm.set_options(**opts)
        K6 = gpm.Pattern.clique(6)
        for n in (7, 40, 160):
            G = gpm.Graph.from_host(gg.complete(n))
            assert gpm.count(G, [K6]) == [math.comb(n, 6)], n
            G.close()
        parts = [5, 9, 3, 12, 7, 4, 6]
        G = gpm.Graph.from_host(gg.complete_multipartite(parts))
        e6 = sum(math.prod(c) for c in __import__("itertools").combinations(parts, 6))
        assert gpm.count(G, [K6]) == [e6]
        G.close()
        for g in [gg.rmat(11, 16.0, seed=21), gg.chung_lu(5000, 16.0, 2.1, seed=24), gg.rmat(12, 16.0, seed=31)]:
            G = gpm.Graph.from_host(g)
            assert gpm.count(G, [K6, gpm.Pattern.clique(5)]) == [O.cliques(g, 6), O.cliques(g, 5)], g.name
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def _hub_graph(nb=420, nc=430, p=0.1, planted=(10, 9), seed=5):
    """Vertex a and an independent set C joined completely to B (B has its own
    sparse edges and planted cliques): a and every vertex of C are roots with
    out-degree |B| = 420 (the 1024-thread CTA class), whose local graph is B."""
    rng = np.random.default_rng(seed)
    B = np.arange(1, 1 + nb)
    C = np.arange(1 + nb, 1 + nb + nc)
    e = [(0, int(b)) for b in B] + [(int(b), int(c)) for b in B for c in C]
    iu = np.triu_indices(nb, 1)
    keep = rng.random(len(iu[0])) < p
    e += [(int(B[i]), int(B[j])) for i, j in zip(iu[0][keep], iu[1][keep])]
    perm = rng.permutation(nb)
    off = 0
    for s in planted:
        vs = B[perm[off:off + s]]
        off += s
        e += [(int(vs[i]), int(vs[j])) for i in range(s) for j in range(i + 1, s)]
    return gg.from_edges(1 + nb + nc, e, name="hub")


@pytest.mark.parametrize("opts", [dict(), dict(warp_max_degree=32, cta_max_degree=32),
                                  dict(warp_max_degree=32, cta_max_degree=96),
                                  dict(warp_max_degree=256, cta_max_degree=1024)])
def test_large_k_cliques_every_root_class(gpm, opts):
    # k = 7..9 by the generic search in every root class (warp, CTA in shared
    # memory, CTA with global-memory bitmaps): closed forms on complete and
    # complete multipartite graphs, the oracle elsewhere
    import itertools
    import math
    old = gpm.get_options()
    try:
        if opts:
            gpm.set_options(**opts)
        for n in (9, 33, 40):
            G = gpm.Graph.from_host(gg.complete(n))
            assert [gpm.count_cliques(G, k) for k in (7, 8, 9)] == [math.comb(n, k) for k in (7, 8, 9)], n
            assert gpm.count(G, [gpm.Pattern.clique(7), gpm.Pattern.clique(8)]) == [math.comb(n, 7), math.comb(n, 8)]
            G.close()
        parts = [3, 2, 4, 1, 3, 2, 5, 3, 1, 2]
        G = gpm.Graph.from_host(gg.complete_multipartite(parts))
        want = [sum(math.prod(c) for c in itertools.combinations(parts, k)) for k in (7, 8, 9)]
        assert [gpm.count_cliques(G, k) for k in (7, 8, 9)] == want
        G.close()
        for g in [_hub_graph(), gg.rmat(10, 16.0, seed=21), gg.rmat(12, 8.0, seed=22),
                  gg.chung_lu(5000, 16.0, 2.1, seed=24)]:
            G = gpm.Graph.from_host(g)
            assert [gpm.count_cliques(G, k) for k in (7, 8, 9)] == [O.cliques(g, k) for k in (7, 8, 9)], g.name
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def _bipartite_with_planted_clique(na, nb, q):
    """Complete bipartite A x B (A = 0..na-1, B = na..na+nb-1) plus a clique on
    the last q vertices of B, as a symmetric sorted CSR: a k-clique holds at
    most one vertex of A and a clique of B, so there are C(q, k) + na C(q, k-1)
    of them (k >= 3). Every vertex of A has the whole of B as out-neighbours in
    the degree order (equal degrees, larger ids)."""
    n = na + nb
    planted = np.arange(n - q, n)
    rows = []
    for v in range(na):
        rows.append(np.arange(na, n, dtype=np.uint32))
    for v in range(na, n):
        r = np.arange(0, na, dtype=np.uint32)
        if v >= n - q:
            r = np.concatenate([r, planted[planted != v].astype(np.uint32)])
        rows.append(r)
    rowptr = np.zeros(n + 1, dtype=np.uint64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    return rowptr, np.concatenate(rows).astype(np.uint32), n


def test_large_k_cliques_outdegree_above_4096(gpm):
    # roots of out-degree 4130 (local-graph rows of 130 words): the generic
    # search with 16 words of a candidate set per lane; closed form
    import math
    import torch
    na, nb, q = 4130, 4130, 8
    rowptr, col, n = _bipartite_with_planted_clique(na, nb, q)
    G = gpm.Graph(torch.from_numpy(rowptr.view(np.int64)), torch.from_numpy(col.view(np.int32)), n)
    for k in (7, 8, 9):
        assert gpm.count_cliques(G, k) == math.comb(q, k) + na * math.comb(q, k - 1), k
    assert G.info()["max_out_degree"] == nb + q - 1 or G.info()["max_out_degree"] > 4096
    G.close()


def test_count_cliques_ranges_and_small_k(gpm):
    # gpm_count_cliques: root ranges partition the total; k = 3..6 agree with
    # the fused pass; a mixed call (k <= 6 and k >= 7 patterns) fills both
    g = gg.rmat(12, 8.0, seed=22)
    G = gpm.Graph.from_host(g)
    cuts = [0, 1, 1000, 2047, 2048, 3000, g.n]
    for k in (7, 9):
        parts = [gpm.count_cliques(G, k, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
        assert parts == [O.cliques(g, k, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])], k
        assert sum(parts) == gpm.count_cliques(G, k)
    assert [gpm.count_cliques(G, k) for k in (3, 4, 5, 6)] == [O.cliques(g, k) for k in (3, 4, 5, 6)]
    mixed = [gpm.Pattern.clique(4), gpm.Pattern.clique(8), gpm.Pattern.spec(O.CYCLE4, induced=False),
             gpm.Pattern.clique(7), gpm.Pattern.clique(3)]
    assert gpm.count(G, mixed) == [O.cliques(g, 4), O.cliques(g, 8), O.cycles4(g), O.cliques(g, 7), O.cliques(g, 3)]
    assert gpm.count_roots(G, mixed[:2], 100, 2500) == [O.cliques(g, 4, 100, 2500), O.cliques(g, 8, 100, 2500)]
    for bad in (0, 2, 10):
        with pytest.raises(gpm.GpmError):
            gpm.count_cliques(G, bad)
    with pytest.raises(gpm.GpmError):
        gpm.count_cliques(G, 7, 5, 3)
    G.close()


def test_listing_deep_cliques_dense(gpm):
    # k = 6..8 listing on graphs dense enough to hold many of them: complete
    # graphs (C(n, k) tuples), a complete multipartite graph and a dense G(n, p)
    for g in [gg.complete(12), gg.complete_multipartite([2, 3, 1, 2, 2, 1, 3, 2, 1]), gg.random_small(20, 0.7, 23)]:
        G = gpm.Graph.from_host(g)
        for k in (6, 7, 8):
            adj = O.clique_pattern(k)
            P = gpm.Pattern.spec(adj, induced=True)
            want = O.cliques(g, k)  # distinct valid cliques, as many as the oracle counts: all of them
            tuples, total = gpm.list_embeddings(G, P, cap=want + 3)
            assert total == want == len(tuples), (g.name, k)
            assert len(_check_tuples(g, adj, P.info(), tuples)) == want
            if total > 1:
                part, total2 = gpm.list_embeddings(G, P, cap=total // 2)
                assert total2 == total and len(part) == total // 2
                _check_tuples(g, adj, P.info(), part)
        G.close()


def test_exists_matches_oracle_counts(gpm):
    # the existence query (early exit at the first match): found exactly when
    # the oracle's count is non-zero; the witness is an embedding of the pattern
    graphs = SMALL[:8] + SMALL[12:20] + [gg.path(9), gg.star(7), gg.cycle(7), gg.complete_multipartite([3, 3, 3]),
                                         gg.rmat(10, 16.0, seed=21), gg.chung_lu(5000, 16.0, 2.1, seed=24)]
    pats = [(O.clique_pattern(k), True) for k in range(3, 9)] + LIST_PATTERNS[:4]
    for g in graphs:
        G = gpm.Graph.from_host(g)
        for adj, induced in pats:
            P = gpm.Pattern.spec(adj, induced=induced)
            k = adj.shape[0]
            nedges = int(np.triu(adj).sum())
            want = O.cliques(g, k) if induced else (O.diamonds(g) if nedges == 5 else O.cycles4(g))
            found, w = gpm.exists(G, P)
            assert found == (want > 0), (g.name, k)
            if found:
                assert len(set(w.tolist())) == k
                for i in range(k):
                    for j in range(i + 1, k):
                        if adj[i, j]:
                            assert _adjacent(g, w[i], w[j]), (g.name, w, i, j)
        G.close()


def _keyed_out_degrees(g, key):
    d = np.diff(g.rowptr).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), d)
    dst = g.col.astype(np.int64)
    c = key.astype(np.int64)
    keep = (c[src] < c[dst]) | ((c[src] == c[dst]) & (src < dst))
    return np.bincount(src[keep], minlength=g.n)


@pytest.mark.parametrize("opts", [dict(), dict(warp_max_degree=32, cta_max_degree=96)])
def test_core_numbers_and_core_orientation(gpm, opts):
    # the k-core peel against the oracle's bucket-queue core numbers; under the
    # core value based (degeneracy) order the totals are those of the degree
    # order, the root ranges follow (peel round, id) and no vertex has more
    # successors than its core number; switching back restores the degree order
    old = gpm.get_options()
    try:
        if opts:
            gpm.set_options(**opts)
        K = [gpm.Pattern.clique(k) for k in (3, 4, 5, 6)]
        for g in SMALL[:8] + _medium() + [gg.complete(40), gg.empty(5), gg.star(9)]:
            G = gpm.Graph.from_host(g)
            core = O.core_numbers(g)
            order = O.core_order(g)
            assert G.core_numbers().tolist() == core.tolist(), g.name
            G.set_orientation("core")
            info = G.prepare().info()
            assert info["dag_arcs"] == g.m
            assert info["max_out_degree"] == (int(_keyed_out_degrees(g, order).max()) if g.n else 0), g.name
            assert info["max_out_degree"] <= (int(core.max()) if g.n else 0)
            assert G.core_numbers().tolist() == core.tolist()
            assert gpm.count(G, K) == [O.cliques(g, k) for k in (3, 4, 5, 6)], g.name
            assert gpm.count_cliques(G, 7) == O.cliques(g, 7), g.name
            assert gpm.count(G, gpm.Pattern.motifs(4)) == O.motifs(g, 4), g.name
            cuts = [0, g.n // 3, g.n // 3 + 1, g.n]
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                assert gpm.count_roots(G, K[1:3], lo, hi) == [O.cliques_keyed(g, order, k, lo, hi) for k in (4, 5)], \
                    (g.name, lo, hi)
                assert gpm.count_cliques(G, 7, lo, hi) == O.cliques_keyed(g, order, 7, lo, hi), (g.name, lo, hi)
            G.set_orientation("degree")
            assert gpm.count_roots(G, K[1:2], 0, g.n // 3) == [O.cliques(g, 4, 0, g.n // 3)]
            G.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def test_core_orientation_fullsize_rmat21(gpm):
    # the headline graph under the core order: core numbers against the
    # oracle, 4- and 5-clique totals against the stored oracle totals
    g = gg.workload_clique_rmat21()
    gold = _golden().get("clique_rmat21", {})
    G = gpm.Graph.from_host(g)
    core = O.core_numbers(g)
    assert G.core_numbers().tolist() == core.tolist()
    G.set_orientation("core")
    got = gpm.count(G, [gpm.Pattern.clique(4), gpm.Pattern.clique(5)])
    assert G.info()["max_out_degree"] == int(_keyed_out_degrees(g, O.core_order(g)).max()) <= int(core.max())
    if gold:
        assert gold["digest"] == g.digest()
        assert got == [gold["clique4"], gold["clique5"]]
    G.set_orientation("degree")
    assert gpm.count(G, [gpm.Pattern.clique(4), gpm.Pattern.clique(5)]) == got
    G.close()


def test_counts_past_64_bits_are_reported(gpm):
    # K_{5, 3,000,000}: five hubs of degree 3,000,000. Each C(d, 3) fits in 64
    # bits (d(d-1)(d-2) does not), but the edge-induced 3-star count
    # 5 C(3e6, 3) + 3e6 C(5, 3) ~ 2.25e19 does not: the count reports
    # GPM_E_OVERFLOW instead of a wrapped value; counts below 2^64 on the same
    # graph stay exact (closed forms)
    import math
    a, b = 5, 3_000_000
    e = np.stack([np.repeat(np.arange(a), b), a + np.tile(np.arange(b), a)], 1)
    g = gg.from_edges(a + b, e, name="K_5_3M")
    G = gpm.Graph.from_host(g)
    star = gpm.Pattern.spec(O.pattern(4, [(0, 1), (0, 2), (0, 3)]), induced=False)
    with pytest.raises(gpm.GpmError) as err:
        gpm.count(G, [star])
    assert err.value.name == "OVERFLOW"
    C4 = gpm.Pattern.spec(O.CYCLE4, induced=False)
    wedge = gpm.Pattern.spec(O.pattern(3, [(0, 1), (1, 2)]), induced=False)
    assert gpm.count(G, [C4, wedge, gpm.Pattern.clique(3)]) == [
        math.comb(a, 2) * math.comb(b, 2), a * math.comb(b, 2) + b * math.comb(a, 2), 0]
    G.close()
