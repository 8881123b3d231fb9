"""Pattern-guided search (gpm_count_guided; gpm_count on 6..8-vertex patterns;
gpm_list and gpm_exists on every pattern without a dedicated kernel) against
the CPU oracle, through the C-ABI.

Counts of patterns with 3..8 vertices, induced and edge-induced, equal the
oracle's brute force on graphs of at most 30 vertices; listings equal the
oracle's set of distinct subgraphs; on medium graphs the guided counts equal
the library's other, independently pinned paths (local counting, the
pattern-oblivious enumeration, the clique search). Integers: equality.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_03135_b300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_03135_b300 import gpm as m
    return m


# edge lists: 4-path, 5-cycle, house, bull, star K_{1,4}, kite, 6-cycle,
# two triangles joined by an edge, tailed triangle, wedge, triangle, 4-clique,
# 7-cycle with a chord, 8-vertex "cube", 6-vertex wheel W5, K_{3,3}
PATTERNS = [
    [(0, 1), (1, 2), (2, 3), (3, 4)],
    [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)],
    [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)],
    [(0, 1), (1, 2), (2, 0), (0, 3), (1, 4)],
    [(0, 1), (0, 2), (0, 3), (0, 4)],
    [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (3, 4)],
    [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0)],
    [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3)],
    [(0, 1), (0, 2), (0, 3), (1, 2)],
    [(0, 1), (1, 2)],
    [(0, 1), (1, 2), (0, 2)],
    [(a, b) for a in range(4) for b in range(a + 1, 4)],
    [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6), (6, 0), (0, 3)],
    [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7)],
    [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (1, 2), (2, 3), (3, 4), (4, 5), (5, 1)],
    [(a, b) for a in (0, 1, 2) for b in (3, 4, 5)],
]


def _pat(es):
    return O.pattern(max(max(e) for e in es) + 1, es)


# brute force over injective maps: every pattern on graphs of up to 16
# vertices, patterns of up to 6 vertices on the 20-vertex graphs
SMALL = [gg.complete(7), gg.complete_multipartite([2, 3, 3]), gg.petersen(), gg.cycle(8), gg.star(6),
         gg.path(7), gg.empty(4)] + [gg.random_small(n, p, s) for s, (n, p) in enumerate(
             [(10, 0.5), (12, 0.45), (14, 0.35), (16, 0.3), (20, 0.25), (13, 0.6)])] \
    + [gg.rmat(4, 4.0, seed=s) for s in range(2)] + [gg.rmat(5, 3.0, seed=2)]


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_guided_counts_small_graphs(gpm, gi):
    g = SMALL[gi]
    G = gpm.Graph.from_host(g)
    pats = [_pat(es) for es in PATTERNS if g.n <= 16 or max(max(e) for e in es) + 1 <= 6]
    for ind in (True, False):
        P = [gpm.Pattern.spec(p, induced=ind) for p in pats]
        want = [O.bf_induced(g, p) if ind else O.bf_noninduced(g, p) for p in pats]
        assert gpm.count_guided(G, P) == want, (g.name, ind)
        assert gpm.count(G, P) == want, (g.name, ind)  # every path gpm_count picks
    G.close()


def _edge_set(es, t):
    return frozenset((min(t[a], t[b]), max(t[a], t[b])) for a, b in es)


@pytest.mark.parametrize("gi", [1, 2, 7, 8, 9, 12])
def test_guided_listing_small_graphs(gpm, gi):
    # every distinct edge-induced subgraph listed once (as the oracle's set of
    # edge sets); a capped listing writes valid, distinct matches; existence
    g = SMALL[gi]
    G = gpm.Graph.from_host(g)
    for es in PATTERNS[:8] + PATTERNS[12:]:
        p = _pat(es)
        P = gpm.Pattern.spec(p, induced=False)
        want = O.bf_subgraph_set(g, p)
        tuples, total = gpm.list_embeddings(G, P, cap=len(want) + 5)
        assert total == len(want) and len(tuples) == total, (g.name, es)
        got = {_edge_set(es, t) for t in tuples}
        assert got == want, (g.name, es)
        if total > 3:
            part, total2 = gpm.list_embeddings(G, P, cap=3)
            assert total2 == total and len(part) == 3
            assert len({_edge_set(es, t) for t in part}) == 3 and {_edge_set(es, t) for t in part} <= want
        found, w = gpm.exists(G, P)
        assert found == (total > 0)
        if found:
            assert _edge_set(es, w) in want
        # induced: every listed tuple is an induced copy (non-edges stay non-edges)
        Pi = gpm.Pattern.spec(p, induced=True)
        ti, tot_i = gpm.list_embeddings(G, Pi, cap=10 ** 5)
        assert tot_i == O.bf_induced(g, p) and len(ti) == tot_i
        k = p.shape[0]
        for t in ti:
            for a in range(k):
                for b in range(a + 1, k):
                    nb = g.neighbors(int(t[a]))
                    adj = np.searchsorted(nb, t[b]) < len(nb) and nb[np.searchsorted(nb, t[b])] == t[b]
                    assert bool(adj) == bool(p[a, b]), (g.name, es, t)
        assert len({tuple(t) for t in ti}) == len(ti)
    G.close()


def _medium():
    return [gg.rmat(10, 8.0, seed=21), gg.erdos_renyi(3000, 0.003, seed=23, permute=True),
            gg.chung_lu(3000, 6.0, 2.5, seed=24)]


def test_guided_matches_other_paths_medium(gpm):
    # 3- and 4-vertex patterns: local counting; 5-vertex: the enumeration;
    # cliques: the clique search -- all independent of the guided search
    for g in _medium():
        G = gpm.Graph.from_host(g)
        for k in (3, 4):
            for ind in (True, False):
                P = [gpm.Pattern.spec(p, induced=ind) for p in (O.MOTIF3_PATTERNS if k == 3 else O.MOTIF4_PATTERNS)]
                assert gpm.count_guided(G, P) == gpm.count(G, P), (g.name, k, ind)
        five = [gpm.Pattern.spec(_pat(es), induced=ind) for es in PATTERNS[:6] for ind in (True, False)]
        assert gpm.count_guided(G, five) == gpm.count_enumerate(G, five), g.name
        cl = [gpm.Pattern.clique(k) for k in (4, 5, 6)]
        assert gpm.count_guided(G, cl) == [O.cliques(g, k) for k in (4, 5, 6)], g.name
        G.close()


def test_guided_rejects(gpm):
    G = gpm.Graph.from_host(gg.complete(5))
    with pytest.raises(gpm.GpmError):
        gpm.count_guided(G, [gpm.Pattern.clique(2)])
    with pytest.raises(gpm.GpmError):  # root ranges are not defined for the guided search
        gpm.count_roots(G, [gpm.Pattern.spec(_pat(PATTERNS[6]), induced=False)], 0, 3)
    G.close()


def test_guided_fullsize_er1m(gpm):
    # the guided bench workload (Erdos-Renyi 2^20 vertices, mean degree 8):
    # the 5-vertex path through the guided search equals the enumeration's
    # count (an independent path, pinned to the oracle on sampled root ranges
    # of this graph); the 6-cycle count does not depend on the pattern's
    # numbering (another matching order and other symmetry-breaking bounds)
    g = gg.workload_motif5_er1m()
    G = gpm.Graph.from_host(g)
    p5 = gpm.Pattern.spec(_pat(PATTERNS[0]), induced=False)
    want = gpm.count_enumerate(G, [p5])
    assert gpm.count_guided(G, [p5]) == want and want[0] > 10 ** 9
    c6a = gpm.Pattern.spec(_pat([(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0)]), induced=False)
    c6b = gpm.Pattern.spec(_pat([(3, 0), (0, 5), (5, 1), (1, 4), (4, 2), (2, 3)]), induced=False)
    assert c6a.info()["matching_order"] != c6b.info()["matching_order"] or \
        c6a.info()["sb_pairs"] != c6b.info()["sb_pairs"]
    a, b = gpm.count_guided(G, [c6a, c6b])
    assert a == b and a > 0
    G.close()
