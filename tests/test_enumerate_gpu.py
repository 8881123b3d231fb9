"""Pattern-oblivious enumeration with connectivity codes (gpm_count_enumerate,
and gpm_count on 5-vertex patterns) against the CPU oracle, through the C-ABI.

Induced 5-vertex motif counts are compared class by class with the oracle's
ESU enumeration (itself pinned by the networkx atlas, closed forms and subset
brute force); the 3- and 4-vertex counts of the enumeration are compared with
the local-counting path and the oracle (an independent check of local
counting); edge-induced 5-vertex patterns with the oracle's brute force.
All counts are integers: the bar is equality.
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


SMALL = [
    gg.complete(5), gg.complete(8), gg.complete_multipartite([2, 3, 4]), gg.complete_multipartite([1, 4]),
    gg.petersen(), gg.cycle(5), gg.cycle(9), gg.star(7), gg.path(6), gg.empty(5),
    gg.from_edges(4, [(0, 1), (1, 2), (2, 3)]),
] + [gg.random_small(n, p, s) for s, (n, p) in enumerate(
    [(10, 0.5), (14, 0.4), (18, 0.35), (22, 0.3), (25, 0.25), (28, 0.2), (30, 0.3), (16, 0.8), (24, 0.15)])] \
    + [gg.rmat(5, 6.0, seed=s) for s in range(3)]

# 5-vertex patterns (edge lists): 4-path, 5-cycle, house, bull, star, kite,
# cricket, K5 minus an edge, wheel W4, K_{2,3}
PAT5 = [
    [(0, 1), (1, 2), (2, 3), (3, 4)],
    [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)],
    [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)],
    [(0, 1), (1, 2), (2, 0), (0, 3), (1, 4)],
    [(0, 1), (0, 2), (0, 3), (0, 4)],
    [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (3, 4)],
    [(0, 1), (0, 2), (1, 2), (0, 3), (0, 4)],
    [(a, b) for a in range(5) for b in range(a + 1, 5) if (a, b) != (3, 4)],
    [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 3), (3, 4), (4, 1)],
    [(a, b) for a in (0, 1) for b in (2, 3, 4)],
]


def _adj5(mask):
    """Adjacency of a 5-vertex pair mask: bit b for the b-th pair of (0,1), (0,2), ..., (3,4)."""
    a = np.zeros((5, 5), np.uint8)
    b = 0
    for i in range(5):
        for j in range(i + 1, 5):
            if mask >> b & 1:
                a[i, j] = a[j, i] = 1
            b += 1
    return a


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_motifs5_small_every_class(gpm, gi):
    g = SMALL[gi]
    want, masks = O.motifs5(g)
    G = gpm.Graph.from_host(g)
    M = gpm.Pattern.motifs(5)
    assert len(M) == 21
    assert gpm.count(G, M[:16]) == want[:16]  # at most 16 patterns per call
    assert gpm.count(G, M[16:]) == want[16:]
    assert gpm.count_enumerate(G, M[:16]) == want[:16]
    # each class found from its own adjacency (independent of the class order)
    for c, m in enumerate(masks):
        P = gpm.Pattern.spec(_adj5(m), induced=True)
        assert P.info()["motif_index"] == c
        assert gpm.count(G, [P]) == [want[c]], (g.name, c)
    G.close()


def _medium5():
    return [gg.erdos_renyi(1500, 0.006, seed=41, permute=True), gg.chung_lu(1500, 5.0, 2.7, seed=42),
            gg.rmat(8, 4.0, seed=43), gg.erdos_renyi(2500, 0.0024, seed=44, permute=True)]


@pytest.mark.parametrize("gi", range(4))
def test_motifs5_medium(gpm, gi):
    g = _medium5()[gi]
    want, _ = O.motifs5(g)
    G = gpm.Graph.from_host(g)
    M = gpm.Pattern.motifs(5)
    got = gpm.count(G, M[:11]) + gpm.count(G, M[11:])
    assert got == want, g.name
    # root ranges partition the total. Root: the smallest vertex for the
    # enumerated classes; the 5-clique (class 20) is counted by the clique
    # path, whose root is its first vertex in the orientation order
    cuts = [0, 1, g.n // 3, g.n // 3 + 1, g.n - 7, g.n]
    acc = [0] * 21
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        part = gpm.count_roots(G, M[:11], lo, hi) + gpm.count_roots(G, M[11:], lo, hi)
        assert part == O.motifs5(g, lo, hi)[0][:20] + [O.cliques(g, 5, lo, hi)], (g.name, lo, hi)
        acc = [x + y for x, y in zip(acc, part)]
    assert acc == want
    G.close()


def _medium34():
    return [gg.rmat(10, 8.0, seed=21), gg.erdos_renyi(3000, 0.004, seed=23, permute=True),
            gg.chung_lu(4000, 8.0, 2.1, seed=24), gg.from_edges(3, [(0, 1), (1, 2)])]


@pytest.mark.parametrize("k", [3, 4])
def test_enumeration_checks_local_counting(gpm, k):
    # the enumeration's 3- and 4-vertex counts equal local counting's and the
    # oracle's, induced and edge-induced
    pats = O.MOTIF3_PATTERNS if k == 3 else O.MOTIF4_PATTERNS
    for g in _medium34() + SMALL[:8]:
        G = gpm.Graph.from_host(g)
        M = gpm.Pattern.motifs(k)
        want = O.motifs(g, k)
        assert gpm.count_enumerate(G, M) == want, g.name
        assert gpm.count(G, M) == want, g.name
        ni = [gpm.Pattern.spec(p, induced=False) for p in pats]
        assert gpm.count_enumerate(G, ni) == O.noninduced_terms(g, k), g.name
        G.close()


def test_noninduced_five_vertex_patterns(gpm):
    for g in SMALL:
        G = gpm.Graph.from_host(g)
        pats = [O.pattern(5, es) for es in PAT5]
        ni = [gpm.Pattern.spec(p, induced=False) for p in pats]
        ind = [gpm.Pattern.spec(p, induced=True) for p in pats]
        assert gpm.count(G, ni) == [O.bf_noninduced(g, p) for p in pats], g.name
        assert gpm.count(G, ind) == [O.bf_induced(g, p) for p in pats], g.name
        G.close()


def test_enumeration_rejects(gpm):
    G = gpm.Graph.from_host(gg.complete(6))
    with pytest.raises(gpm.GpmError):
        gpm.count_enumerate(G, [gpm.Pattern.motifs(3)[0], gpm.Pattern.motifs(4)[0]])
    with pytest.raises(gpm.GpmError):
        gpm.count_enumerate(G, [gpm.Pattern.clique(6)])
    # the 5-clique through the enumeration equals C(6, 5)
    assert gpm.count_enumerate(G, [gpm.Pattern.clique(5)]) == [6]
    G.close()


def test_motif5_fullsize_sampled(gpm):
    # the 5-motif workload (Erdos-Renyi 2^20 vertices, mean degree 8): root
    # ranges the oracle counts in seconds, and a partition of the roots whose
    # parts add up to the total
    g = gg.workload_motif5_er1m()
    G = gpm.Graph.from_host(g)
    M = gpm.Pattern.motifs(5)
    for lo, hi in [(0, 120), (g.n // 2, g.n // 2 + 400), (g.n - 600, g.n)]:
        # 5-cliques (class 20) are rooted by the clique path's convention
        want = O.motifs5(g, lo, hi)[0][:20] + [O.cliques(g, 5, lo, hi)]
        assert gpm.count_roots(G, M, lo, hi) == want, (lo, hi)
    total = gpm.count(G, M)
    cuts = [0, 12345, g.n // 2, g.n - 1, g.n]
    parts = [gpm.count_roots(G, M, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:])]
    assert [sum(c) for c in zip(*parts)] == total
    assert sum(total) > 4 * 10 ** 9
    G.close()
