"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expected value is a
closed form, a textbook count, a library routine (scipy sparse products), a
brute-force enumeration written independently in this file, or a worked
example printed in the paper (tests/golden/*.json, each with its citation).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2011_03135_b300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sym(n, edges):
    return gg.from_edges(n, edges)


def _esym(ks, k):
    """elementary symmetric polynomial e_k(ks)"""
    return sum(math.prod(c) for c in itertools.combinations(ks, k))


def _py_adj(g):
    return [set(int(x) for x in g.neighbors(v)) for v in range(g.n)]


SMALL = [
    lambda: gg.random_small(18, 0.45, 11),
    lambda: gg.random_small(24, 0.3, 12),
    lambda: gg.random_small(28, 0.2, 13),
    lambda: gg.rmat(5, 4.0, seed=14),
    lambda: gg.petersen(),
    lambda: gg.complete_multipartite([1, 2, 3, 3]),
]


# ---------------- k-cliques ----------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 8, 11])
@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8, 9])
def test_cliques_complete_graph(n, k):
    g = gg.complete(n) if n > 0 else gg.empty(0)
    assert O.cliques(g, k) == math.comb(n, k)


@pytest.mark.parametrize("parts", [[2, 3], [1, 1, 1, 1], [2, 2, 2], [3, 1, 4, 2], [5, 5, 1], [2, 1, 3, 1, 2, 2, 1],
                                   [1, 2, 1, 3, 1, 2, 1, 1, 2, 1]])
@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8, 9])
def test_cliques_complete_multipartite(parts, k):
    g = gg.complete_multipartite(parts)
    assert O.cliques(g, k) == _esym(parts, k)


@pytest.mark.parametrize("g", [gg.path(9), gg.star(7), gg.empty(5), gg.cycle(7),
                               gg.from_edges(8, [(0, 1), (1, 2), (1, 3), (3, 4), (4, 5), (4, 6), (6, 7)])])
def test_cliques_trees_and_cycles_have_none(g):
    for k in (3, 4, 5, 6):
        assert O.cliques(g, k) == 0


def test_triangles_trace_identity_small_and_rmat14():
    for g in [gg.random_small(30, 0.3, 3), gg.rmat(10, 8.0, seed=5), gg.workload_tc_rmat14()]:
        e = g.edges()
        A = sp.coo_matrix((np.ones(2 * len(e), dtype=np.int64),
                           (np.r_[e[:, 0], e[:, 1]], np.r_[e[:, 1], e[:, 0]])), shape=(g.n, g.n)).tocsr()
        A2 = A @ A
        tr = int(A.multiply(A2).sum())
        assert tr % 6 == 0
        assert O.triangles(g) == tr // 6


@pytest.mark.parametrize("mk", SMALL)
def test_cliques_match_subset_brute_force(mk):
    g = mk()
    adj = _py_adj(g)
    for k in (3, 4, 5, 6):
        bf = sum(1 for W in itertools.combinations(range(g.n), k)
                 if all(b in adj[a] for a, b in itertools.combinations(W, 2)))
        assert O.cliques(g, k) == bf


@pytest.mark.parametrize("mk", [lambda: gg.random_small(16, 0.75, 21), lambda: gg.random_small(19, 0.65, 22)])
def test_large_cliques_match_subset_brute_force(mk):
    # k = 7..9 by a recursive extension over sorted candidate lists (written
    # here, independent of the oracle's code)
    g = mk()
    adj = _py_adj(g)

    def ext(cands, r):
        if r == 0:
            return 1
        return sum(ext([w for w in cands[i + 1:] if w in adj[v]], r - 1) for i, v in enumerate(cands))

    for k in (7, 8, 9):
        assert O.cliques(g, k) == ext(list(range(g.n)), k), k


def test_cliques_hub_identity():
    # a vertex set B with its own edges, joined completely to an independent
    # set C and to one more vertex a: every k-clique is either inside B or one
    # vertex of {a} + C with a (k-1)-clique of B
    rng = np.random.default_rng(5)
    nb, nc = 60, 70
    B = np.arange(1, 1 + nb)
    inner = [(int(B[i]), int(B[j])) for i in range(nb) for j in range(i + 1, nb) if rng.random() < 0.3]
    inner += [(int(B[i]), int(B[j])) for i in range(9) for j in range(i + 1, 9)]
    e = [(0, int(b)) for b in B] + [(int(b), int(c)) for b in B for c in range(1 + nb, 1 + nb + nc)] + inner
    g = gg.from_edges(1 + nb + nc, e)
    gb = gg.from_edges(1 + nb, inner)
    for k in (3, 5, 7, 8, 9):
        assert O.cliques(g, k) == (1 + nc) * O.cliques(gb, k - 1) + O.cliques(gb, k), k


@pytest.mark.parametrize("mk", SMALL[:4])
def test_clique_root_ranges_partition_and_match_definition(mk):
    """Root = clique vertex minimal in the order (degree, id)."""
    g = mk()
    adj = _py_adj(g)
    deg = [len(a) for a in adj]
    for k in (3, 4):
        roots = [0] * g.n
        for W in itertools.combinations(range(g.n), k):
            if all(b in adj[a] for a, b in itertools.combinations(W, 2)):
                roots[min(W, key=lambda v: (deg[v], v))] += 1
        cuts = [0, g.n // 3, g.n // 2, g.n]
        parts = [O.cliques(g, k, cuts[i], cuts[i + 1]) for i in range(3)]
        assert parts == [sum(roots[cuts[i]:cuts[i + 1]]) for i in range(3)]


# ---------------- 3-motifs and the wedge identity ----------------

@pytest.mark.parametrize("mk", SMALL + [lambda: gg.workload_tc_rmat14()])
def test_wedge_identity(mk):
    g = mk()
    d = g.degrees()
    s2 = int(np.sum(d * (d - 1) // 2))
    wedge, tri = O.motifs(g, 3)
    assert wedge + 3 * tri == s2
    assert tri == O.triangles(g)


@pytest.mark.parametrize("m", [2, 3, 5, 9])
def test_star_motifs(m):
    g = gg.star(m)
    assert O.motifs(g, 3) == [math.comb(m, 2), 0]
    assert O.motifs(g, 4) == [math.comb(m, 3), 0, 0, 0, 0, 0]


@pytest.mark.parametrize("n", [4, 5, 6, 9])
def test_cycle_motifs(n):
    g = gg.cycle(n)
    assert O.motifs(g, 3) == [n, 0]
    m4 = O.motifs(g, 4)
    if n == 4:
        assert m4 == [0, 0, 0, 1, 0, 0]
    else:
        assert m4 == [0, n, 0, 0, 0, 0]


def test_cycle3_motifs():
    assert O.motifs(gg.cycle(3), 3) == [0, 1]


# ---------------- 4-motifs ----------------

@pytest.mark.parametrize("n", [4, 5, 7, 10])
def test_motifs_complete(n):
    assert O.motifs(gg.complete(n), 4) == [0, 0, 0, 0, 0, math.comb(n, 4)]


@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (3, 4), (4, 6)])
def test_motifs_complete_bipartite(a, b):
    g = gg.complete_multipartite([a, b])
    S = a * math.comb(b, 3) + b * math.comb(a, 3)
    assert O.motifs(g, 4) == [S, 0, 0, math.comb(a, 2) * math.comb(b, 2), 0, 0]


def test_motifs_petersen():
    assert O.motifs(gg.petersen(), 4) == [10, 60, 0, 0, 0, 0]


def _connected(adj, W):
    W = list(W)
    seen = {W[0]}
    stack = [W[0]]
    while stack:
        x = stack.pop()
        for y in W:
            if y not in seen and y in adj[x]:
                seen.add(y)
                stack.append(y)
    return len(seen) == len(W)


@pytest.mark.parametrize("mk", SMALL)
def test_motif_total_is_connected_subsets(mk):
    g = mk()
    adj = _py_adj(g)
    for k in (3, 4):
        conn = sum(1 for W in itertools.combinations(range(g.n), k) if _connected(adj, W))
        assert sum(O.motifs(g, k)) == conn


@pytest.mark.parametrize("mk", SMALL)
def test_motifs_match_brute_force_per_pattern(mk):
    g = mk()
    assert O.motifs(g, 4) == [O.bf_induced(g, p) for p in O.MOTIF4_PATTERNS]
    assert O.motifs(g, 3) == [O.bf_induced(g, p) for p in O.MOTIF3_PATTERNS]


@pytest.mark.parametrize("mk", SMALL)
def test_noninduced_terms_each_match_brute_force(mk):
    """Each closed-form non-induced count is pinned separately, so a dropped
    term in any one formula fails here even if the inversion hid it."""
    g = mk()
    assert O.noninduced_terms(g, 4) == [O.bf_noninduced(g, p) for p in O.MOTIF4_PATTERNS]
    assert O.noninduced_terms(g, 3) == [O.bf_noninduced(g, p) for p in O.MOTIF3_PATTERNS]


def test_noninduced_brute_force_is_injective_maps_over_automorphisms():
    # a 4-cycle graph has 8 injective maps of C4 and |Aut(C4)| = 8
    g = gg.cycle(4)
    assert len(O.bf_maps(g, O.CYCLE4)) == 8
    assert O.bf_noninduced(g, O.CYCLE4) == 1
    # K4 has 4! maps of K4, |Aut(K4)| = 24
    assert len(O.bf_maps(gg.complete(4), O.clique_pattern(4))) == 24


def test_automorphism_group_orders():
    # textbook orders: K_{1,3}: 3!, P4: 2, paw: 2, C4: dihedral 8, diamond: 4, K4: 4!
    assert [O.automorphisms(p) for p in O.MOTIF4_PATTERNS] == [6, 2, 2, 8, 4, 24]
    assert [O.automorphisms(p) for p in O.MOTIF3_PATTERNS] == [2, 6]


# ---------------- subgraph listing counts (edge-induced) ----------------

@pytest.mark.parametrize("n", [4, 5, 6, 9])
def test_sl_complete(n):
    g = gg.complete(n)
    assert O.diamonds(g) == 6 * math.comb(n, 4)
    assert O.cycles4(g) == 3 * math.comb(n, 4)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 3), (2, 7), (5, 4)])
def test_sl_complete_bipartite(a, b):
    g = gg.complete_multipartite([a, b])
    assert O.cycles4(g) == math.comb(a, 2) * math.comb(b, 2)
    assert O.diamonds(g) == 0


@pytest.mark.parametrize("mk", SMALL)
def test_sl_match_injective_map_brute_force(mk):
    g = mk()
    # distinct edge sets from a direct python enumeration of 4-vertex tuples
    adj = _py_adj(g)
    dia, cyc = set(), set()
    for t in itertools.permutations(range(g.n), 4):
        a, b, c, d = t
        if b in adj[a] and c in adj[a] and d in adj[a] and c in adj[b] and d in adj[b]:
            dia.add(frozenset(map(frozenset, [(a, b), (a, c), (a, d), (b, c), (b, d)])))
        if b in adj[a] and c in adj[b] and d in adj[c] and a in adj[d]:
            cyc.add(frozenset(map(frozenset, [(a, b), (b, c), (c, d), (d, a)])))
    assert O.diamonds(g) == len(dia)
    assert O.cycles4(g) == len(cyc)
    assert O.bf_noninduced(g, O.DIAMOND) == len(dia)
    assert O.bf_noninduced(g, O.CYCLE4) == len(cyc)
    assert len(O.bf_subgraph_set(g, O.DIAMOND)) == len(dia)


@pytest.mark.parametrize("mk", SMALL[:4])
def test_sl_root_ranges_partition_and_match_definition(mk):
    g = mk()
    adj = _py_adj(g)
    deg = [len(a) for a in adj]
    key = lambda v: (deg[v], v)
    dia_root = [0] * g.n
    cyc_root = [0] * g.n
    seen_d, seen_c = set(), set()
    for t in itertools.permutations(range(g.n), 4):
        a, b, c, d = t
        if b in adj[a] and c in adj[a] and d in adj[a] and c in adj[b] and d in adj[b]:
            es = frozenset(map(frozenset, [(a, b), (a, c), (a, d), (b, c), (b, d)]))
            if es not in seen_d:
                seen_d.add(es)
                dia_root[min((a, b), key=key)] += 1
        if b in adj[a] and c in adj[b] and d in adj[c] and a in adj[d]:
            es = frozenset(map(frozenset, [(a, b), (b, c), (c, d), (d, a)]))
            if es not in seen_c:
                seen_c.add(es)
                cyc_root[max(t, key=key)] += 1
    cuts = [0, g.n // 4, g.n // 2, g.n]
    for i in range(3):
        assert O.diamonds(g, cuts[i], cuts[i + 1]) == sum(dia_root[cuts[i]:cuts[i + 1]])
        assert O.cycles4(g, cuts[i], cuts[i + 1]) == sum(cyc_root[cuts[i]:cuts[i + 1]])


# ---------------- orientation ----------------

def test_orientation_rule():
    # appendix "Orientation (Total Order)": towards the higher degree, ties to the larger id
    g = _sym(5, [(0, 1), (1, 2), (2, 3), (3, 4), (1, 3)])  # degrees 1,3,2,3,1
    od = O.out_degrees(g)
    # 0->1 ; 1->3 (tie deg 3, larger id) ; 2->1, 2->3 ; 4->3
    assert list(od) == [1, 1, 2, 0, 1]
    g2 = gg.workload_tc_rmat14()
    assert int(O.out_degrees(g2).sum()) == g2.m


# ---------------- worked examples printed in the paper ----------------

def test_eq1_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "eq1_example.json")))
    assert O.eq1_local_wedges(ex["deg_u"], ex["deg_v"], ex["c_tri"]) == ex["c_wdg"]
    g = _sym(7, ex["graph_edges"])
    d = g.degrees()
    u, v = ex["u"], ex["v"]
    assert (d[u], d[v]) == (ex["deg_u"], ex["deg_v"])
    common = len(set(g.neighbors(u)) & set(g.neighbors(v)))
    assert common == ex["c_tri"]
    assert O.edge_wedges_direct(g, u, v) == ex["c_wdg"]


@pytest.mark.parametrize("mk", SMALL[:3])
def test_eq1_on_every_edge(mk):
    g = mk()
    adj = _py_adj(g)
    d = g.degrees()
    for u, v in g.edges():
        t = len(adj[u] & adj[v])
        direct = sum(1 for w in range(g.n) if w not in (u, v) and ((w in adj[u]) != (w in adj[v])))
        assert O.eq1_local_wedges(int(d[u]), int(d[v]), t) == direct


def test_connectivity_code_example():
    ex = json.load(open(os.path.join(GOLDEN, "connectivity_code_example.json")))
    g = _sym(4, ex["graph_edges"])
    assert O.connectivity_code(g, ex["embedding"]) == ex["code"]
    adj = O.code_to_adjacency(4, ex["code"])
    assert int(adj.sum()) // 2 == ex["edges"]
    rebuilt = gg.from_edges(4, [(i, j) for i in range(4) for j in range(i + 1, 4) if adj[i, j]])
    assert O.bf_induced(rebuilt, O.DIAMOND) == 1


def test_connectivity_map_example():
    ex = json.load(open(os.path.join(GOLDEN, "connectivity_map_example.json")))
    g = _sym(4, ex["graph_edges"])
    assert O.connectivity_map_lookup(g, ex["embedding"], ex["lookup"]) == ex["positions"]


def test_orders_satisfying_counts_permutations():
    # no constraint: all k! orders; a full chain 0<1<2<3: exactly one
    assert O.orders_satisfying(4, []) == 24
    assert O.orders_satisfying(4, [(0, 1), (1, 2), (2, 3)]) == 1
    assert O.orders_satisfying(3, [(0, 1)]) == 3


# ---------------- core numbers and the core value based orientation ----------------

@pytest.mark.parametrize("mk", SMALL + [lambda: gg.rmat(10, 8.0, seed=5), lambda: gg.chung_lu(3000, 12.0, 2.1, seed=6),
                                        lambda: gg.complete(7), lambda: gg.empty(4)])
def test_core_numbers_match_networkx(mk):
    import networkx as nx
    g = mk()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(g.edges().tolist())
    want = nx.core_number(G)
    assert O.core_numbers(g).tolist() == [want[v] for v in range(g.n)]


@pytest.mark.parametrize("mk", SMALL[:6] + [lambda: gg.rmat(10, 16.0, seed=21)])
def test_cliques_under_core_order(mk):
    # the total does not depend on the order; root ranges follow the order
    # (key, id) by the definition (brute force on the small graphs)
    g = mk()
    core = O.core_numbers(g)
    for k in (3, 4, 5):
        assert O.cliques_keyed(g, core, k) == O.cliques(g, k)
    if g.n <= 30:
        adj = _py_adj(g)
        for k in (3, 4):
            roots = [0] * g.n
            for W in itertools.combinations(range(g.n), k):
                if all(b in adj[a] for a, b in itertools.combinations(W, 2)):
                    roots[min(W, key=lambda v: (int(core[v]), v))] += 1
            cuts = [0, g.n // 3, g.n // 2, g.n]
            assert [O.cliques_keyed(g, core, k, cuts[i], cuts[i + 1]) for i in range(3)] == \
                [sum(roots[cuts[i]:cuts[i + 1]]) for i in range(3)]
    # with the degrees as the key it is the degree order
    deg = np.diff(g.rowptr).astype(np.uint32)
    assert O.cliques_keyed(g, deg, 4, 0, g.n // 2) == O.cliques(g, 4, 0, g.n // 2)


@pytest.mark.parametrize("mk", SMALL + [lambda: gg.rmat(12, 16.0, seed=31), lambda: gg.chung_lu(5000, 16.0, 2.1, seed=24),
                                        lambda: gg.complete(9), lambda: gg.star(8), lambda: gg.empty(3)])
def test_core_order_is_a_degeneracy_order(mk):
    # ordered by (round, id): no vertex has more successors than its core
    # number, core numbers never decrease along the order, and the totals of
    # the clique counts do not change
    g = mk()
    core = O.core_numbers(g).astype(np.int64)
    order = O.core_order(g).astype(np.int64)
    d = np.diff(g.rowptr).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), d)
    dst = g.col.astype(np.int64)
    keep = (order[src] < order[dst]) | ((order[src] == order[dst]) & (src < dst))
    outdeg = np.bincount(src[keep], minlength=g.n)
    assert np.all(outdeg <= core)
    by = np.lexsort((np.arange(g.n), order))
    assert np.all(np.diff(core[by]) >= 0)
    for k in (3, 4):
        assert O.cliques_keyed(g, order, k) == O.cliques(g, k)


# ---------------- 5-vertex motifs ----------------

def _mask_graph5(mask):
    import networkx as nx
    pairs = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    G = nx.Graph()
    G.add_nodes_from(range(5))
    G.add_edges_from(p for i, p in enumerate(pairs) if mask >> i & 1)
    return G


def test_motif5_classes_are_the_21_connected_graphs():
    # the class masks are pairwise non-isomorphic connected 5-vertex graphs,
    # one per connected 5-vertex graph of the networkx graph atlas
    import networkx as nx
    _, masks = O.motifs5(gg.complete(5))
    assert len(masks) == 21
    gs = [_mask_graph5(m) for m in masks]
    assert all(nx.is_connected(G) for G in gs)
    atlas = [G for G in nx.graph_atlas_g() if G.number_of_nodes() == 5 and nx.is_connected(G)]
    assert len(atlas) == 21
    for A in atlas:
        assert sum(nx.is_isomorphic(A, G) for G in gs) == 1
    edges = [G.number_of_edges() for G in gs]
    assert edges == sorted(edges)


# want = {edge count of the only class present: its count}
@pytest.mark.parametrize("mk, want", [
    (lambda: gg.complete(8), {10: 56}),          # K5: C(8, 5)
    (lambda: gg.path(9), {4: 5}),                # 5-paths: n - 4
    (lambda: gg.cycle(5), {5: 1}),               # one 5-cycle
    (lambda: gg.star(6), {4: 15}),               # 4-stars: C(6, 4)
])
def test_motifs5_closed_forms(mk, want):
    import networkx as nx
    g = mk()
    counts, masks = O.motifs5(g)
    assert sum(counts) == sum(want.values())
    # the class holding the count has the expected shape
    (edges, c), = want.items()
    got = [i for i, x in enumerate(counts) if x]
    assert len(got) == 1 and counts[got[0]] == c
    G = _mask_graph5(masks[got[0]])
    assert G.number_of_edges() == edges
    if g.n >= 5 and edges == 4:
        deg = sorted(d for _, d in G.degree())
        assert deg == ([1, 1, 1, 1, 4] if g.name.startswith("S") else [1, 1, 2, 2, 2])


@pytest.mark.parametrize("mk", [lambda: gg.random_small(11, 0.4, 31), lambda: gg.random_small(13, 0.3, 32),
                                lambda: gg.petersen(), lambda: gg.complete_multipartite([2, 3, 2]),
                                lambda: gg.random_small(10, 0.7, 33)])
def test_motifs5_match_subset_brute_force(mk):
    # every 5-subset, its induced subgraph classified by networkx isomorphism
    import networkx as nx
    g = mk()
    adj = _py_adj(g)
    counts, masks = O.motifs5(g)
    gs = [_mask_graph5(m) for m in masks]
    want = [0] * 21
    for W in itertools.combinations(range(g.n), 5):
        H = nx.Graph()
        H.add_nodes_from(W)
        H.add_edges_from((a, b) for a, b in itertools.combinations(W, 2) if b in adj[a])
        if not nx.is_connected(H):
            continue
        want[[i for i, G in enumerate(gs) if nx.is_isomorphic(G, H)][0]] += 1
    assert counts == want


def test_motifs5_root_ranges_brute_force():
    # restricted to the subsets whose smallest vertex lies in [lo, hi): every
    # 5-subset classified by networkx isomorphism; the ranges partition the total
    import networkx as nx
    g = gg.random_small(12, 0.45, 34)
    adj = _py_adj(g)
    total, masks = O.motifs5(g)
    gs = [_mask_graph5(m) for m in masks]
    cuts = [0, 1, 4, 5, 9, g.n]
    acc = [0] * 21
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        want = [0] * 21
        for W in itertools.combinations(range(g.n), 5):
            if not lo <= W[0] < hi:
                continue
            H = nx.Graph()
            H.add_nodes_from(W)
            H.add_edges_from((a, b) for a, b in itertools.combinations(W, 2) if b in adj[a])
            if nx.is_connected(H):
                want[[i for i, G in enumerate(gs) if nx.is_isomorphic(G, H)][0]] += 1
        got, _ = O.motifs5(g, lo, hi)
        assert got == want, (lo, hi)
        acc = [a + b for a, b in zip(acc, got)]
    assert acc == total
