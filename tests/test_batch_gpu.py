"""Batched form: one persistent kernel over many queries gives, per query, the
same exact counts as the plain one-query-per-call path and as the oracle."""
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


def _oracle(g, kind, gpm):
    if kind == gpm.QUERY_MOTIF3:
        return O.motifs(g, 3)
    if kind == gpm.QUERY_MOTIF4:
        return O.motifs(g, 4)
    return [O.cliques(g, {gpm.QUERY_TC: 3, gpm.QUERY_CLIQUE4: 4, gpm.QUERY_CLIQUE5: 5}[kind])]


def test_batch_mixed_small(gpm):
    specs = gg.batch_query_specs(24, base_seed=500, log2n_range=(6, 11), dbar_range=(4.0, 24.0))
    graphs = [gg.graph_from_spec(s) for s in specs]
    kinds = [gpm.QUERY_MOTIF3 if s["k"] == 3 else gpm.QUERY_MOTIF4 for s in specs]
    kinds[0] = gpm.QUERY_TC
    kinds[1] = gpm.QUERY_CLIQUE4
    kinds[2] = gpm.QUERY_CLIQUE5
    Gs = [gpm.Graph.from_host(g) for g in graphs]
    B = gpm.Batch(list(zip(Gs, kinds)))
    for rep in range(3):  # autotune run, then replays
        got = B.run()
        for i, (g, k) in enumerate(zip(graphs, kinds)):
            assert got[i] == _oracle(g, k, gpm), (rep, i, g.name, k)
    info = B.info()
    assert info["items"] > 0 and info["grid"] > 0
    B.close()
    # the plain path on the same graphs agrees
    for G, g, k in zip(Gs, graphs, kinds):
        assert gpm.count(G, gpm.plain_patterns(k)) == _oracle(g, k, gpm)


@pytest.mark.parametrize("direct_us", [1, 0xFFFFFFFF])
def test_batch_direct_and_item_queries(gpm, direct_us):
    # every query run as its plain path inside the graph (1 us), or every
    # query as items (never); a graph used by several queries included
    old = gpm.get_options()
    try:
        gpm.set_options(batch_direct_us=direct_us)
        specs = gg.batch_query_specs(10, base_seed=700, log2n_range=(7, 11), dbar_range=(4.0, 24.0))
        graphs = [gg.graph_from_spec(s) for s in specs]
        Gs = [gpm.Graph.from_host(g) for g in graphs]
        qs = [(G, gpm.QUERY_MOTIF4 if i % 2 else gpm.QUERY_MOTIF3) for i, G in enumerate(Gs)]
        qs += [(Gs[0], gpm.QUERY_CLIQUE5), (Gs[1], gpm.QUERY_TC), (Gs[1], gpm.QUERY_MOTIF4)]
        B = gpm.Batch(qs)
        for rep in range(3):
            got = B.run()
            for i, (G, k) in enumerate(qs):
                g = graphs[Gs.index(G)]
                assert got[i] == _oracle(g, k, gpm), (rep, i, k)
        B.close()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})


def test_batch_same_graph_several_queries(gpm):
    g = gg.rmat(11, 16.0, seed=9)
    G = gpm.Graph.from_host(g)
    qs = [(G, gpm.QUERY_MOTIF4), (G, gpm.QUERY_MOTIF4), (G, gpm.QUERY_MOTIF3), (G, gpm.QUERY_CLIQUE5)]
    got = gpm.count_batch(qs)
    assert got == [O.motifs(g, 4), O.motifs(g, 4), O.motifs(g, 3), [O.cliques(g, 5)]]


def test_batch_heavy_roots_and_empty_graphs(gpm):
    graphs = [gg.chung_lu(20000, 20.0, 2.1, seed=4), gg.empty(10), gg.from_edges(2, [(0, 1)]),
              gg.rmat(12, 32.0, seed=5)]
    Gs = [gpm.Graph.from_host(g) for g in graphs]
    qs = [(G, gpm.QUERY_MOTIF4) for G in Gs] + [(Gs[3], gpm.QUERY_CLIQUE5)]
    got = gpm.count_batch(qs)
    want = [O.motifs(g, 4) for g in graphs] + [[O.cliques(graphs[3], 5)]]
    assert got == want
