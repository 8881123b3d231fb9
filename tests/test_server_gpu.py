"""Served form: requests submitted while others run (continuous batching) give
the same exact counts as each request alone, as the plain count path and as
the oracle."""
import time

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


def _graphs():
    return [gg.rmat(10, 8.0, seed=101), gg.rmat(12, 16.0, seed=102), gg.erdos_renyi(4000, 0.004, seed=103),
            gg.chung_lu(8000, 12.0, 2.1, seed=104), gg.empty(5), gg.from_edges(3, [(0, 1), (1, 2)])]


def _drain(S, want, timeout=120.0):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout:
        for tag, gi, kind, status, counts in S.poll():
            assert status == 0
            got[tag] = (gi, kind, counts)
        time.sleep(0.001)
    assert len(got) == want, f"only {len(got)} of {want} requests finished"
    return got


def _plain(gpm, G, kind):
    return gpm.count(G, gpm.plain_patterns(kind))


def test_server_mix_equals_alone_and_plain(gpm):
    graphs = _graphs()
    Gs = [gpm.Graph.from_host(g) for g in graphs]
    kinds = [gpm.QUERY_TC, gpm.QUERY_CLIQUE4, gpm.QUERY_CLIQUE5, gpm.QUERY_MOTIF4, gpm.QUERY_MOTIF3]
    plain = {(i, k): _plain(gpm, G, k) for i, G in enumerate(Gs) for k in kinds}
    # every (graph, kind) against the oracle, so that alone, in the mix and
    # plain are all compared with it
    for i, g in enumerate(graphs):
        want = {gpm.QUERY_TC: [O.triangles(g)], gpm.QUERY_CLIQUE4: [O.cliques(g, 4)],
                gpm.QUERY_CLIQUE5: [O.cliques(g, 5)], gpm.QUERY_MOTIF4: O.motifs(g, 4),
                gpm.QUERY_MOTIF3: O.motifs(g, 3)}
        for k in kinds:
            assert plain[(i, k)] == want[k], (g.name, k)
    S = gpm.Server(Gs, max_inflight=32)
    # alone: one request at a time
    alone = {}
    for i in range(len(Gs)):
        for k in kinds:
            S.submit(i, k, 1000 + 10 * i + k)
            r = _drain(S, 1)
            alone[(i, k)] = list(r.values())[0][2]
    assert alone == plain
    # in the mix: 200 requests submitted back to back
    rng = np.random.default_rng(7)
    reqs = [(int(rng.integers(len(Gs))), int(kinds[rng.integers(len(kinds))])) for _ in range(200)]
    for tag, (i, k) in enumerate(reqs):
        S.submit(i, k, tag)
    got = _drain(S, len(reqs))
    for tag, (i, k) in enumerate(reqs):
        assert got[tag] == (i, k, plain[(i, k)]), (tag, i, k)
    assert S.stats() == dict(inflight=0, pending=0)
    S.stop()


def test_server_admission_waits_for_memory(gpm):
    # an arena that holds one 4-motif request at a time and 4 request slots:
    # the rest wait in the host FIFO and are admitted as completions free room
    g = gg.rmat(12, 16.0, seed=105)
    G = gpm.Graph.from_host(g)
    want = _plain(gpm, G, gpm.QUERY_MOTIF4)
    assert want == O.motifs(g, 4)
    S = gpm.Server([G], max_inflight=4, arena_bytes=4 * (g.m + 64))
    for tag in range(12):
        S.submit(0, gpm.QUERY_MOTIF4, tag)
    st = S.stats()
    assert st["inflight"] + st["pending"] >= 1
    got = _drain(S, 12)
    assert all(v == (0, gpm.QUERY_MOTIF4, want) for v in got.values())
    S.stop()


def test_server_idle_exit_and_relaunch(gpm):
    g = gg.rmat(9, 8.0, seed=106)
    G = gpm.Graph.from_host(g)
    S = gpm.Server([G], max_inflight=8)
    S.submit(0, gpm.QUERY_TC, 1)
    first = _drain(S, 1)
    time.sleep(0.2)  # longer than the kernel's idle limit: it exits
    S.submit(0, gpm.QUERY_TC, 2)
    second = _drain(S, 1)
    assert first[1][2] == second[2][2] == [O.triangles(g)]
    S.stop()


def test_server_small_requests_overtake_blocked_large_ones(gpm):
    # the arena holds one large 4-motif request; two more wait for it. Small
    # (express) requests submitted after them are admitted at once and finish
    # before the last large one.
    big = gg.rmat(14, 16.0, seed=107)
    small = gg.rmat(7, 8.0, seed=108)
    Gb, Gs = gpm.Graph.from_host(big), gpm.Graph.from_host(small)
    want_big = _plain(gpm, Gb, gpm.QUERY_MOTIF4)
    want_small = _plain(gpm, Gs, gpm.QUERY_TC)
    assert want_big == O.motifs(big, 4) and want_small == [O.triangles(small)]
    S = gpm.Server([Gb, Gs], max_inflight=8, arena_bytes=4 * (big.m + 64))
    for tag in range(3):
        S.submit(0, gpm.QUERY_MOTIF4, tag)
    for tag in range(100, 110):
        S.submit(1, gpm.QUERY_TC, tag)
    order, got = [], {}
    t0 = time.time()
    while len(got) < 13 and time.time() - t0 < 120:
        for tag, gi, kind, status, counts in S.poll():
            assert status == 0
            got[tag] = counts
            order.append(tag)
        time.sleep(0.0005)
    assert len(got) == 13
    assert all(got[t] == want_big for t in range(3)) and all(got[t] == want_small for t in range(100, 110))
    assert max(order.index(t) for t in range(100, 110)) < order.index(2)
    S.stop()


def test_server_hub_items(gpm):
    # a low hub threshold makes hundreds of 4-cycle roots hub roots: the served
    # form splits each into PART and SUM items over a small pool of shared
    # tally slots, reused many times within and across requests
    old = gpm.get_options()
    try:
        gpm.set_options(c4_hub_bound=600)
        graphs = [gg.rmat(11, 16.0, seed=109), gg.chung_lu(6000, 16.0, 2.1, seed=110), gg.rmat(12, 8.0, seed=111)]
        Gs = [gpm.Graph.from_host(g) for g in graphs]
        want = [O.motifs(g, 4) for g in graphs]
        S = gpm.Server(Gs, max_inflight=16)
        tags = [(t, t % len(Gs)) for t in range(24)]
        for t, gi in tags:
            S.submit(gi, gpm.QUERY_MOTIF4, t)
        got = _drain(S, len(tags))
        for t, gi in tags:
            assert got[t] == (gi, gpm.QUERY_MOTIF4, want[gi]), t
        # the same requests one at a time
        for gi in range(len(Gs)):
            S.submit(gi, gpm.QUERY_MOTIF4, 100 + gi)
            assert list(_drain(S, 1).values())[0][2] == want[gi]
        S.stop()
    finally:
        gpm.set_options(**{k: v for k, v in old.items() if v})
