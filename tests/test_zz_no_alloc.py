"""The allocation-free 4-cycle entry point, called through the C-ABI, gives the
same count as the regular counting path, on two calls in a row (the fixed
scratch array keeps the previous call's contents and must be cleared by the
entry point itself). Collected last so that a failure here does not hide the
other tests."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2011_03135_b300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_03135_b300 import gpm
    return gpm, torch


def _call(gpm, torch, g, out):
    rp = torch.from_numpy(g.rowptr.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda() if g.nnz else torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = gpm._lib.gpm_count_cycles4_noalloc(ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                            ctypes.c_uint32(g.n), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("mk", [lambda: gg.rmat(12, 16.0, seed=3), lambda: gg.chung_lu(30000, 12.0, 2.1, seed=5),
                                lambda: gg.complete_multipartite([3, 4, 5])])
def test_noalloc_matches_regular_count_twice(env, mk):
    gpm, torch = env
    g = mk()
    G = gpm.Graph.from_host(g)
    want = gpm.count(G, [gpm.Pattern.spec(O.CYCLE4, induced=False)])[0]
    G.close()
    assert want == O.cycles4(g)
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        out.fill_(-1)
        assert _call(gpm, torch, g, out) == 0, gpm._lib.gpm_last_error()
        assert int(out.item()) == want


def test_noalloc_near_the_size_limit(env):
    # a ladder with m rungs (2m vertices, close to the largest n the fixed
    # array takes, so a single tally slot): exactly m - 1 four-cycles; then a
    # small graph again, whose slots overlap what the large call left behind
    gpm, torch = env
    m = 2_750_000
    i = np.arange(m, dtype=np.int64)
    e = np.concatenate([np.stack([2 * i, 2 * i + 1], 1), np.stack([2 * i[:-1], 2 * i[1:]], 1),
                        np.stack([2 * i[:-1] + 1, 2 * i[1:] + 1], 1)])
    g = gg.from_edges(2 * m, e, name="ladder")
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert _call(gpm, torch, g, out) == 0, gpm._lib.gpm_last_error()
    assert int(out.item()) == m - 1
    h = gg.rmat(12, 16.0, seed=3)
    assert _call(gpm, torch, h, out) == 0, gpm._lib.gpm_last_error()
    assert int(out.item()) == O.cycles4(h)


def test_noalloc_rejects_oversize_graph(env):
    gpm, torch = env
    n = 6_000_000  # more vertices than the fixed array can hold; rejected before any launch
    rp = np.zeros(n + 1, dtype=np.uint64)
    g = gg.Graph(n, rp, np.zeros(0, dtype=np.uint32))
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = _call(gpm, torch, g, out)
    assert rc == -1
    assert b"too large" in gpm._lib.gpm_last_error()
