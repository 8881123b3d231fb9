"""The seeded input generators produce valid, reproducible inputs (no mining arithmetic here)."""
import numpy as np
import pytest

from paper_2011_03135_b300 import graphgen as gg


def _valid(g):
    rp, col = g.rowptr, g.col
    assert rp.dtype == np.uint64 and col.dtype == np.uint32
    assert rp[0] == 0 and len(rp) == g.n + 1 and int(rp[-1]) == len(col)
    d = np.diff(rp.astype(np.int64))
    assert (d >= 0).all()
    src = np.repeat(np.arange(g.n, dtype=np.int64), d)
    dst = col.astype(np.int64)
    assert (src != dst).all(), "self-loop"
    key = src * g.n + dst
    assert (np.diff(key) > 0).all(), "unsorted or duplicate"
    rkey = np.sort(dst * g.n + src)
    assert np.array_equal(rkey, key), "asymmetric"


@pytest.mark.parametrize("mk", [
    lambda: gg.rmat(8, 8.0, seed=3), lambda: gg.erdos_renyi(500, 0.02, seed=4, permute=True),
    lambda: gg.chung_lu(3000, 12.0, 2.1, seed=5), gg.petersen, lambda: gg.complete(6),
    lambda: gg.complete_multipartite([2, 3, 1]), lambda: gg.empty(3), lambda: gg.workload_tc_rmat14(),
])
def test_valid_csr(mk):
    _valid(mk())


def test_deterministic():
    a, b = gg.rmat(9, 8.0, seed=7), gg.rmat(9, 8.0, seed=7)
    assert a.digest() == b.digest()
    c = gg.rmat(9, 8.0, seed=8)
    assert a.digest() != c.digest()
    assert gg.chung_lu(2000, 10.0, 2.1, 9).digest() == gg.chung_lu(2000, 10.0, 2.1, 9).digest()


def test_chung_lu_mean_degree_and_cutoff():
    g = gg.chung_lu(50000, 24.0, 2.1, seed=3)
    d = g.degrees()
    assert 21.0 < d.mean() < 24.5
    # largest weight is the structural cutoff sqrt(n * dbar)
    assert abs(g.meta["max_weight"] - (50000 * 24.0) ** 0.5) < 1e-6 * g.meta["max_weight"]


def test_er_density():
    g = gg.erdos_renyi(2000, 0.01, seed=1)
    expect = 0.01 * 2000 * 1999 / 2
    assert abs(g.m - expect) < 5 * expect ** 0.5


def test_batch_specs_shape():
    s = gg.batch_query_specs(512)
    assert len(s) == 512
    kinds = {x["kind"] for x in s}
    assert kinds == {"er", "rmat"}
    assert {x["k"] for x in s} == {3, 4}
    for x in s:
        assert 2 ** 10 - 1 <= x["n"] <= 2 ** 20 + 1
