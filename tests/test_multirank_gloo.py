"""Multi-rank path on CPU: world-size-2 gloo ranks shard one graph's count by
root ranges and all-reduce the uint64 partials; the sum must equal the
single-rank count. The per-rank count here is the oracle's root-range count
(the GPU path calls gpm_count_roots with the same ranges)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2011_03135_b300 import graphgen as gg
from paper_2011_03135_b300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat(11, 16.0, seed=77)
    costs = shard.root_costs(g.rowptr, g.col)
    got = shard.sharded_count(
        lambda lo, hi: [O.cliques(g, 3, lo, hi), O.cliques(g, 4, lo, hi), O.diamonds(g, lo, hi),
                        O.cycles4(g, lo, hi)],
        g.n, costs, rank, world)
    # the core value based order: roots and costs follow the peel rounds, and
    # large k goes through the same ranges
    order = O.core_order(g)
    got_core = shard.sharded_count(
        lambda lo, hi: [O.cliques_keyed(g, order, 4, lo, hi), O.cliques_keyed(g, order, 7, lo, hi)],
        g.n, shard.root_costs(g.rowptr, g.col, key=order), rank, world)
    # a value above 2^32 survives the exact split reduction
    big = shard.allreduce_counts([(1 << 40) + rank, 2 ** 63 + 5 * rank])
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array(got + got_core + big, dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_partition_properties():
    rng = np.random.default_rng(0)
    c = rng.pareto(1.5, size=10000) + 1
    for world in (1, 2, 3, 8):
        parts = shard.partition(c, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(c)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        loads = [c[lo:hi].sum() for lo, hi in parts]
        assert max(loads) <= c.sum() / world + c.max() + 1e-9


def test_split_join_roundtrip():
    vals = [0, 1, 2 ** 32 - 1, 2 ** 32, 2 ** 64 - 1, 123456789012345]
    assert shard.join_u64(shard.split_u64(vals), len(vals)) == vals


def test_two_gloo_ranks_sum_to_single_rank(tmp_path):
    import oracle as O
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    r0 = list(np.load(tmp_path / "r0.npy", allow_pickle=True))
    r1 = list(np.load(tmp_path / "r1.npy", allow_pickle=True))
    assert r0 == r1
    g = gg.rmat(11, 16.0, seed=77)
    assert r0[:4] == [O.cliques(g, 3), O.cliques(g, 4), O.diamonds(g), O.cycles4(g)]
    assert r0[4:6] == [O.cliques(g, 4), O.cliques(g, 7)]
    assert r0[6:] == [2 * (1 << 40) + 1, 2 * 2 ** 63 + 5]


def test_root_costs_follow_the_key():
    g = gg.rmat(9, 8.0, seed=3)
    import oracle as O
    order = O.core_order(g)
    c_deg = shard.root_costs(g.rowptr, g.col)
    c_key = shard.root_costs(g.rowptr, g.col, key=order)
    core = O.core_numbers(g)
    # under the degeneracy order no out-degree exceeds the core number
    assert np.all(np.sqrt(c_key - 1.0) <= core + 1e-9)
    assert c_deg.sum() == shard.root_costs(g.rowptr, g.col, key=np.diff(g.rowptr)).sum()
