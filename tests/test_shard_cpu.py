"""Sharding a batch of scenes over ranks (no GPU): the partition is complete, disjoint,
deterministic and balanced by nnz(S~); two gloo ranks that each compute their own shard from
the library's host precompute agree on it without exchanging it, and together hold every
scene once."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2503_15078_b300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_is_complete_disjoint_and_sorted():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 10_000, size=37).tolist()
    for world in (1, 2, 3, 8, 40):
        parts = shard.partition(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)


def test_partition_balance_within_the_lpt_bound():
    # the longest-processing-time rule: the largest load is at most the mean load plus the
    # largest single cost, and equal costs split evenly
    rng = np.random.default_rng(1)
    costs = (rng.pareto(1.5, size=64) * 1000 + 1).tolist()
    for world in (2, 4, 8):
        loads = [sum(costs[i] for i in p) for p in shard.partition(costs, world)]
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    parts = shard.partition([5.0] * 12, 4)
    assert [len(p) for p in parts] == [3, 3, 3, 3]


def test_partition_small_cases_by_hand():
    # decreasing costs 9, 7, 6, 5, 4 on two ranks: 9 -> r0, 7 -> r1, 6 -> r1 (13), 5 -> r0
    # (14), 4 -> r1 (17); ties go to the lower rank
    assert shard.partition([6, 9, 5, 7, 4], 2) == [[1, 2], [0, 3, 4]]
    assert shard.partition([1, 1], 3) == [[0], [1], []]
    with pytest.raises(ValueError):
        shard.partition([1, -1], 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import scenegen as sg
    from paper_2503_15078_b300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scenes = sg.batch(n_scenes=12, seed=3, m_lo=4, m_hi=9)
    idx, mine = S.shard(scenes, rank, world)
    # the check only: gather what every rank chose (the data path exchanges nothing)
    got = [None] * world
    dist.all_gather_object(got, idx)
    costs = S.scene_costs(scenes)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, [sc.n_verts for sc in mine], costs))


def test_two_gloo_ranks_compute_the_same_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, got0, _, costs), (r1, got1, _, _) = res
    assert got0 == got1                       # both ranks computed the same partition
    assert sorted(got0[0] + got0[1]) == list(range(12))
    assert not set(got0[0]) & set(got0[1])
    loads = [sum(costs[i] for i in p) for p in got0]
    assert max(loads) <= sum(costs) / 2 + max(costs)
