"""The bench's multi-process plumbing on CPU (gloo, two ranks): rank/world discovery from the
launcher's environment and the max-over-ranks reduction of the timed value; the reference
arm's non-zero ranks exit without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, loc = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    m = bench.max_over_ranks(1.5 + 10 * r, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, loc, m))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(r[3] == 11.5 for r in res)


def test_single_process_reduction_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25


def test_reference_arm_non_zero_rank_does_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        n_side, steps, warmup, placement = 42, 1, 1, 0.1025
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
