"""The N > 1 path of bench.py (independent replicas, whole-job aggregation)
on CPU ranks over gloo: the slowest rank's time and the sum of all ranks'
pairs; rank 0 alone runs the reference arm."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    busy = [0.50, 0.75][rank]
    pairs = [1000, 3000][rank]
    got = bench.reduce_over_ranks(dist, busy, pairs, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


@pytest.mark.parametrize("world", [2])
def test_replicas_reduce_max_time_sum_pairs(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r] == (0.75, 4000.0)


def test_single_rank_has_no_collective():
    import bench

    assert bench.reduce_over_ranks(None, 0.25, 7, "cpu") == (0.25, 7.0)


def test_reference_arm_only_on_rank0(capsys, monkeypatch):
    import bench

    class A:
        workload, scale, warmup, steps = "self_20k", 1.0, 0, 1

    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""
