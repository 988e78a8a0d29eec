"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own (independent)
job timing; the aggregate uses the slowest rank and counts every rank's samples."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (slowest, bench.job_throughput(world, 3, 1000, 50, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 180.0
    # 2 ranks x 3 steps x 1000 chains x 50 samples over the slowest rank's 0.18 s
    assert out[0][1] == pytest.approx(2 * 3 * 1000 * 50 / 0.18)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
