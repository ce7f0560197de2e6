"""bench.py's multi-rank path on CPU: two gloo ranks, each timing its own
independent box; the whole-job rate uses the slowest rank's time (weak
scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = 0.010 + 0.005 * rank  # rank 1 is the slower one
    mx = bench.reduce_max(local_seconds, dist, "cpu")
    rate = bench.whole_job_rate(1000, 4, world, mx)
    out[rank] = (mx, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_use_the_slowest_rank():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        mx, rate = out[r]
        assert mx == pytest.approx(0.015)
        assert rate == pytest.approx(2 * 1000 * 4 / 0.015 / 1e6)


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(0.25, None, "cpu") == 0.25
    assert bench.whole_job_rate(10, 2, 1, 0.5) == pytest.approx(40 / 1e6)
