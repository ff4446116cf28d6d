"""The N > 1 benchmark path on CPU: two gloo ranks, each timing its own independent replica (the
transform shards into independent problems with no data-path collective); the job's time is the
max over ranks and the throughput counts the units of all ranks."""
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
    my_ms = [120.0, 135.5][rank]
    job_ms = bench.aggregate_max(my_ms, world)
    units_per_rank, steps = 1 << 20, 10
    value = units_per_rank * steps * world / (job_ms / 1e3)
    out[rank] = (job_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling_units():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 135.5
    assert abs(out[0][1] - (1 << 20) * 10 * 2 / 0.1355) < 1e-6 * out[0][1]


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_max(42.0, 1) == 42.0
