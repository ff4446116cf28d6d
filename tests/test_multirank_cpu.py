"""The N > 1 benchmark path on CPU: two gloo ranks, each timing its own independent replica (the
transform shards into independent problems with no data-path collective); the job's time is the
max over ranks and the throughput counts the units of all ranks.  Each rank also draws its own
replica's inputs (the benchmark's per-rank recipe, at a small size) and transforms them with the
FP64 oracle: the ranks must hold different, reproducible problems, and a rank's result must not
depend on which process computed it."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SMALL = dict(N=3000, M=2000, grid=16, order=4, sigma=0.05)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica_result(rank):
    import bench
    import oracle
    wl = bench.replica_workload(rank, **SMALL)
    d = oracle.OracleDesc(dim=3, grid=wl.grid, order=wl.order, sigma=wl.sigma)
    sel = np.arange(0, wl.M, 97)
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    return oracle.forward(d, f64(wl.p), f64(wl.w), f64(wl.q), sel=sel)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_ms = [120.0, 135.5][rank]
    job_ms = bench.aggregate_max(my_ms, world)
    units_per_rank, steps = 1 << 20, 10
    value = bench.job_value(units_per_rank, steps, world, job_ms)
    y = torch.from_numpy(_replica_result(rank))
    ys = [torch.zeros_like(y) for _ in range(world)]
    dist.all_gather(ys, y)
    out[rank] = (job_ms, value, [t.numpy().tolist() for t in ys])
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
    # both ranks saw the same gathered results; the two replicas differ; each rank's result is the
    # one its seed gives in this process too
    g0, g1 = (np.array(v) for v in out[0][2]), (np.array(v) for v in out[1][2])
    g0, g1 = list(g0), list(g1)
    assert all(np.array_equal(a, b) for a, b in zip(g0, g1))
    assert not np.allclose(g0[0], g0[1])
    for r in range(2):
        assert np.array_equal(g0[r], _replica_result(r))


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_max(42.0, 1) == 42.0
    assert bench.job_value(100, 2, 1, 1000.0) == 200.0
    w0 = bench.replica_workload(0, **SMALL)
    assert np.array_equal(w0.p, bench.replica_workload(0, **SMALL).p)
