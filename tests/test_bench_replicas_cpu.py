"""The N > 1 bench path (independent replicas, one per GPU) aggregates with a
MAX over ranks of the step time and reports the whole-job throughput; this
runs that aggregation on two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slower one
    ms, value = bench.aggregate(ms_local, 1_000_000, dist, "cpu")
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_replicas_report_max_time_and_whole_job_value():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1_000_000 / 15e-3 / 1e9)


def test_single_process_aggregate_is_identity():
    import bench
    ms, value = bench.aggregate(20.0, 2_000_000)
    assert ms == 20.0 and value == pytest.approx(2_000_000 / 20e-3 / 1e9)
