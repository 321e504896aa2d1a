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


SMALL = dict(desc="test cavity", dims=(12, 10, 8), ghost=1, nu=1e-3, steps=10, order=2,
             jacobi_iters=6, bc="cavity", ic="ldc_noise", seed=1)


def _ref_args(steps=3, workload="ldc_small"):
    import argparse
    return argparse.Namespace(steps=steps, warmup=3, workload=workload)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints; the other
    ranks return at once."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    def no_call(*a, **k):
        raise AssertionError("rank 1 ran the oracle")
    monkeypatch.setattr(bench.workloads, "ldc_noise", no_call)
    bench.run_reference(_ref_args(workload="ldc512"))
    assert capsys.readouterr().out == ""


def _line(monkeypatch, capsys, steps):
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setitem(bench.workloads.WORKLOADS, "ldc_small", SMALL)
    bench.run_reference(_ref_args(steps))
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_times_the_steps_it_reports(monkeypatch, capsys):
    """Rank 0 prints one JSON line for the configured workload: steps timed,
    their mean time, value = cells x steps / timed seconds; cpu_baseline and
    e2e carry the same figure (no host transfers).  The oracle's state after
    the line's steps equals a direct run of the same steps."""
    import math
    import pytest
    import workloads
    from oracle import Oracle
    d = _line(monkeypatch, capsys, 3)
    nx, ny, nz = SMALL["dims"]
    assert d["impl"] == "reference" and d["steps"] == 3 and d["steps_requested"] == 3
    assert d["config"]["workload"] == "ldc_small" and d["config"]["dims"] == [nx, ny, nz]
    total = sum(d["step_seconds"])
    assert len(d["step_seconds"]) == 3
    assert d["ms_per_step"] * d["steps"] == pytest.approx(total * 1e3)
    assert d["value"] == pytest.approx(nx * ny * nz * 3 / total / 1e9)
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["higher_is_better"] is True
    h = tuple(1.0 / n for n in SMALL["dims"])
    o = Oracle(SMALL["dims"], ghost=1, h=h, bc="cavity", nu=SMALL["nu"])
    u, p = o.state(workloads.ldc_noise(SMALL["dims"], seed=1))
    o.run(u, p, workloads.cfl_dt(h), SMALL["jacobi_iters"], 3)
    ke, umax, divmax = o.reduce(u)
    assert d["check"] == {"kinetic_energy": ke, "max_abs_u": umax, "max_abs_div": divmax}
    assert math.isfinite(ke) and ke > 0


def test_reference_arm_stops_at_its_budget(monkeypatch, capsys):
    import bench
    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.0)
    d = _line(monkeypatch, capsys, 4)
    assert d["steps"] == 1 and d["steps_requested"] == 4
    assert "stopped after 1 of 4 requested steps" in d["cpu_baseline"]["sample"]
    assert d["ms_per_step"] == sum(d["step_seconds"]) * 1e3


def test_bench_arguments(monkeypatch):
    import bench
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.warmup, a.e2e_in_flight, a.impl) == (1, 5, 3, "gb300")
    for bad in (["--warmup", "2"], ["--e2e-in-flight", "1"]):
        monkeypatch.setattr("sys.argv", ["bench.py"] + bad)
        with pytest.raises(SystemExit):
            bench.parse()
