"""Throughput of the staggered-grid Navier-Stokes RK2 step on GB300.

One step = one full Heun RK2 step of the lid-driven cavity (Sec. 4.2's
workload, Re = 1000, 512^3 cells by default): per stage the RHS + stage
combine, ghost fills, divergence, 50 Jacobi sweeps and the projection, all
in the CUDA library, replayed from one CUDA graph per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line: GLUP/s (interior cells x steps / s / 1e9), the Jacobi
sweep against the measured HBM roofline, an end-to-end figure through the C
ABI with host buffers, and the FP64 oracle timed on the host cores.
N > 1 (torchrun): N independent replicas, one per GPU ("replicas only": the
single-GPU path has no data exchange between GPUs); value = cells of all
ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "GLUP/s and HBM GB/s vs peak per sweep; batched/bf16 vs plain; adjoint/fwd ratio"
UNIT = "GLUP/s"
JACOBI_BYTES_PER_CELL = {"f32": 12, "bf16": 6, "f16": 6}
KERNEL_SRC = os.path.join(ROOT, "paper_1201_2118_gb300", "csrc", "stencil_kernels.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "jacobi_dram_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ldc512", choices=["ldc512", "ldc256"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    a = ap.parse_args()
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def traffic_for(kernel_hash: str, cells: int):
    """DRAM bytes per Jacobi launch from the committed ncu summary, scaled to
    this launch's cells; None when the kernel changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("kernel_sha256") != kernel_hash:
        return None
    return t["dram_bytes_per_cell"] * cells


def file_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


# --------------------------------------------------------------- oracle leg

def oracle_sample(seconds_hint=False):
    """One RK2 step of the same cavity scheme on a 256^3 grid by the FP64
    oracle on all host cores (bounded sample of the 512^3 workload; the
    per-cell work is identical)."""
    from oracle import Oracle
    n = 256
    h = (1.0 / n,) * 3
    o = Oracle((n, n, n), ghost=1, h=h, bc="cavity", nu=1e-3)
    u, p = o.state(workloads.ldc_noise(n, seed=1))
    dt = workloads.cfl_dt(h)
    scratch = [o.zeros() for _ in range(8)]
    t0 = time.perf_counter()
    o.rk2_step(u, p, dt, 50, scratch)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n ** 3 / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "1 RK2 step (2 x 50 Jacobi sweeps) of the 256^3 lid-driven cavity, "
                      "FP64 C oracle, OpenMP over z; %.1f s" % el}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name = a.workload
    cfg = workloads.WORKLOADS[name]
    steps = []
    base = None
    for _ in range(a.warmup if a.warmup < 1 else 0):
        pass
    for i in range(a.steps):
        s = oracle_sample()
        steps.append(s["value"])
        base = s
    value = statistics.median(steps)
    ms = cfg["dims"][0] ** 3 / (value * 1e9) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "dims": list(cfg["dims"]), "bc": "lid-driven cavity",
                       "nu": cfg["nu"], "jacobi_iters": cfg["jacobi_iters"],
                       "sample": base["sample"]},
            "cpu_baseline": dict(base, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

def run_gpu(a):
    import numpy as np
    import torch

    from paper_1201_2118_gb300 import Grid, U, V, W, P, library_path

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    name = a.workload
    cfg = workloads.WORKLOADS[name]
    dims = cfg["dims"]
    n = dims[0]
    cells = n ** 3
    h = workloads.workload_h(name)
    dt = workloads.cfl_dt(h)
    stream = torch.cuda.Stream()
    g = Grid(dims, ghost=cfg["ghost"], h=h, dtype=a.dtype, stream=stream)
    g.set_cavity(1.0)
    g.set_params(cfg["nu"], cfg["jacobi_iters"], 1.0, cfg["order"])
    g.upload(workloads.ldc_noise(n, seed=cfg["seed"]))

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (captures the step graph)
    for _ in range(a.warmup):
        g.step(dt, 1)
    torch.cuda.synchronize()
    g.check()

    # ---- timed region: K full RK2 steps
    l0 = g.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            g.step(dt, 1)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = g.launches - l0
    ms = e0.elapsed_time(e1) / a.steps
    g.check()
    if dist is not None:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * cells / (ms * 1e-3) / 1e9
    ke, umax, divmax = g.reduce(0)

    # ---- dominant kernel: the Jacobi sweep, timed alone on the grid's stream
    sweeps = 100
    j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.jacobi(4)
    torch.cuda.synchronize()
    j0.record(stream)
    g.jacobi(sweeps)
    j1.record(stream)
    torch.cuda.synchronize()
    sweep_ms = j0.elapsed_time(j1) / sweeps
    bytes_per_launch = JACOBI_BYTES_PER_CELL[a.dtype] * cells
    achieved = bytes_per_launch / (sweep_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = traffic_for(file_hash(KERNEL_SRC), cells)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_jacobi (one weighted Jacobi sweep, %d^3, %s)" % (n, a.dtype),
                "bytes_per_launch": bytes_per_launch, "launch_ms": sweep_ms,
                "peak_source": "%s hbm_gbs (burst copy)" % peak_kind,
                "sweep_glups": cells / (sweep_ms * 1e-3) / 1e9}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not a.no_e2e:
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
        host_in = [torch.empty((n, n, n), dtype=tdt, pin_memory=True) for _ in range(4)]
        host_out = [torch.empty((n, n, n), dtype=tdt, pin_memory=True) for _ in range(4)]
        for k, arr in enumerate((U, V, W, P)):
            g.copy_interior(arr, host_out[k].data_ptr(), to_device=False)
        torch.cuda.synchronize()
        for k in range(4):
            host_in[k].copy_(host_out[k])
        k_e2e = max(3, a.steps // 2)
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        x0.record(stream)
        for _ in range(k_e2e):
            for k, arr in enumerate((U, V, W, P)):
                g.copy_interior(arr, host_in[k].data_ptr(), to_device=True)
            g.step(dt, 1)
            for k, arr in enumerate((U, V, W, P)):
                g.copy_interior(arr, host_out[k].data_ptr(), to_device=False)
        x1.record(stream)
        torch.cuda.synchronize()
        ems = x0.elapsed_time(x1) / k_e2e
        if dist is not None:
            t = torch.tensor([ems], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        es = host_in[0].element_size()
        e2e = {"value": world * cells / (ems * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * cells * es, "d2h_bytes_per_step": 4 * cells * es,
               "ms_per_step": ems, "steps": k_e2e,
               "api": "cfd_copy_interior (pinned host -> device, u,v,w,p) + cfd_step + "
                      "cfd_copy_interior (device -> pinned host, u,v,w,p)"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = oracle_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
            "config": {"workload": name, "dims": list(dims), "bc": "lid-driven cavity, lid u=1",
                       "nu": cfg["nu"], "dt": dt, "jacobi_iters": cfg["jacobi_iters"],
                       "rk": "Heun RK2, projection per stage", "ghost": cfg["ghost"],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (each %d^3 field %.0f MB vs 129 MB L2)"
                             % (n, cells * g.torch.tensor([], dtype=g.tdtype).element_size() / 1e6)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "check": {"kinetic_energy": ke, "max_abs_u": umax, "max_abs_div": divmax},
            "library": os.path.relpath(library_path(), ROOT),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
