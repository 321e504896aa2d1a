"""Throughput of the staggered-grid Navier-Stokes RK2 step on GB300.

One step = one full Heun RK2 step of the lid-driven cavity (Sec. 4.2's
workload, Re = 1000, 512^3 cells by default): per stage the RHS + stage
combine, ghost fills, divergence, 50 Jacobi sweeps and the projection, all
in the CUDA library, replayed from one CUDA graph per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line: GLUP/s (interior cells x steps / s / 1e9), the Jacobi
sweep against the measured HBM roofline, an end-to-end figure through the C
ABI with page-locked host buffers (u, v, w, p copied in and out every step;
three independent problems in flight, their copies by the pack kernel on
one CTA per eight SMs, and one problem alone as e2e.serial), and the FP64
oracle timed on the host cores.
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
CSRC = os.path.join(ROOT, "paper_1201_2118_gb300", "csrc")


def kernel_sources(kind: int):
    """Source files of the Jacobi variant `kind` (the TMA variants live in
    jacobi_tma.cu, the others in stencil_kernels.cu)."""
    main = "jacobi_tma.cu" if kind in (1, 7, 9) else "stencil_kernels.cu"
    return [os.path.join(CSRC, f) for f in (main, "dev_common.cuh", "tiles.cuh", "tma_ptx.cuh",
                                            "cfd_internal.h")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "jacobi_dram_traffic.txt")


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
    ap.add_argument("--e2e-in-flight", type=int, default=3,
                    help="independent problems in flight in the end-to-end measurement")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the reduced-precision, block-set and adjoint comparisons")
    ap.add_argument("--precision-steps", type=int, default=20)
    ap.add_argument("--e2e-copy", default="narrow", choices=["narrow", "engine", "kernel"],
                    help="route of the pipelined end-to-end leg's host copies: the pack kernel "
                         "on one CTA per eight SMs over the host link (default), copy engines "
                         "through the staging region, or the pack kernel on the whole GPU")
    ap.add_argument("--e2e-host-mem", default="pinned", choices=["pinned", "hugepages"],
                    help="host buffers of the end-to-end leg: torch's page-locked allocator, or "
                         "anonymous memory advised for transparent huge pages and registered "
                         "with CUDA")
    ap.add_argument("--cuda-connections", type=int, default=0,
                    help="CUDA_DEVICE_MAX_CONNECTIONS for this process (0: leave as is); "
                         "hardware work queues shared by the streams")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (reused when it holds this GPU and grid)")
    a = ap.parse_args()
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    if a.e2e_in_flight < 2:
        ap.error("--e2e-in-flight must be >= 2 (e2e.serial is the one-problem figure)")
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


def profile_record(kernel_hash: str, config):
    """The committed ncu record of the Jacobi launch (DRAM bytes and warp
    instructions per cell), or None when the kernel source or the variant's
    tile (kind, vx, ty, zc) differs from the captured one (the ring depth,
    the last config entry, does not change which bytes move)."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("kernel_sha256") != kernel_hash or list(t.get("config", []))[:4] != list(config)[:4]:
        return None
    return t


def traffic_for(kernel_hash: str, cells: int, config):
    """DRAM bytes per Jacobi launch from the committed ncu record, scaled to
    this launch's cells; None when the record does not apply."""
    t = profile_record(kernel_hash, config)
    return None if t is None else t["dram_bytes_per_cell"] * cells


def file_hash(paths):
    """sha256 over the Jacobi kernels' sources, in order."""
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# --------------------------------------------------------------- oracle leg

def _oracle_step_time(n, threads):
    """Seconds for one RK2 step of the n^3 cavity by the FP64 oracle on the
    given number of host threads (0: all)."""
    from oracle import Oracle, set_threads
    used = set_threads(threads)
    h = (1.0 / n,) * 3
    o = Oracle((n, n, n), ghost=1, h=h, bc="cavity", nu=1e-3)
    u, p = o.state(workloads.ldc_noise(n, seed=1))
    dt = workloads.cfl_dt(h)
    scratch = [o.zeros() for _ in range(8)]
    t0 = time.perf_counter()
    o.rk2_step(u, p, dt, 50, scratch)
    el = time.perf_counter() - t0
    set_threads(0)
    return el, used


def oracle_sample(seconds_hint=False, detail=True):
    """One RK2 step of the same cavity scheme on a 256^3 grid by the FP64
    oracle on all host cores (bounded sample of the 512^3 workload; the
    per-cell work is identical); with detail, also one 128^3 step on one
    thread and on all threads."""
    n = 256
    el, cores = _oracle_step_time(n, 0)
    out = {"value": n ** 3 / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "1 RK2 step (2 x 50 Jacobi sweeps) of the 256^3 lid-driven cavity, "
                     "FP64 C oracle, OpenMP over rows (k, j); %.1f s" % el}
    if detail:
        m = 128
        e1, _ = _oracle_step_time(m, 1)
        ea, ca = _oracle_step_time(m, 0)
        out["scaling_128"] = {"one_thread": m ** 3 / e1 / 1e9, "all_threads": m ** 3 / ea / 1e9,
                              "threads": ca, "unit": UNIT,
                              "sample": "1 RK2 step of the 128^3 cavity: %.1f s on 1 thread, "
                                        "%.2f s on %d" % (e1, ea, ca)}
    return out


# wall-clock budget of the reference arm's timed steps (each a full oracle
# step of the configured workload; about 12 s per 512^3 step on 16 cores)
REF_BUDGET_S = 150.0


def run_reference(a):
    """The reference arm: the FP64 oracle as it stands, on the host cores,
    taking consecutive RK2 steps of the configured cavity from the bench's
    start (the same grid, parameters and seed as the GPU arm).  It times
    --steps steps, or stops early once the next step would pass
    REF_BUDGET_S; `steps` is the number it timed and ms_per_step their mean,
    so steps x ms_per_step is the timed region.  The warm-up steps are not
    run: the oracle has no caches, graphs or compilation to warm."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import Oracle, set_threads
    name = a.workload
    cfg = workloads.WORKLOADS[name]
    dims = tuple(cfg["dims"])
    cells = dims[0] * dims[1] * dims[2]
    cores = set_threads(0)
    h = workloads.workload_h(name)
    dt = workloads.cfl_dt(h)
    o = Oracle(dims, ghost=cfg["ghost"], h=h, bc="cavity", nu=cfg["nu"])
    u, p = o.state(workloads.ldc_noise(dims, seed=cfg["seed"]))
    scratch = [o.zeros() for _ in range(8)]
    times = []
    t_start = time.perf_counter()
    for i in range(a.steps):
        t0 = time.perf_counter()
        o.rk2_step(u, p, dt, cfg["jacobi_iters"], scratch)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start + times[-1] > REF_BUDGET_S:
            break
    steps = len(times)
    total = sum(times)
    value = cells * steps / total / 1e9
    ke, umax, divmax = o.reduce(u)
    sample = ("%d consecutive RK2 steps (2 x %d Jacobi sweeps each) of the %dx%dx%d lid-driven "
              "cavity from the bench's start, FP64 C oracle, OpenMP over rows (k, j) on %d host threads; "
              "%.1f s timed%s" % (steps, cfg["jacobi_iters"], dims[0], dims[1], dims[2], cores,
                                  total, "" if steps == a.steps else
                                  "; stopped after %d of %d requested steps (%.0f s budget)"
                                  % (steps, a.steps, REF_BUDGET_S)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "steps_requested": a.steps, "warmup": a.warmup,
            "ms_per_step": total / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "dims": list(dims), "bc": "lid-driven cavity, lid u=1",
                       "nu": cfg["nu"], "dt": dt, "jacobi_iters": cfg["jacobi_iters"],
                       "rk": "Heun RK2, projection per stage", "ghost": cfg["ghost"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "check": {"kinetic_energy": ke, "max_abs_u": umax, "max_abs_div": divmax},
            "step_seconds": times}
    print(json.dumps(line), flush=True)


def aggregate(ms_local: float, cells: int, dist=None, device="cpu"):
    """Slowest rank's time and the whole-job throughput of N replicas:
    value = N * cells / max_rank(ms) (GLUP/s)."""
    import torch
    world = 1
    ms = ms_local
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * cells / (ms * 1e-3) / 1e9


class HostBuffers:
    """Page-locked host tensors for the end-to-end leg: torch's pinned
    allocator, or (hugepages) anonymous mappings advised for transparent huge
    pages, touched, then registered with cudaHostRegister, so that the host
    side of the link translates 2 MB pages instead of 4 KB ones."""

    def __init__(self, torch, hugepages):
        self.torch, self.huge, self.keep = torch, hugepages, []

    def empty(self, shape, dtype):
        torch = self.torch
        if not self.huge:
            return torch.empty(shape, dtype=dtype, pin_memory=True)
        import mmap
        nbytes = math.prod(shape) * torch.empty((), dtype=dtype).element_size()
        size = (nbytes + (2 << 20) - 1) // (2 << 20) * (2 << 20)
        m = mmap.mmap(-1, size, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        m.madvise(mmap.MADV_HUGEPAGE)
        raw = torch.frombuffer(m, dtype=torch.uint8)
        raw[::4096].zero_()  # fault the pages in after the advice
        err = torch.cuda.cudart().cudaHostRegister(raw.data_ptr(), size, 0)
        if int(err) != 0:
            raise RuntimeError("cudaHostRegister failed: %s" % err)
        self.keep.append((m, raw))
        return raw[:nbytes].view(dtype).view(shape)

    def release(self):
        for m, raw in self.keep:
            self.torch.cuda.cudart().cudaHostUnregister(raw.data_ptr())
        self.keep.clear()


def anon_huge_kb():
    """AnonHugePages of /proc/meminfo in kB (None where unreadable)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("AnonHugePages:"):
                    return int(line.split()[1])
    except OSError:
        pass
    return None


def pipeline_schedule(origin, marks):
    """Summary of the end-to-end pipeline from its timing events (ms after
    `origin`): per problem-step the input copies, the wait for the previous
    problem's step, the step and the output copies; and the SMs' idle time
    between consecutive steps (a step that waits for its own input copies,
    or for nothing, shows up there)."""
    rows = [[origin.elapsed_time(e) for e in ev] for ev in marks]
    h2d = [r[1] - r[0] for r in rows]
    wait = [r[2] - r[1] for r in rows]
    step = [r[3] - r[2] for r in rows]
    d2h = [r[4] - r[3] for r in rows]
    starts = sorted((r[2], r[3]) for r in rows)
    gaps = [max(0.0, b[0] - a[1]) for a, b in zip(starts, starts[1:])]
    span = starts[-1][1] - starts[0][0] if starts else 0.0

    def mean(x):
        return sum(x) / len(x) if x else None
    return {"h2d_ms": mean(h2d), "h2d_max_ms": max(h2d) if h2d else None,
            "wait_ms": mean(wait), "step_ms": mean(step), "step_max_ms": max(step) if step else None,
            "d2h_ms": mean(d2h), "d2h_max_ms": max(d2h) if d2h else None,
            "gap_between_steps_ms": mean(gaps), "gap_max_ms": max(gaps) if gaps else None,
            "steps_busy_frac": sum(step) / span if span > 0 else None,
            "first_steps_ms": [round(r[2], 2) for r in rows[:6]]}


# ------------------------------------------------------ secondary measures

def _time_steps(torch, g, dt, warm, steps):
    for _ in range(warm):
        g.step(dt, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(g.stream)
    for _ in range(steps):
        g.step(dt, 1)
    b.record(g.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


TG512_STEPS = 500     # run length of the reduced-precision workload


def oracle_tg_plane(n, nu, steps, out_path):
    """FP64 oracle run of the n^3 periodic Taylor-Green workload as its
    n x n x 1 plane: the flow has no z dependence and the scheme keeps it so
    bit for bit, so the plane's arithmetic is that of every z-plane of the
    3-D run.  Saves the interiors of u, v, w, p after `steps` RK2 steps (50
    Jacobi sweeps per solve) with the seconds taken and the threads used."""
    import numpy as np
    from oracle import Oracle, set_threads
    threads = set_threads(0)
    h = (2 * math.pi / n,) * 3
    o = Oracle((n, n, 1), ghost=1, h=h, nu=nu)
    u, p = o.state(workloads.taylor_green((n, n, 1), h=h))
    t0 = time.perf_counter()
    o.run(u, p, workloads.cfl_dt(h), 50, steps)
    el = time.perf_counter() - t0
    np.savez(out_path, u=o.interior(u[0])[0], v=o.interior(u[1])[0], w=o.interior(u[2])[0],
             p=o.interior(p)[0], seconds=el, threads=threads)


def start_oracle_tg_plane(n, nu, steps):
    """Starts oracle_tg_plane in a child process (a new interpreter, so no
    CUDA state is inherited); returns (process, output path)."""
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    code = "import bench; bench.oracle_tg_plane(%d, %r, %d, %r)" % (n, nu, steps, path)
    proc = subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, stdout=subprocess.DEVNULL,
                            stderr=subprocess.PIPE)
    return proc, path


def _rel_err(got, ref, field):
    import numpy as np
    if field == "p":
        got, ref = got - got.mean(), ref - ref.mean()
    return float(np.abs(got - ref).max() / np.abs(ref).max())


def measure_precision(torch, steps):
    """512^3 periodic Taylor-Green (nu = 0.005), two ghost layers (the
    fastest FP32 form: two Jacobi sweeps per launch) with FP32, BF16 and
    FP16 storage: step time over `steps` timed steps after 3 warm-up steps,
    then the run continued to TG512_STEPS steps; plane z = n/3 of every
    field is kept for the error against the FP64 oracle (finish_precision),
    the FP32 run and the exact solution."""
    import numpy as np
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    n = 512
    h = (2 * math.pi / n,) * 3
    dt = workloads.cfl_dt(h)
    nu = workloads.WORKLOADS["tg512"]["nu"]
    plane = workloads.taylor_green((n, n, 1), h=h)
    warm = 3
    out, planes = {}, {}
    for dt_name in ("f32", "bf16", "f16"):
        s = torch.cuda.Stream()
        g = Grid((n, n, n), ghost=2, h=h, dtype=dt_name, stream=s)
        g.set_params(nu, 50, 1.0, 2)
        with torch.cuda.stream(s):
            for arr, c in ((U, "u"), (V, "v"), (W, "w"), (P, "p")):
                src = torch.from_numpy(plane[c][0]).to(g.tdtype).cuda()
                g.interior(arr).copy_(src.expand(n, n, n))
        g.ghost_fill(0b1111)
        g.autotune(None)
        ms = _time_steps(torch, g, dt, warm, steps)
        g.step(dt, TG512_STEPS - warm - steps)
        torch.cuda.synchronize()
        g.check()
        with torch.cuda.stream(s):
            planes[dt_name] = {c: g.interior(a)[n // 3].double().cpu().numpy()
                               for a, c in ((U, "u"), (V, "v"), (W, "w"), (P, "p"))}
            z_same = all(torch.equal(g.interior(a)[0], g.interior(a)[n // 3]) for a in (U, V, P))
        T = TG512_STEPS * dt
        ex = workloads.taylor_green((n, n, 1), h=h, t=T, nu=nu)
        out[dt_name] = {"ms_per_step": ms, "glups": n ** 3 / (ms * 1e-3) / 1e9,
                        "err_vs_exact": {c: _rel_err(planes[dt_name][c], ex[c][0], c)
                                         for c in "uvp"},
                        "max_abs_w": float(np.abs(planes[dt_name]["w"]).max()),
                        "planes_z_independent": bool(z_same),
                        "jacobi_config": g.kernel_config()[0]}
        del g
        torch.cuda.empty_cache()
    for dt_name in ("bf16", "f16"):
        out[dt_name]["err_vs_f32"] = {c: _rel_err(planes[dt_name][c], planes["f32"][c], c)
                                      for c in "uvp"}
        out[dt_name]["speedup_vs_f32"] = out["f32"]["ms_per_step"] / out[dt_name]["ms_per_step"]
    out["workload"] = ("512^3 periodic Taylor-Green, nu=0.005, two ghost layers, %d RK2 steps "
                       "(%d timed after %d warm-up); errors on plane z = n/3 after the %d steps"
                       % (TG512_STEPS, steps, warm, TG512_STEPS))
    return out, planes


def finish_precision(out, planes, proc, path, timeout_s=1500):
    """Adds each storage type's error against the FP64 oracle's plane run
    (e = max |f - f_oracle| / max |f_oracle| per field, p without its mean;
    w as max |w|, which is 0 in the oracle)."""
    import numpy as np
    try:
        _, err = proc.communicate(timeout=timeout_s)
    except subprocess.TimeoutExpired:
        proc.kill()
        out["oracle"] = {"error": "oracle run took longer than %d s" % timeout_s}
        return out
    if proc.returncode != 0:
        out["oracle"] = {"error": err.decode(errors="replace")[-400:]}
        return out
    ref = np.load(path)
    os.remove(path)
    out["oracle"] = {"steps": TG512_STEPS, "seconds": float(ref["seconds"]),
                     "threads": int(ref["threads"]),
                     "run": "FP64 C oracle on the 512x512x1 plane of the same start, "
                            "%d steps, host cores" % TG512_STEPS}
    for dt_name, pl in planes.items():
        e = {c: _rel_err(pl[c], ref[c], c) for c in "uvp"}
        e["w_abs"] = float(np.abs(pl["w"] - ref["w"]).max())
        out[dt_name]["err_vs_oracle"] = e
    out["f32"]["within_1e-3_after_run"] = all(out["f32"]["err_vs_oracle"][c] <= 1e-3
                                              for c in "uvp")
    return out


def measure_blocks(torch):
    """64 uneven periodic blocks (4x4x4, widths U{16..96}, seed 2), curl-noise
    start (seed 3), nu = 0.01: batched (one persistent launch per kernel over
    all blocks, autotuned, graph) against one launch per block per kernel."""
    from paper_1201_2118_gb300 import Grid
    cfg = workloads.WORKLOADS["blocks64"]
    gd, blocks = workloads.block_tiling(seed=cfg["tiling_seed"])
    h = workloads.workload_h("blocks64")
    dt = workloads.cfl_dt(h)
    fl = workloads.random_div_free(gd, h, seed=cfg["ic_seed"])
    per = workloads.split_blocks(fl, blocks)
    cells = gd[0] * gd[1] * gd[2]
    out = {"global_dims": list(gd), "blocks": len(blocks), "cells": cells}
    for ghost in (1, 2):
        res = {}
        for mode in ("batched", "per_block"):
            s = torch.cuda.Stream()
            g = Grid(ghost=ghost, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks],
                     global_dims=gd, stream=s)
            g.set_params(cfg["nu"], cfg["jacobi_iters"], 1.0, 2 * ghost)
            g.upload_blocks(per)
            g.autotune(None)
            g.set_launch_mode(mode == "per_block")
            l0 = g.launches
            ms = _time_steps(torch, g, dt, 3, 10)
            res[mode] = {"ms_per_step": ms, "glups": cells / (ms * 1e-3) / 1e9,
                         "launches_per_step": (g.launches - l0) / 13}
            del g
        res["speedup_batched_vs_per_block"] = res["per_block"]["ms_per_step"] / res["batched"]["ms_per_step"]
        out["ghost%d_order%d" % (ghost, 2 * ghost)] = res
    return out


def measure_adjoint(torch):
    """128^3 periodic curl-noise start (seed 4), 200 RK2 steps, sqrt(T)
    checkpointing (15): time of the checkpointed forward against the
    backward (segment recomputation + adjoint steps)."""
    from paper_1201_2118_gb300 import Rollout, LU, LV, LW, LP
    cfg = workloads.WORKLOADS["adj128"]
    n = cfg["dims"]
    h = workloads.workload_h("adj128")
    dt = workloads.cfl_dt(h)
    steps = cfg["steps"]
    ro = Rollout(n, h, steps, dt, jacobi_iters=cfg["jacobi_iters"], seg=15)
    g = ro.grid
    fl = workloads.random_div_free(n, h, seed=cfg["seed"])
    u0 = [torch.tensor(fl[c], dtype=torch.float32, device="cuda") for c in "uvw"]
    g.autotune(None)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    times = {"forward": [], "backward": []}
    for rep in range(2):
        a, b, c = ev(), ev(), ev()
        torch.cuda.synchronize()
        a.record(g.stream)
        ro.forward_only(*u0, cfg["nu"])
        b.record(g.stream)
        with torch.cuda.stream(g.stream):
            for arr in (LU, LV, LW):
                g.interior(arr).fill_(1e-3)
            g.interior(LP).zero_()
        g.rollout_backward(dt, steps, ro.seg, ro.store_ptr, ro.nbytes)
        c.record(g.stream)
        torch.cuda.synchronize()
        times["forward"].append(a.elapsed_time(b))
        times["backward"].append(b.elapsed_time(c))
    fwd, bwd = min(times["forward"]), min(times["backward"])
    return {"forward_ms": fwd, "backward_ms": bwd, "backward_vs_forward": bwd / fwd,
            "forward_ms_per_step": fwd / steps, "backward_ms_per_step": bwd / steps,
            "checkpoint_every": ro.seg, "steps": steps, "dims": list(n),
            "note": "backward = recomputation of every segment from its checkpoint + adjoint steps"}


def measure_multigrid(torch):
    """512^3 lid-driven cavity, R = D W / dt with W the seeded cavity noise:
    the pressure equation solved to ||L P - R|| <= 1e-5 ||R|| by V-cycles
    (V(2,2), weighted Jacobi 6/7, all levels down to 2^3), against the
    residual that the same time buys in Jacobi sweeps of the bench's
    configured kernel."""
    from paper_1201_2118_gb300 import Grid, P, R, U, V, W, WU, WV, WW, mask
    n = 512
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    s = torch.cuda.Stream()
    g = Grid((n, n, n), ghost=1, h=h, stream=s)
    g.set_cavity(1.0)
    g.upload(workloads.ldc_noise(n, seed=1))
    with torch.cuda.stream(s):
        for a_, b_ in ((U, WU), (V, WV), (W, WW)):
            g.interior(b_).copy_(g.interior(a_))
    g.ghost_fill(mask(WU, WV, WW))
    g.autotune(None)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def zero_p():
        with torch.cuda.stream(s):
            g.interior(P).zero_()
        g.ghost_fill(mask(P))

    zero_p()
    g.pressure_solve_mg(dt, 1e-5, 30)  # warm-up (graphs, caches)
    zero_p()
    torch.cuda.synchronize()
    a_, b_ = ev(), ev()
    a_.record(s)
    cycles, res = g.pressure_solve_mg(dt, 1e-5, 30)
    b_.record(s)
    torch.cuda.synchronize()
    solve_ms = a_.elapsed_time(b_)
    with torch.cuda.stream(s):
        rnorm = g.interior(R).double().norm().item()
    a_, b_ = ev(), ev()
    a_.record(s)
    g.mg_vcycles(10)
    b_.record(s)
    torch.cuda.synchronize()
    cycle_ms = a_.elapsed_time(b_) / 10
    # Jacobi from the same start for the same time
    zero_p()
    g.jacobi(4)
    torch.cuda.synchronize()
    a_, b_ = ev(), ev()
    a_.record(s)
    g.jacobi(100)
    b_.record(s)
    torch.cuda.synchronize()
    sweep_ms = a_.elapsed_time(b_) / 100
    sweeps = max(2, int(round(solve_ms / sweep_ms / 2)) * 2)
    zero_p()
    _, jres = g.pressure_solve_converged(dt, 0.0, sweeps, sweeps)
    # the cavity step with 50 Jacobi sweeps per stage solve against 2 V-cycles
    steps = {}
    for solver in ("jacobi", "mg"):
        g.upload(workloads.ldc_noise(n, seed=1))
        g.set_pressure_solver(solver, 2)
        ms = _time_steps(torch, g, dt, 3, 10)
        _, _, divmax = g.reduce(0)
        steps[solver] = {"ms_per_step": ms, "glups": n ** 3 / (ms * 1e-3) / 1e9,
                         "max_abs_div_after_13_steps": divmax}
    steps["jacobi"]["solve"] = "50 weighted Jacobi sweeps (omega 1) per stage"
    steps["mg"]["solve"] = "2 V-cycles per stage"
    g.check()
    return {"workload": "512^3 cavity, R = D(cavity noise)/dt", "rtol": 1e-5,
            "steps": steps,
            "cycles": cycles, "solve_ms": solve_ms, "ms_per_vcycle": cycle_ms,
            "rel_residual": res / rnorm, "levels": g.multigrid_levels(),
            "cycle": "V(2,2), weighted Jacobi omega 6/7, 30 sweeps on the coarsest level",
            "jacobi_same_time": {"sweeps": sweeps, "ms_per_sweep": sweep_ms,
                                 "rel_residual": jres / rnorm,
                                 "jacobi_config": g.kernel_config()[0]}}


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
    g.autotune(a.tune_cache)
    jcfg = g.kernel_config()

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
    ms, value = aggregate(ms, cells, dist, "cuda")
    ke, umax, divmax = g.reduce(0)

    # ---- dominant kernel: the Jacobi sweep, timed alone on the grid's stream
    # (a fused launch of kind 5 or 9 does two sweeps; its compulsory traffic is
    # still one read of p and r and one write of p per launch)
    sweeps = 100
    fused = jcfg[0][0] in (5, 9)
    per_launch = 2 if fused else 1
    j0, j1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.jacobi(4)
    torch.cuda.synchronize()
    j0.record(stream)
    g.jacobi(sweeps)
    j1.record(stream)
    torch.cuda.synchronize()
    launch_ms = j0.elapsed_time(j1) / (sweeps // per_launch)
    bytes_per_launch = JACOBI_BYTES_PER_CELL[a.dtype] * cells
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = traffic_for(file_hash(kernel_sources(jcfg[0][0])), cells, jcfg[0])
    kernel_names = {0: "k_jacobi", 1: "k_jacobi_tma", 2: "k_jacobi_direct", 3: "k_jacobi_async",
                    5: "k_jacobi2", 7: "k_jacobi_ws", 9: "k_jacobi2_ws"}
    kname = "%s (%s, config %s, %d^3, %s)" % (
        kernel_names.get(jcfg[0][0], "?"),
        "two fused weighted Jacobi sweeps per launch" if fused else "one weighted Jacobi sweep per launch",
        list(jcfg[0]), n, a.dtype)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                "bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                "sweeps_per_launch": per_launch,
                "peak_source": "%s hbm_gbs (burst copy)" % peak_kind,
                "sweep_glups": per_launch * cells / (launch_ms * 1e-3) / 1e9,
                # single-sweep bytes per sweep time: what the sweeps would move
                # without temporal blocking (equals achieved for one sweep per launch)
                "effective_gbs": per_launch * bytes_per_launch / (launch_ms * 1e-3) / 1e9}
    # the instruction-issue side of the same launch: warp instructions per
    # cell from the ncu record, against 4 issues per SM cycle at the SM
    # clock sampled during the timed steps
    rec = profile_record(file_hash(kernel_sources(jcfg[0][0])), jcfg[0])
    issue = None
    clk_summary = clk.summary()
    if rec is not None and rec.get("warp_instructions_per_cell") and clk_summary.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        inst = rec["warp_instructions_per_cell"] * cells
        ach = inst / (launch_ms * 1e-3)
        pk = 4.0 * sms * clk_summary["sm_mhz"] * 1e6
        issue = {"achieved": ach, "peak": pk, "unit": "warp instructions/s", "frac": ach / pk,
                 "instructions_per_launch": inst,
                 "peak_source": "4 issue slots per SM per cycle x %d SMs x median SM clock %.0f MHz"
                                % (sms, clk_summary["sm_mhz"])}
    roofline["issue"] = issue

    # the plain sweep (one weighted Jacobi sweep per launch, the TMA-staged
    # kernel) on the same grid, for the single-sweep roofline fraction
    if a.dtype == "f32" and fused:
        plain_cfg = (1, 4, 16, 16, 4)
        g.set_kernel_config(jacobi=plain_cfg)
        g.jacobi(4)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        g.jacobi(40)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1) / 40
        roofline["plain_sweep"] = {"kernel": "k_jacobi_tma, config %s" % list(plain_cfg),
                                   "launch_ms": plain_ms,
                                   "achieved": bytes_per_launch / (plain_ms * 1e-3) / 1e9,
                                   "frac": bytes_per_launch / (plain_ms * 1e-3) / 1e9 / peak}
        g.set_kernel_config(jacobi=jcfg[0])
        g.step(dt, 1)  # re-captures the step graph outside any timed region
        torch.cuda.synchronize()

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not a.no_e2e:
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
        hb = HostBuffers(torch, a.e2e_host_mem == "hugepages")
        huge0 = anon_huge_kb()
        host_in = [hb.empty((n, n, n), tdt) for _ in range(4)]
        nf = a.e2e_in_flight
        host_out = [[hb.empty((n, n, n), tdt) for _ in range(4)] for _ in range(nf)]
        huge1 = anon_huge_kb()
        for k, arr in enumerate((U, V, W, P)):
            g.copy_interior(arr, host_out[0][k].data_ptr(), to_device=False)
        torch.cuda.synchronize()
        for k in range(4):
            host_in[k].copy_(host_out[0][k])
        k_e2e = max(3, a.steps // 2)

        def host_step(grid, out):
            for k, arr in enumerate((U, V, W, P)):
                grid.copy_interior(arr, host_in[k].data_ptr(), to_device=True)
            grid.step(dt, 1)
            for k, arr in enumerate((U, V, W, P)):
                grid.copy_interior(arr, out[k].data_ptr(), to_device=False)

        # one problem: copy in, step, copy out, one after the other
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        x0.record(stream)
        for _ in range(k_e2e):
            host_step(g, host_out[0])
        x1.record(stream)
        torch.cuda.synchronize()
        serial_ms, serial_value = aggregate(x0.elapsed_time(x1) / k_e2e, cells, dist, "cuda")

        # nf independent problems in flight, one stream each, copies by the
        # copy engines.  Events chain the input copies and the steps of the
        # problems in turn, so they stay a fraction of a period apart: the
        # others' host transfers run while one problem's step has the SMs.
        # each problem's copies and step are bracketed by timing events, so
        # the pipeline's schedule can be read back: when each input copy,
        # step and output copy ran, and how long the SMs waited between steps
        marks = []

        def piped_step(grid, out, after):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            if after[0] is not None:
                grid.stream.wait_event(after[0])
            ev[0].record(grid.stream)
            for k, arr in enumerate((U, V, W, P)):
                grid.copy_interior(arr, host_in[k].data_ptr(), to_device=True)
            ev[1].record(grid.stream)
            if after[1] is not None:
                grid.stream.wait_event(after[1])
            ev[2].record(grid.stream)
            grid.step(dt, 1)
            ev[3].record(grid.stream)
            for k, arr in enumerate((U, V, W, P)):
                grid.copy_interior(arr, out[k].data_ptr(), to_device=False)
            ev[4].record(grid.stream)
            marks.append(ev)
            return ev[1], ev[3]

        grids = [g]
        for _ in range(nf - 1):
            gx = Grid(dims, ghost=cfg["ghost"], h=h, dtype=a.dtype, stream=torch.cuda.Stream())
            gx.set_cavity(1.0)
            gx.set_params(cfg["nu"], cfg["jacobi_iters"], 1.0, cfg["order"])
            gx.set_kernel_config(jacobi=jcfg[0], stencil=jcfg[1])
            grids.append(gx)
        for grid in grids:
            grid.set_host_copy(a.e2e_copy)
        for grid, out in zip(grids, host_out):  # warm-up: captures the step graphs
            host_step(grid, out)
        torch.cuda.synchronize()
        marks.clear()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        x0.record(stream)
        for grid in grids[1:]:
            grid.stream.wait_event(x0)
        after = (None, None)
        for _ in range(k_e2e):
            for grid, out in zip(grids, host_out):
                after = piped_step(grid, out, after)
        for grid in grids[1:]:
            y = torch.cuda.Event()
            y.record(grid.stream)
            stream.wait_event(y)
        x1.record(stream)
        torch.cuda.synchronize()
        for grid in grids:
            grid.check()
        # every problem took the same step from the same input
        same = all(torch.equal(host_out[0][k], host_out[j][k])
                   for j in range(1, nf) for k in range(4))
        g.set_host_copy("kernel")
        del grids, gx
        torch.cuda.empty_cache()
        hb.release()
        ems, e2e_value = aggregate(x0.elapsed_time(x1) / (nf * k_e2e), cells, dist, "cuda")
        schedule = pipeline_schedule(x0, marks)
        es = host_in[0].element_size()
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 4 * cells * es, "d2h_bytes_per_step": 4 * cells * es,
               "ms_per_step": ems, "steps": nf * k_e2e, "in_flight": nf,
               "outputs_equal": same, "schedule": schedule,
               "host_mem": {"kind": a.e2e_host_mem,
                            "anon_huge_pages_gb": None if huge0 is None or huge1 is None
                            else (huge1 - huge0) / 2 ** 20},
               "api": "per step: cfd_copy_interior (pinned host -> device, u,v,w,p; %s) "
                      "+ cfd_step + cfd_copy_interior (device -> pinned host, u,v,w,p); %d "
                      "independent %d^3 problems, one stream each, their input copies and steps "
                      "chained by events in turn" % (
                          {"engine": "copy engine", "kernel": "pack kernel over the host link",
                           "narrow": "pack kernel on one CTA per eight SMs over the host link"}
                          [a.e2e_copy], nf, n),
               "serial": {"value": serial_value, "ms_per_step": serial_ms, "steps": k_e2e,
                          "in_flight": 1,
                          "api": "the same calls on one problem, pack kernel over the host "
                                 "link, each step's copies and step one after the other"}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = oracle_sample()

    secondary = None
    if rank == 0 and world == 1 and not a.no_secondary:
        del g
        torch.cuda.empty_cache()
        # the oracle's reference run for the precision errors starts after
        # the CPU baseline has been timed and runs beside the GPU work
        oproc, opath = start_oracle_tg_plane(512, workloads.WORKLOADS["tg512"]["nu"],
                                             TG512_STEPS)
        prec, planes = measure_precision(torch, a.precision_steps)
        secondary = {"blocks": measure_blocks(torch),
                     "adjoint": measure_adjoint(torch),
                     "multigrid": measure_multigrid(torch)}
        secondary["precision"] = finish_precision(prec, planes, oproc, opath)

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
                             % (n, cells * (4 if a.dtype == "f32" else 2) / 1e6)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk_summary,
            "check": {"kinetic_energy": ke, "max_abs_u": umax, "max_abs_div": divmax},
            "jacobi_config": jcfg,
            "secondary": secondary,
            "library": os.path.relpath(library_path(), ROOT),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.cuda_connections > 0:  # read when the CUDA context is created
        os.environ["CUDA_DEVICE_MAX_CONNECTIONS"] = str(a.cuda_connections)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
