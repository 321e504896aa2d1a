"""cfd_copy_interior: compact host arrays <-> the padded device layout,
by the pack kernel over the host link or through the staging region (a
copy engine and the pack kernel).  Bitwise checks against the torch view
of the same interior, on a full-vector row width, a row width that is not
a multiple of the 16-byte vector, 16-bit storage and a block set
(per-block copies); and two grids on two streams whose engine copies and
steps interleave, against the same steps taken one grid at a time."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["kernel", "engine", "narrow"])
@pytest.mark.parametrize("dims,dtype,shift", [((64, 20, 7), "f32", 0), ((64, 20, 7), "f32", 1),
                                              ((45, 37, 21), "f32", 0), ((70, 9, 5), "bf16", 0),
                                              ((64, 9, 5), "bf16", 0), ((33, 16, 4), "f16", 0)])
def test_copy_interior_round_trip(dims, dtype, shift, mode):
    """shift 1: the host buffer starts one element past a 16-byte boundary
    (the pack kernels then move elements one by one)."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, P, R
    g = Grid(dims, ghost=1, h=(0.1, 0.1, 0.1), dtype=dtype)
    g.set_host_copy(mode)
    g.fill(float("nan"))
    td = g.tdtype
    rng = np.random.default_rng(3)
    cells = dims[0] * dims[1] * dims[2]
    big = torch.from_numpy(rng.uniform(-1, 1, cells + shift)).to(td).pin_memory()
    src = big[shift:].view(dims[::-1])
    for arr in (U, P):
        g.copy_interior(arr, src.data_ptr(), to_device=True)
        torch.cuda.synchronize()
        assert torch.equal(g.interior(arr).cpu(), src)
    # the ghosts stay as they were (NaN here): only the interior is written
    full = g.array(U).cpu().float()
    assert torch.isnan(full[0]).all() and torch.isnan(full[:, 0]).all()
    # device -> host of a different array
    g.interior(R).copy_(torch.from_numpy(rng.uniform(-2, 2, dims[::-1])).to(td).cuda())
    dst = torch.empty(cells + shift, dtype=td).pin_memory()[shift:].view(dims[::-1])
    g.copy_interior(R, dst.data_ptr(), to_device=False)
    torch.cuda.synchronize()
    assert torch.equal(dst, g.interior(R).cpu())
    g.check()


def test_copy_interior_pageable_host_memory():
    """Host memory that is not page-locked takes the staging path."""
    import torch
    from paper_1201_2118_gb300 import Grid, W
    dims = (45, 37, 21)
    g = Grid(dims, ghost=1, h=(0.1, 0.1, 0.1))
    src = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, dims[::-1])).float()
    assert not src.is_pinned()
    g.copy_interior(W, src.data_ptr(), to_device=True)
    torch.cuda.synchronize()
    assert torch.equal(g.interior(W).cpu(), src)
    back = torch.zeros_like(src)
    g.copy_interior(W, back.data_ptr(), to_device=False)
    torch.cuda.synchronize()
    assert torch.equal(back, src)
    g.check()


def test_copy_interior_block_set():
    import torch
    from paper_1201_2118_gb300 import Grid, V
    gd, blocks = workloads.block_tiling(seed=2, nb=2, lo=9, hi=40)
    g = Grid(ghost=1, h=(0.1, 0.1, 0.1), blocks=[(b["dims"], b["origin"]) for b in blocks],
             global_dims=gd)
    rng = np.random.default_rng(4)
    for b, d in enumerate(x["dims"] for x in blocks):
        src = torch.from_numpy(rng.uniform(-1, 1, d[::-1])).float().pin_memory()
        g.copy_interior(V, src.data_ptr(), to_device=True, block=b)
        torch.cuda.synchronize()
        assert torch.equal(g.interior(V, b).cpu(), src)
        back = torch.empty_like(src).pin_memory()
        g.copy_interior(V, back.data_ptr(), to_device=False, block=b)
        torch.cuda.synchronize()
        assert torch.equal(back, src)
    g.check()


def test_set_host_copy_rejects_unknown_mode():
    from paper_1201_2118_gb300 import CfdError, Grid
    from paper_1201_2118_gb300._lib import call
    g = Grid((16, 16, 16), ghost=1, h=(0.1, 0.1, 0.1))
    with pytest.raises(CfdError) as e:
        call("cfd_set_host_copy", g.handle, 3)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        g.set_host_copy("dma")
    g.check()


@pytest.mark.parametrize("route", ["engine", "narrow"])
def test_two_grids_pipelined_copies_equal_serial_steps(route):
    """Two independent cavity problems on two streams: each step copies its
    inputs in (engine or narrow route), steps and copies u, v, w, p out, with the
    other grid's copies and step in flight.  Results are bitwise those of
    the same steps taken one grid after the other with the kernel route."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    n = 48
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    init = [workloads.ldc_noise(n, seed=s) for s in (1, 2)]
    src = [[torch.from_numpy(f[c]).float().pin_memory() for c in "uvwp"] for f in init]

    def run(mode, streams):
        grids = []
        for k in range(2):
            with torch.cuda.stream(streams[k]):
                g = Grid((n, n, n), ghost=1, h=h, stream=streams[k])
                g.set_cavity()
                g.set_params(1e-3, 30, 1.0, 2)
                g.set_host_copy(mode)
                grids.append(g)
        out = [[torch.empty((n, n, n)).pin_memory() for _ in range(4)] for _ in range(2)]
        torch.cuda.synchronize()
        for step in range(3):
            for k in range(2):
                g = grids[k]
                for c, arr in enumerate((U, V, W, P)):
                    g.copy_interior(arr, src[k][c].data_ptr(), to_device=True)
                g.step(dt, 1)
                for c, arr in enumerate((U, V, W, P)):
                    g.copy_interior(arr, out[k][c].data_ptr(), to_device=False)
            torch.cuda.synchronize()
        for g in grids:
            g.check()
        return out

    cur = torch.cuda.current_stream()
    serial = run("kernel", [cur, cur])
    piped = run(route, [torch.cuda.Stream(), torch.cuda.Stream()])
    for k in range(2):
        for c in range(4):
            assert torch.equal(piped[k][c], serial[k][c]), (k, c)
        assert not torch.equal(serial[k][0], src[k][0])
