"""cfd_copy_interior: compact host arrays <-> the padded device layout,
through the staging region and the pack kernel.  Bitwise checks against
the torch view of the same interior, on a full-vector row width, a row
width that is not a multiple of the 16-byte vector, 16-bit storage and a
block set (per-block copies)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,dtype", [((64, 20, 7), "f32"), ((45, 37, 21), "f32"),
                                        ((70, 9, 5), "bf16"), ((33, 16, 4), "f16")])
def test_copy_interior_round_trip(dims, dtype):
    import torch
    from paper_1201_2118_gb300 import Grid, U, P, R
    g = Grid(dims, ghost=1, h=(0.1, 0.1, 0.1), dtype=dtype)
    g.fill(float("nan"))
    td = g.tdtype
    rng = np.random.default_rng(3)
    src = torch.from_numpy(rng.uniform(-1, 1, dims[::-1])).to(td).pin_memory()
    for arr in (U, P):
        g.copy_interior(arr, src.data_ptr(), to_device=True)
        torch.cuda.synchronize()
        assert torch.equal(g.interior(arr).cpu(), src)
    # the ghosts stay as they were (NaN here): only the interior is written
    full = g.array(U).cpu().float()
    assert torch.isnan(full[0]).all() and torch.isnan(full[:, 0]).all()
    # device -> host of a different array
    g.interior(R).copy_(torch.from_numpy(rng.uniform(-2, 2, dims[::-1])).to(td).cuda())
    dst = torch.empty(dims[::-1], dtype=td).pin_memory()
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
