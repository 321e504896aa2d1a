"""Failure detection on the GPU without a GPU fault, and checkpoint/resume.

* Memory: binding less than cfd_memory_bytes gives CFD_ENOMEM; a grid whose
  arrays need terabytes makes cfd_alloc_memory's cudaMalloc fail, and that
  comes back as CFD_ENOMEM (not an exception, not a sticky CUDA error).
* Device waits: the self-test kernel waits on an mbarrier that nothing
  completes through the same bounded wait as the TMA-staged Jacobi kernels;
  the wait runs out after its limit, the kernel sets the device error flag
  and returns, cfd_check reports CFD_ETIMEOUT, and the context and the grid
  stay usable.  No trap, no bad address, no endless loop.  While the flag
  is set the TMA-staged sweep kernels do no work; binding memory again
  clears it.
* Checkpoint/resume: the state saved from one grid (u, v, w, p through the
  host-copy entry point, t and the step counter) and restored into a fresh
  grid continues bit for bit like the uninterrupted run.
"""
import ctypes
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _create(dims, ghost=1):
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    g = ctypes.c_void_p()
    st = L.cfd_grid_create(_lib.ints(*dims), ghost, _lib.doubles(1, 1, 1), 0, None, ctypes.byref(g))
    assert st == 0, L.cfd_last_error()
    nbytes = ctypes.c_size_t()
    assert L.cfd_memory_bytes(g, ctypes.byref(nbytes)) == 0
    return L, g, nbytes.value


def test_bind_too_little_memory_is_enomem():
    import torch
    L, g, need = _create((24, 20, 16))
    try:
        mem = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
        base = mem.data_ptr() + (-mem.data_ptr()) % 256
        st = L.cfd_bind_memory(g, ctypes.c_void_p(base), need - 256)
        assert st == 2, st
        assert b"need" in L.cfd_last_error()
        # nothing bound: work is refused with CFD_ESTATE, not attempted
        assert L.cfd_ghost_fill(g, 0xF) == 4
        assert L.cfd_bind_memory(g, ctypes.c_void_p(base), need) == 0
        assert L.cfd_ghost_fill(g, 0xF) == 0
        assert L.cfd_check(g) == 0
        torch.cuda.synchronize()
    finally:
        assert L.cfd_grid_destroy(g) == 0


def test_failed_device_allocation_is_reported_not_raised():
    """3000^3 cells x 16 arrays x 4 bytes is about 1.7 TB, beyond the
    device: cudaMalloc refuses it and cfd_alloc_memory returns CFD_ENOMEM.
    The CUDA context stays clean, so another grid works right after."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, P, mask
    L, g, need = _create((3000, 3000, 3000))
    try:
        assert need > 1.5e12
        st = L.cfd_alloc_memory(g)
        assert st == 2, st
        assert b"cudaMalloc" in L.cfd_last_error()
        assert L.cfd_check(g) == 0          # no memory bound: nothing to check, no error
        assert L.cfd_ghost_fill(g, 0xF) == 4
    finally:
        assert L.cfd_grid_destroy(g) == 0
    small = Grid((16, 12, 8), ghost=1)
    small.upload({c: np.ones((8, 12, 16)) for c in "uvwp"})
    small.ghost_fill(mask(U, V, W, P))
    small.check()
    torch.cuda.synchronize()
    assert float(small.array(U).float().sum()) == small.array(U).numel()


@pytest.mark.parametrize("form", [0, 1])
def test_device_wait_runs_out_and_check_reports_timeout(form):
    import time
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, P, mask, _lib
    L = _lib.lib()
    g = Grid((32, 16, 8), ghost=1)
    g.upload({c: np.full((8, 16, 32), 0.5) for c in "uvwp"})
    g.check()
    t0 = time.perf_counter()
    g.selftest_wait_timeout(form)
    st = L.cfd_check(g.handle)            # synchronises with the self-test
    waited = time.perf_counter() - t0
    assert st == 7, (st, L.cfd_last_error())
    assert b"device error flag 2" in L.cfd_last_error()
    assert 1.5 < waited < 30.0, waited   # the wait's limit is 2 s of %globaltimer
    # the context and the grid keep working; the flag keeps being reported
    g.ghost_fill(mask(U, V, W, P))
    torch.cuda.synchronize()
    assert float(g.interior(U).float().mean()) == 0.5
    assert L.cfd_check(g.handle) == 7
    # binding memory again clears the flag
    assert L.cfd_bind_memory(g.handle, ctypes.c_void_p(g.mem.data_ptr() + g._shift), g.nbytes) == 0
    assert L.cfd_check(g.handle) == 0
    assert L.cfd_selftest_wait_timeout(g.handle, 2) == 1


@pytest.mark.parametrize("jacobi", [(9, 4, 16, 16, 6), (7, 4, 16, 32, 8), (1, 4, 16, 16, 4)])
def test_sweeps_do_no_work_once_a_wait_gave_up(jacobi):
    """A TMA-staged sweep launch that finds the device error flag set does
    nothing (a failed solve then costs one wait limit, not one per launch):
    after the self-test has set the flag, four sweeps leave P as it was;
    once memory is bound again they run."""
    import torch
    from paper_1201_2118_gb300 import Grid, P, _lib
    L = _lib.lib()
    n = (64, 32, 16)
    g = Grid(n, ghost=1, h=tuple(1.0 / d for d in n))
    g.set_cavity(1.0)
    g.set_kernel_config(jacobi=jacobi)
    g.set_params(1e-3, 10, 1.0, 2)
    g.upload(workloads.ldc_noise(n, seed=1))
    g.step(1e-3, 1)                      # R, P and its ghosts from a full step
    g.check()
    p0 = g.download(P)
    assert np.isfinite(p0).all()
    g.selftest_wait_timeout(0)
    assert L.cfd_check(g.handle) == 7
    g.jacobi(4)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.download(P), p0)
    assert L.cfd_check(g.handle) == 7
    assert L.cfd_bind_memory(g.handle, ctypes.c_void_p(g.mem.data_ptr() + g._shift), g.nbytes) == 0
    g.jacobi(4)
    g.check()
    p1 = g.download(P)
    assert np.isfinite(p1).all() and np.abs(p1 - p0).max() > 0


@pytest.mark.parametrize("case", ["cavity", "periodic_tg"])
def test_checkpoint_restore_continues_bitwise(case):
    """Run A: n1 steps, save, n2 more.  Run B: a fresh grid restored from
    the save, n2 steps.  Fields, time and step counter agree exactly."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, P, mask
    n = (48, 40, 32)
    if case == "cavity":
        h = tuple(1.0 / d for d in n)
        start, nu = workloads.ldc_noise(n, seed=1), 1e-3
    else:
        h = tuple(2 * math.pi / d for d in n)
        start, nu = workloads.taylor_green(n, h=h), 0.01
    dt = workloads.cfl_dt(h)
    n1, n2 = 3, 4

    def make():
        g = Grid(n, ghost=1, h=h)
        if case == "cavity":
            g.set_cavity(1.0)
        g.set_params(nu, 20, 1.0, 2)
        return g

    a = make()
    a.upload(start)
    a.step(dt, n1)
    saved = {}
    for arr in (U, V, W, P):
        host = torch.empty(n[::-1], dtype=torch.float32, pin_memory=True)
        a.copy_interior(arr, host.data_ptr(), to_device=False)
        saved[arr] = host
    torch.cuda.synchronize()
    t_saved, step_saved = a.time
    assert step_saved == n1 and t_saved == pytest.approx(n1 * dt)
    a.step(dt, n2)
    torch.cuda.synchronize()
    ref = {arr: a.interior(arr).clone() for arr in (U, V, W, P)}

    b = make()
    for arr in (U, V, W, P):
        b.copy_interior(arr, saved[arr].data_ptr(), to_device=True)
    b.ghost_fill(mask(U, V, W, P))
    b.set_time(t_saved, step_saved)
    b.step(dt, n2)
    torch.cuda.synchronize()
    a.check()
    b.check()
    for arr in (U, V, W, P):
        assert torch.equal(b.interior(arr), ref[arr]), arr
    assert b.time == a.time
