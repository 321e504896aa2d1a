"""The allocation-free reduction entry point, checked against cfd_reduce.

cfd_reduce_velocity_noalloc serves callers that cannot allocate device
memory when they want the diagnostics (inside a stream capture, under a
foreign pool allocator, or in a loop that must not synchronise the device);
its scratch is a static device array of the library.  This file is collected
last so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


DTYPES = {"f32": 0, "bf16": 1, "f16": 2}


def _noalloc(lib, ints, doubles, g, dims, h, out, arrays, dtype):
    ptrs = [ctypes.c_void_p(g.interior(a).data_ptr()) for a in arrays]
    sz, sy, _ = g.array(arrays[0]).stride()
    return lib.cfd_reduce_velocity_noalloc(ptrs[0], ptrs[1], ptrs[2], DTYPES[dtype], ints(*dims),
                                           sy, sz,
                                           doubles(*h), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(g.stream.cuda_stream))


@pytest.mark.parametrize("dtype", sorted(DTYPES))
def test_noalloc_reduce_matches_grid_reduce_on_two_calls(dtype):
    """Every storage type: the same three quantities as the grid's own
    reduction, on two calls in a row (the second sees the first call's
    partial sums left in the shared static array)."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, SET_U, _lib
    L = _lib.lib()
    dims, h = (45, 37, 21), (0.3, 0.2, 0.1)
    rng = np.random.default_rng(21)
    g = Grid(dims, ghost=1, h=h, dtype=dtype)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        g.upload({c: rng.uniform(-1, 1, dims[::-1]) * (call + 1) for c in "uvwp"})
        ke, umax, divmax = g.reduce(SET_U)
        st = _noalloc(L, _lib.ints, _lib.doubles, g, dims, h, out, (U, V, W), dtype)
        assert st == 0, L.cfd_noalloc_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ke, rel=1e-12), call
        assert got[1] == pytest.approx(umax, rel=1e-12), call
        assert got[2] == pytest.approx(divmax, rel=1e-12), call
        assert got[3] == 0.0


def test_noalloc_rejects_more_planes_than_its_static_scratch():
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    fake = ctypes.c_void_p(256)
    st = L.cfd_reduce_velocity_noalloc(fake, fake, fake, 0, _lib.ints(8, 8, 5000), 8, 64,
                                       _lib.doubles(1, 1, 1), fake, None)
    assert st == 1
    assert b"static scratch" in L.cfd_noalloc_last_error()
