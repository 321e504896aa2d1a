"""The seeded input generators: the block tiling is a rectilinear partition
with widths in range that the library's host-side tiling check accepts;
cutting global fields into blocks and putting them back is the identity;
the cavity start holds its wall-normal faces at zero; the Taylor-Green
start is the closed form at its staggered points."""
import math

import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("seed,nb,lo,hi", [(2, 4, 16, 96), (2, 4, 8, 20), (7, 3, 5, 9), (1, 1, 4, 4)])
def test_block_tiling_is_a_rectilinear_partition(seed, nb, lo, hi):
    gd, blocks = workloads.block_tiling(seed=seed, nb=nb, lo=lo, hi=hi)
    assert len(blocks) == nb ** 3
    cover = np.zeros(gd[::-1], dtype=np.int32)
    for k, b in enumerate(blocks):
        (nx, ny, nz), (ox, oy, oz) = b["dims"], b["origin"]
        assert all(lo <= n <= hi for n in b["dims"])
        bx, by, bz = b["index"]
        assert k == (bz * nb + by) * nb + bx  # x fastest
        cover[oz:oz + nz, oy:oy + ny, ox:ox + nx] += 1
    assert (cover == 1).all()
    # the same draw again: the generator is seeded
    assert workloads.block_tiling(seed=seed, nb=nb, lo=lo, hi=hi) == (gd, blocks)


def test_library_accepts_the_tiling():
    """cfd_blockset_create's tiling check passes (on a host without a GPU the
    call then stops at the first device call with CFD_ECUDA)."""
    import ctypes
    from paper_1201_2118_gb300 import _lib
    gd, blocks = workloads.block_tiling(seed=2)
    L = _lib.lib()
    out = ctypes.c_void_p()
    dims = [x for b in blocks for x in b["dims"]]
    origin = [x for b in blocks for x in b["origin"]]
    st = L.cfd_blockset_create(len(blocks), _lib.ints(*dims), _lib.ints(*origin), _lib.ints(*gd),
                               1, _lib.doubles(0.1, 0.1, 0.1), 0, None, ctypes.byref(out))
    assert st in (0, 3), L.cfd_last_error()
    if st == 0:
        assert L.cfd_grid_destroy(out) == 0


def test_split_blocks_round_trip():
    gd, blocks = workloads.block_tiling(seed=3, nb=3, lo=4, hi=9)
    rng = np.random.default_rng(0)
    fields = {c: rng.standard_normal(gd[::-1]) for c in "uvwp"}
    parts = workloads.split_blocks(fields, blocks)
    for c in "uvwp":
        back = np.full(gd[::-1], np.nan)
        for b, part in zip(blocks, parts):
            (nx, ny, nz), (ox, oy, oz) = b["dims"], b["origin"]
            assert part[c].shape == (nz, ny, nx) and part[c].flags.c_contiguous
            back[oz:oz + nz, oy:oy + ny, ox:ox + nx] = part[c]
        assert np.array_equal(back, fields[c])


def test_ldc_noise_walls_and_range():
    f = workloads.ldc_noise((12, 9, 7), seed=1, amp=1e-3)
    assert f["u"].shape == (7, 9, 12)
    assert (f["u"][:, :, -1] == 0).all() and (f["v"][:, -1, :] == 0).all()
    assert (f["w"][-1, :, :] == 0).all() and (f["p"] == 0).all()
    for c in "uvw":
        assert np.abs(f[c]).max() <= 1e-3
    assert not np.array_equal(f["u"], workloads.ldc_noise((12, 9, 7), seed=2)["u"])


def test_taylor_green_closed_form_at_staggered_points():
    n = 16
    h = (2 * math.pi / n,) * 3
    f = workloads.taylor_green((n, n, n), h, amp=1.0)
    # u at x-faces ((i+1)h, (j+1/2)h), v at y-faces ((i+1/2)h, (j+1)h)
    i, j = 3, 5
    xu, yu = (i + 1) * h[0], (j + 0.5) * h[1]
    xv, yv = (i + 0.5) * h[0], (j + 1) * h[1]
    assert f["u"][2, j, i] == pytest.approx(math.sin(xu) * math.cos(yu), abs=1e-14)
    assert f["v"][2, j, i] == pytest.approx(-math.cos(xv) * math.sin(yv), abs=1e-14)
    assert (f["w"] == 0).all()
