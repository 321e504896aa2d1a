"""Conservative (flux) form of the advection term on the CUDA path against
the FP64 oracle's flux form, element by element, through the C ABI.

Same bar as the advective form: e(f) = max|f_gpu - f_ref| / max|f_ref|
<= 1e-5 per stage or step for FP32 storage, half an ulp of the output (plus
FP32 rounding) for 16-bit storage; at the full 512^3 size, sampled boxes
against the oracle fed the device's own neighbours, and the momentum and
energy identities of the scheme.
"""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import make_pair, rel_err, rounded

pytestmark = pytest.mark.gpu

DIMS = (70, 37, 21)


def rand(dims, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return {c: scale * rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}


def _stage2(o, grid, dims, seed, dtype="f32"):
    """Stage-2 form out = 1/2 U + 1/2 U1 + c F(U1) with distinct inputs."""
    from paper_1201_2118_gb300 import U1, V1, W1, SET_U, SET_U1, SET_W, mask
    f1 = rounded(rand(dims, seed), dtype)
    for k, a in enumerate((U1, V1, W1)):
        grid.interior(a).copy_(grid.torch.from_numpy(f1["uvw"[k]]).to(grid.tdtype).cuda())
    grid.ghost_fill(mask(U1, V1, W1))
    u1 = [o.ghost_fill(o.embed(f1["uvw"[k]]), k) for k in range(3)]
    return u1


@pytest.mark.parametrize("stencil", [(8, 16, 2), (4, 8, 4), (8, 32, 0), (4, 32, 0), (8, 32, 1),
                                     (4, 16, 1), (8, 7, 1), (4, 32, 3), (4, 5, 3)])
@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_flux_stage_variants_match_oracle(stencil, bc):
    from paper_1201_2118_gb300 import WU, WV, WW, SET_U, SET_U1, SET_W
    o, grid, u, p = make_pair(DIMS, bc=bc, nu=0.03, fields=rand(DIMS, 7), form="flux")
    grid.set_kernel_config(stencil=stencil)
    assert grid.kernel_config()[1] == stencil
    u1 = _stage2(o, grid, DIMS, 8)
    grid.stage(0.5, SET_U, 0.5, SET_U1, 0.013, SET_W)
    ref = o.stage(0.5, u, 0.5, u1, 0.013)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(ref[k])) < 1e-5, k


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_flux_rhs_eval(bc):
    from paper_1201_2118_gb300 import WU, WV, WW
    o, grid, u, p = make_pair((45, 37, 21), bc=bc, nu=0.05, fields=rand((45, 37, 21), 3),
                              form="flux")
    grid.rhs_eval()
    F = o.stage(0.0, None, 0.0, u, 1.0)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(F[k])) < 1e-5, k


def test_flux_differs_from_advective_form():
    """The two forms agree only for a divergence-free field: on a random one
    the device results differ by far more than the tolerance."""
    from paper_1201_2118_gb300 import WU
    res = []
    for form in ("advective", "flux"):
        o, grid, u, p = make_pair(DIMS, nu=0.0, fields=rand(DIMS, 9), form=form)
        grid.rhs_eval()
        res.append(grid.download(WU))
    assert rel_err(res[1], res[0]) > 1e-2


@pytest.mark.parametrize("dtype,bits", [("bf16", 8), ("f16", 11)])
def test_flux_16bit_stage(dtype, bits):
    """16-bit storage, FP32 arithmetic, one rounding of the output."""
    from paper_1201_2118_gb300 import WU, WV, WW, SET_U, SET_U1, SET_W
    dims = (150, 77, 40)
    o, grid, u, p = make_pair(dims, h=(0.11, 0.13, 0.17), fields=rand(dims, 4), dtype=dtype,
                              nu=0.05, form="flux")
    u1 = _stage2(o, grid, dims, 5, dtype)
    grid.stage(0.5, SET_U, 0.5, SET_U1, 0.01, SET_W)
    ref = o.stage(0.5, u, 0.5, u1, 0.01)
    half_ulp = 2.0 ** -bits
    for k, a in enumerate((WU, WV, WW)):
        got, r = grid.download(a), o.interior(ref[k])
        assert (np.abs(got - r) <= half_ulp * np.abs(r) + 2e-6 * np.abs(r).max()).all(), k


@pytest.mark.parametrize("jacobi", [(0, 4, 4, 32, 4), (9, 4, 16, 16, 6)])
def test_flux_cavity_steps(jacobi):
    """Lid-driven cavity (Re 1000, CFL 0.2) in the flux form: 1 step at 1e-5,
    10 steps at 1e-4 (velocity) / 1e-3 (pressure)."""
    from gpu_helpers import compare_state
    n = 32
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), bc="cavity", h=h, nu=1e-3,
                              fields=workloads.ldc_noise(n, seed=1), form="flux")
    grid.set_kernel_config(jacobi=jacobi)
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, 50)
    compare_state(o, grid, u, p, 1e-5, 1e-5, "flux ldc step 1")
    grid.step(dt, 9)
    o.run(u, p, dt, 50, 9)
    compare_state(o, grid, u, p, 1e-4, 1e-3, "flux ldc step 10")


def test_flux_blockset_step_equals_global_oracle():
    """64 uneven periodic blocks in one persistent launch, flux form, against
    the single-block oracle on the global grid."""
    from oracle import Oracle
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    gd, blocks = workloads.block_tiling(seed=2, lo=8, hi=20)
    h = (2 * math.pi / 64,) * 3
    fl = rounded(workloads.random_div_free(gd, h, seed=3))
    o = Oracle(gd, ghost=1, h=h, nu=0.01, form="flux")
    u, p = o.state(fl)
    grid = Grid(ghost=1, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
    grid.fill(float("nan"))
    grid.set_params(0.01, 20, 1.0, 2)
    grid.set_advection("flux")
    grid.upload_blocks(workloads.split_blocks(fl, blocks))
    dt = workloads.cfl_dt(h)
    grid.step(dt, 2)
    o.run(u, p, dt, 20, 2)
    for k, a in enumerate((U, V, W, P)):
        got = np.full(gd[::-1], np.nan)
        for b, blk in enumerate(blocks):
            (nx, ny, nz), (ox, oy, oz) = blk["dims"], blk["origin"]
            got[oz:oz + nz, oy:oy + ny, ox:ox + nx] = grid.download(a, block=b)
        ref = o.interior(u[k] if k < 3 else p)
        assert rel_err(got, ref, remove_mean=(k == 3)) < 1e-5, k


def test_flux_form_rejects_order4():
    from paper_1201_2118_gb300 import CfdError, Grid
    g = Grid((16, 16, 16), ghost=2, h=(0.1, 0.1, 0.1))
    g.set_params(0.01, 10, 1.0, 4)
    with pytest.raises(CfdError) as e:
        g.set_advection("flux")
    assert e.value.status == 1
    g.set_params(0.01, 10, 1.0, 2)
    g.set_advection("flux")
    with pytest.raises(CfdError) as e:
        g.set_params(0.01, 10, 1.0, 4)
    assert e.value.status == 1
    g.check()


def _wrap_box(t, start, size):
    """Periodic sub-box (with one ghost layer) of a device (nz, ny, nx) tensor."""
    import torch
    idx = []
    for a in range(3):
        n = t.shape[a]
        idx.append(torch.tensor([(start[a] + q) % n for q in range(-1, size + 1)],
                                device=t.device))
    return t.index_select(0, idx[0]).index_select(1, idx[1]).index_select(2, idx[2])


@pytest.mark.parametrize("stencil", [(8, 32, 1), (4, 64, 3)])
def test_flux_full_size_sampled_boxes_and_momentum(stencil):
    """512^3 periodic grid in one launch (the ring kernel, and the pair kernel
    with two cells per thread): sampled 6^3 boxes (interior, faces,
    corners of the periodic wrap) against the oracle fed the device's own
    neighbour values, and the momentum identity sum_p F_c = 0 (viscous and
    advective sums both telescope) over all 134M points of each component."""
    import torch
    from oracle import Oracle
    from paper_1201_2118_gb300 import Grid, U, V, W, WU, WV, WW, mask
    n = 512
    h = (2 * math.pi / n, 2 * math.pi / n, 1.3 * math.pi / n)
    nu = 0.02
    grid = Grid((n, n, n), ghost=1, h=h)
    grid.set_params(nu, 10, 1.0, 2)
    grid.set_advection("flux")
    grid.set_kernel_config(stencil=stencil)
    gen = torch.Generator(device="cuda").manual_seed(12)
    for a in (U, V, W):
        grid.interior(a).copy_(torch.rand((n, n, n), generator=gen, device="cuda") * 2 - 1)
    grid.ghost_fill(mask(U, V, W))
    grid.rhs_eval()
    grid.check()
    vel = [grid.interior(a) for a in (U, V, W)]
    F = [grid.interior(a) for a in (WU, WV, WW)]
    for c in range(3):
        total = F[c].double().sum().item()
        scale = F[c].double().abs().sum().item()
        assert abs(total) < 1e-6 * scale, (c, total, scale)
    s = 6
    starts = [(0, 0, 0), (n - 3, n - 3, n - 3), (n - s, 17, 250), (101, n - 1, 7), (300, 200, 100)]
    o = Oracle((s, s, s), ghost=1, h=h, nu=nu, form="flux")
    for st in starts:
        # (z, y, x) box starts; the oracle gets the device's neighbours as ghosts
        box = [_wrap_box(v, st, s).double().cpu().numpy() for v in vel]
        ref = o.rhs(*[np.ascontiguousarray(b) for b in box])
        for c in range(3):
            got = _wrap_box(F[c], st, s)[1:-1, 1:-1, 1:-1].double().cpu().numpy()
            assert rel_err(got, o.interior(ref[c])) < 1e-5, (st, c)


def test_flux_energy_identity_on_div_free_field():
    """A discretely divergence-free field (curl of an edge potential), nu = 0:
    the advection term does no work, sum_c sum_p u_c F_c = 0, up to the
    FP32 rounding of the stored field and of F."""
    from paper_1201_2118_gb300 import Grid, U, V, W, WU, WV, WW
    dims = (128, 96, 80)
    h = (0.05, 0.06, 0.07)
    fl = rounded(workloads.random_div_free(dims, h, seed=6))
    grid = Grid(dims, ghost=1, h=h)
    grid.set_params(0.0, 10, 1.0, 2)
    grid.set_advection("flux")
    grid.upload(fl)
    grid.rhs_eval()
    work = sum((grid.interior(a).double() * grid.interior(b).double()).sum().item()
               for a, b in ((U, WU), (V, WV), (W, WW)))
    scale = sum((grid.interior(a).double() * grid.interior(b).double()).abs().sum().item()
                for a, b in ((U, WU), (V, WV), (W, WW)))
    assert abs(work) < 1e-5 * scale, (work, scale)
