"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Sizes span several tiles with ragged tails (tiles are 32 x 8 cells for the
point kernels and (32 vx) x ty for the Jacobi sweep); every array starts as
NaN so a read of an unfilled ghost or pad cell shows up.  Floating-point
tolerance: e(f) = max|f_gpu - f_ref| / max|f_ref| <= 1e-5 per step for FP32
(pressure compared without its mean), <= 1e-3 after a full 100-step run.
"""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import make_pair, compare_state, rel_err, rounded, tg_fields

pytestmark = pytest.mark.gpu

RAGGED = (45, 37, 21)


def rand_fields(dims, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return {c: scale * rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}


@pytest.mark.parametrize("g", [1, 2])
def test_ghost_fill_periodic_bitwise(g):
    from paper_1201_2118_gb300 import U, V, W, P
    o, grid, u, p = make_pair(RAGGED, ghost=g, fields=rand_fields(RAGGED, 1))
    for k, a in enumerate((U, V, W)):
        np.testing.assert_array_equal(grid.download(a, ghosts=True), u[k])
    np.testing.assert_array_equal(grid.download(P, ghosts=True), p)


def test_ghost_fill_cavity():
    from paper_1201_2118_gb300 import U, V, W, P
    o, grid, u, p = make_pair(RAGGED, bc="cavity", fields=rand_fields(RAGGED, 2))
    for k, a in enumerate((U, V, W)):
        np.testing.assert_allclose(grid.download(a, ghosts=True), u[k], rtol=0, atol=2.5e-7)
    np.testing.assert_array_equal(grid.download(P, ghosts=True), p)


def test_blockset_ghosts_equal_global_periodic_wrap():
    """64 uneven blocks: every block's ghost cells equal the periodic global
    field around it (np.pad wrap of the global array)."""
    from paper_1201_2118_gb300 import Grid, U, mask
    gd, blocks = workloads.block_tiling(seed=2, lo=8, hi=24)
    rng = np.random.default_rng(5)
    glob = rounded({"u": rng.standard_normal(gd[::-1])})["u"]
    g = 2
    grid = Grid(ghost=g, h=(0.1, 0.1, 0.1), blocks=[(b["dims"], b["origin"]) for b in blocks],
                global_dims=gd)
    grid.fill(float("nan"))
    per = workloads.split_blocks({"u": glob}, blocks)
    for b, f in enumerate(per):
        grid.upload(f, block=b, fill_ghosts=False)
    grid.ghost_fill(mask(U))
    padded = np.pad(glob, g, mode="wrap")
    for b, blk in enumerate(blocks):
        (nx, ny, nz), (ox, oy, oz) = blk["dims"], blk["origin"]
        ref = padded[oz:oz + nz + 2 * g, oy:oy + ny + 2 * g, ox:ox + nx + 2 * g]
        np.testing.assert_array_equal(grid.download(U, block=b, ghosts=True), ref)


@pytest.mark.parametrize("order,g", [(2, 1), (4, 2)])
def test_rhs_eval(order, g):
    from paper_1201_2118_gb300 import WU, WV, WW
    fl = rand_fields(RAGGED, 3)
    o, grid, u, p = make_pair(RAGGED, ghost=g, order=order, nu=0.05, fields=fl)
    grid.rhs_eval()
    F = o.rhs(*u)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(F[k])) < 1e-5


@pytest.mark.parametrize("misalign", [0, 1])
def test_rhs_eval_into_caller_buffers(misalign):
    """cfd_rhs_eval with out_dev: the compact interiors equal WU, WV, WW bit
    for bit, also into buffers that start 4 bytes past a 16-byte boundary
    (element-wise path) and on a block set (blocks one after the other)."""
    import torch
    from paper_1201_2118_gb300 import Grid, WU, WV, WW
    fl = rand_fields(RAGGED, 5)
    o, grid, u, p = make_pair(RAGGED, nu=0.05, fields=fl)
    nx, ny, nz = RAGGED
    cells = nx * ny * nz
    bufs = [torch.full((cells + 4,), float("nan"), device="cuda") for _ in range(3)]
    outs = [b[misalign:misalign + cells] for b in bufs]
    grid.rhs_eval(out=outs)
    torch.cuda.synchronize()
    for t, a in zip(outs, (WU, WV, WW)):
        assert torch.equal(t.view(nz, ny, nx), grid.interior(a))
    F = o.rhs(*u)
    assert rel_err(outs[0].view(nz, ny, nx).double().cpu().numpy(), o.interior(F[0])) < 1e-5
    blocks = [((20, 16, 12), (0, 0, 0)), ((13, 16, 12), (20, 0, 0))]
    bs = Grid(ghost=1, h=(0.2, 0.2, 0.2), blocks=blocks, global_dims=(33, 16, 12))
    bs.set_params(0.05, 10, 1.0, 2)
    rng = np.random.default_rng(6)
    for b, (d, _) in enumerate(blocks):
        bs.upload({c: rng.uniform(-1, 1, d[::-1]) for c in "uvwp"}, block=b, fill_ghosts=False)
    bs.ghost_fill(0b1111)
    total = sum(d[0] * d[1] * d[2] for d, _ in blocks)
    outs = [torch.full((total + 4,), float("nan"), device="cuda")[misalign:misalign + total]
            for _ in range(3)]
    bs.rhs_eval(out=outs)
    torch.cuda.synchronize()
    for t, a in zip(outs, (WU, WV, WW)):
        off = 0
        for b, (d, _) in enumerate(blocks):
            n = d[0] * d[1] * d[2]
            assert torch.equal(t[off:off + n].view(d[2], d[1], d[0]), bs.interior(a, b))
            off += n


def test_rhs_eval_cavity():
    from paper_1201_2118_gb300 import WU, WV, WW
    fl = rand_fields(RAGGED, 4)
    o, grid, u, p = make_pair(RAGGED, bc="cavity", nu=0.05, fields=fl)
    grid.rhs_eval()
    F = o.stage(0.0, None, 0.0, u, 1.0)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(F[k])) < 1e-5


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_stage2_combine(bc):
    """out = 1/2 U + 1/2 U1 + c F(U1) with distinct inputs."""
    from paper_1201_2118_gb300 import WU, WV, WW, U1, V1, W1, SET_U, SET_U1, SET_W, mask
    fl = rand_fields(RAGGED, 5)
    o, grid, u, p = make_pair(RAGGED, bc=bc, nu=0.02, fields=fl)
    f1 = rounded(rand_fields(RAGGED, 6))
    for k, a in enumerate((U1, V1, W1)):
        grid.interior(a).copy_(grid.torch.from_numpy(f1["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(U1, V1, W1))
    u1 = [o.ghost_fill(o.embed(f1["uvw"[k]]), k) for k in range(3)]
    grid.stage(0.5, SET_U, 0.5, SET_U1, 0.013, SET_W)
    ref = o.stage(0.5, u, 0.5, u1, 0.013)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(ref[k])) < 1e-5


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
@pytest.mark.parametrize("iters", [0, 1, 7])
def test_pressure_solve(bc, iters):
    from paper_1201_2118_gb300 import P, R, WU, WV, WW, mask
    fl = rand_fields(RAGGED, 7)
    o, grid, u, p = make_pair(RAGGED, bc=bc, fields=fl)
    w = rounded(rand_fields(RAGGED, 8))
    for k, a in enumerate((WU, WV, WW)):
        grid.interior(a).copy_(grid.torch.from_numpy(w["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    c_dt = 0.037
    res = grid.pressure_solve(c_dt, iters, residual=True)
    r = o.divergence(wo, c_dt)
    assert rel_err(grid.download(R), o.interior(r)) < 1e-5
    o.jacobi(p, r, iters)
    assert rel_err(grid.download(P), o.interior(p)) < 1e-5
    assert res == pytest.approx(o.residual(p, r), rel=1e-4)


@pytest.mark.parametrize("cfg", [(0, 4, 4, 32, 4), (1, 4, 16, 16, 4), (9, 4, 16, 16, 6)])
def test_converged_pressure_solve(cfg):
    """Residual-controlled sweeps stop at the first check (every 6 sweeps)
    where ||L p - r|| <= rtol ||r||; the oracle, run in the same chunks,
    stops at the same check (or one chunk away when FP32 rounding puts a
    check right at the threshold), the result matches the oracle after
    the same number of sweeps, and the reported residual is the oracle's."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    bc = "cavity" if cfg[0] == 9 else "periodic"
    fl = rand_fields(RAGGED, 17)
    o, grid, u, p = make_pair(RAGGED, bc=bc, fields=fl)
    grid.set_kernel_config(jacobi=cfg)
    w = rounded(rand_fields(RAGGED, 18))
    if bc == "cavity":  # no flux through the walls: D w has zero mean (solvable)
        w["u"][:, :, -1] = 0.0
        w["v"][:, -1, :] = 0.0
        w["w"][-1, :, :] = 0.0
    for k, a in enumerate((WU, WV, WW)):
        grid.interior(a).copy_(grid.torch.from_numpy(w["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    c_dt, rtol, chunk, cap = 0.037, 0.2, 6, 600
    iters, res = grid.pressure_solve_converged(c_dt, rtol, cap, chunk)
    r = o.divergence(wo, c_dt)
    target = rtol * np.sqrt(np.sum(o.interior(r) ** 2))
    ref_iters, hist = 0, [o.residual(p, r)]
    p_at = {0: p.copy()}
    while hist[-1] > target and ref_iters < cap:
        o.jacobi(p, r, chunk)
        ref_iters += chunk
        hist.append(o.residual(p, r))
        p_at[ref_iters] = p.copy()
    assert iters % chunk == 0 and 0 < iters < cap
    assert abs(iters - ref_iters) <= chunk
    if iters not in p_at:
        o.jacobi(p, r, iters - ref_iters)
        p_at[iters] = p.copy()
    assert rel_err(grid.download(P), o.interior(p_at[iters])) < 1e-4
    assert res == pytest.approx(o.residual(p_at[iters], r), rel=1e-3)
    assert res <= target * (1 + 1e-3)
    grid.check()


def test_converged_pressure_solve_cap_equals_fixed_sweeps():
    """rtol 0 runs exactly max_iters sweeps: the same bits as
    cfd_pressure_solve with that sweep count."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    res = []
    for conv in (False, True):
        o, grid, u, p = make_pair(RAGGED, bc="periodic", fields=rand_fields(RAGGED, 19))
        w = rounded(rand_fields(RAGGED, 20))
        for k, a in enumerate((WU, WV, WW)):
            grid.interior(a).copy_(grid.torch.from_numpy(w["uvw"[k]]).float().cuda())
        grid.ghost_fill(mask(WU, WV, WW))
        if conv:
            n, _ = grid.pressure_solve_converged(0.05, 0.0, 14, 4)
            assert n == 14
        else:
            grid.pressure_solve(0.05, 14)
        res.append(grid.download(P))
    np.testing.assert_array_equal(res[0], res[1])


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_project(bc):
    from paper_1201_2118_gb300 import U1, V1, W1, WU, WV, WW, SET_U1, mask
    fl = rand_fields(RAGGED, 9)
    o, grid, u, p = make_pair(RAGGED, bc=bc, fields=fl)
    w = rounded(rand_fields(RAGGED, 10))
    for k, a in enumerate((WU, WV, WW)):
        grid.interior(a).copy_(grid.torch.from_numpy(w["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    grid.project(0.021, SET_U1)
    ref = o.project(wo, p, 0.021)
    for k, a in enumerate((U1, V1, W1)):
        o.ghost_fill(ref[k], k)
        got = grid.download(a, ghosts=True)
        assert rel_err(got, ref[k]) < 1e-5


def test_reduce_and_residual():
    from paper_1201_2118_gb300 import SET_U
    fl = rand_fields(RAGGED, 11)
    o, grid, u, p = make_pair(RAGGED, fields=fl)
    ke, um, dm = grid.reduce(SET_U)
    rke, rum, rdm = o.reduce(u)
    assert ke == pytest.approx(rke, rel=1e-12)
    assert um == rum
    assert dm == pytest.approx(rdm, rel=1e-6)


def test_tg32_one_step_and_full_run():
    """32^3 periodic Taylor-Green, nu=0.01, CFL 0.2, 50 Jacobi sweeps per
    solve: e <= 1e-5 after one step, <= 1e-3 after 100 steps (graph replay)."""
    n = 32
    h = (2 * math.pi / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), h=h, nu=0.01, fields=tg_fields((n, n, n)))
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, 50)
    compare_state(o, grid, u, p, 1e-5, 1e-5, "step 1")
    grid.step(dt, 99)
    o.run(u, p, dt, 50, 99)
    errs = compare_state(o, grid, u, p, 1e-3, 1e-3, "step 100")
    t, s = grid.time
    assert s == 100 and t == pytest.approx(100 * dt)
    print("tg32 errors after 100 steps", errs)


def test_rk_stages_equal_graph_step():
    """rk_step(1) + rk_step(2) gives bitwise the same state as step(dt, 1)."""
    from paper_1201_2118_gb300 import U, V, W, P
    n = (40, 24, 18)
    fl = workloads.random_div_free(n, (0.2, 0.2, 0.2), seed=3)
    o, g1, _, _ = make_pair(n, h=(0.2, 0.2, 0.2), fields=fl, iters=9)
    _, g2, _, _ = make_pair(n, h=(0.2, 0.2, 0.2), fields=fl, iters=9)
    g1.rk_step(1, 0.01)
    g1.rk_step(2, 0.01)
    g2.step(0.01, 1)
    for a in (U, V, W, P):
        np.testing.assert_array_equal(g1.download(a), g2.download(a))


@pytest.mark.parametrize("n,steps", [(32, 20), (48, 3)])
def test_cavity_steps(n, steps):
    """Lid-driven cavity Re=1000 (nu=1e-3), h=1/n, dt from CFL 0.2."""
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), bc="cavity", h=h, nu=1e-3,
                              fields=workloads.ldc_noise(n, seed=1))
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, 50)
    compare_state(o, grid, u, p, 1e-5, 1e-5, "ldc step 1")
    grid.step(dt, steps - 1)
    o.run(u, p, dt, 50, steps - 1)
    compare_state(o, grid, u, p, 1e-4, 1e-3, "ldc step %d" % steps)


@pytest.mark.parametrize("order,g", [(2, 1), (4, 2)])
def test_blockset_step_equals_global_oracle(order, g):
    """64 uneven periodic blocks stepped together agree with the single-block
    oracle on the global grid."""
    from oracle import Oracle
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    gd, blocks = workloads.block_tiling(seed=2, lo=8, hi=20)
    h = (2 * math.pi / 64,) * 3
    fl = rounded(workloads.random_div_free(gd, h, seed=3))
    o = Oracle(gd, ghost=g, h=h, nu=0.01, order=order)
    u, p = o.state(fl)
    grid = Grid(ghost=g, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
    grid.fill(float("nan"))
    grid.set_params(0.01, 20, 1.0, order)
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


@pytest.mark.parametrize("order,g,jacobi", [(2, 1, (0, 4, 4, 32, 4)), (4, 2, (0, 4, 4, 32, 4)),
                                             (4, 2, (9, 4, 16, 16, 6)), (4, 2, (9, 4, 8, 32, 6)),
                                             (4, 2, (9, 2, 16, 16, 6)), (4, 2, (9, 2, 8, 32, 6))])
def test_blockset_workload_tiling_equals_global_oracle(order, g, jacobi):
    """The block-set workload's own tiling: 64 blocks with per-axis widths
    U{16..96} (seed 2), curl-noise start (seed 3), two RK2 steps with 20
    Jacobi sweeps per solve, against the oracle on the global grid.  With
    two ghost layers the two-sweep kernel runs in its periodic form over
    all blocks at once, the ghost launch between its launches copying both
    layers from the neighbouring blocks."""
    from oracle import Oracle
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    gd, blocks = workloads.block_tiling(seed=2)
    h = workloads.workload_h("blocks64")
    fl = rounded(workloads.random_div_free(gd, h, seed=3))
    o = Oracle(gd, ghost=g, h=h, nu=0.01, order=order)
    u, p = o.state(fl)
    grid = Grid(ghost=g, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
    grid.fill(float("nan"))
    grid.set_params(0.01, 20, 1.0, order)
    grid.set_kernel_config(jacobi=jacobi)
    grid.upload_blocks(workloads.split_blocks(fl, blocks))
    dt = workloads.cfl_dt(h)
    grid.step(dt, 2)
    o.run(u, p, dt, 20, 2)
    grid.check()
    for k, a in enumerate((U, V, W, P)):
        got = np.full(gd[::-1], np.nan)
        for b, blk in enumerate(blocks):
            (nx, ny, nz), (ox, oy, oz) = blk["dims"], blk["origin"]
            got[oz:oz + nz, oy:oy + ny, ox:ox + nx] = grid.download(a, block=b)
        ref = o.interior(u[k] if k < 3 else p)
        assert rel_err(got, ref, remove_mean=(k == 3)) < 1e-5, k


def test_nan_watchdog_and_errors():
    from paper_1201_2118_gb300 import CfdError, Grid, U, SET_U
    grid = Grid((16, 16, 16), ghost=1, h=(0.1, 0.1, 0.1))
    grid.upload(rand_fields((16, 16, 16), 12))
    grid.interior(U)[3, 4, 5] = float("inf")
    with pytest.raises(CfdError) as e:
        grid.reduce(SET_U)
    assert e.value.status == 6
    with pytest.raises(CfdError) as e:
        grid.set_params(-1.0)
    assert e.value.status == 1
    grid.check()


@pytest.mark.parametrize("dims,ghost", [((2, 3, 2), 1), ((4, 4, 5), 2), ((2, 2, 2), 1)])
@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_degenerate_small_grids_step(dims, ghost, bc):
    """The smallest grids the ghost width allows (two cells on an axis, a
    periodic neighbour that is the cell itself one over): one step and three
    more against the oracle, ghosts included in the comparison's inputs."""
    rng = np.random.default_rng(21)
    fl = {c: rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}
    o, grid, u, p = make_pair(dims, ghost=ghost, bc=bc, nu=0.05, fields=fl, iters=7,
                              order=2 * ghost)
    dt = 0.05 * min(o.h)
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, 7)
    compare_state(o, grid, u, p, 1e-5, 1e-5, "small step 1")
    grid.step(dt, 3)
    o.run(u, p, dt, 7, 3)
    compare_state(o, grid, u, p, 1e-4, 1e-3, "small step 4")


def test_cavity_full_run_32():
    """The cavity case over a whole run (Re 1000, CFL 0.2, 1000 steps at 32^3)
    against the oracle at the full-run bar (1e-3), with the invariants the
    scheme keeps: wall-normal face values exactly 0 and no net mass flux."""
    n, steps = 32, 1000
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), bc="cavity", h=h, nu=1e-3,
                              fields=workloads.ldc_noise(n, seed=1))
    grid.step(dt, steps)
    o.run(u, p, dt, 50, steps)
    errs = compare_state(o, grid, u, p, 1e-3, 1e-3, "ldc32 step %d" % steps)
    from paper_1201_2118_gb300 import U, V, W
    gu, gv, gw = grid.download(U), grid.download(V), grid.download(W)
    assert (gu[:, :, -1] == 0).all() and (gv[:, -1, :] == 0).all() and (gw[-1, :, :] == 0).all()
    div = ((gu - np.pad(gu, ((0, 0), (0, 0), (1, 0)))[:, :, :-1]) / h[0] +
           (gv - np.pad(gv, ((0, 0), (1, 0), (0, 0)))[:, :-1, :]) / h[1] +
           (gw - np.pad(gw, ((1, 0), (0, 0), (0, 0)))[:-1, :, :]) / h[2])
    assert abs(div.sum()) * h[0] * h[1] * h[2] < 1e-6
    print("ldc32 errors after %d steps" % steps, errs)


def test_cavity_256_first_steps():
    """The 256^3 cavity workload itself: the first two steps against the
    oracle.  u, v and p at the one-step bar (1e-5).  w is the 1e-3 seeded
    noise alone while the lid drives p to O(1): the projection changes w by
    dt dp/dz, and storing p in FP32 already costs ulp(max|p|) dt / h_z in
    absolute terms (one ulp of each of the two values differenced, and as
    much again from the solve's own last-place error), so e(w) is held to
    four times ulp(max|p|) dt / h_z over max|w| (about 3.2e-5 at this step)
    where that exceeds 1e-5."""
    from paper_1201_2118_gb300 import P, W
    n = 256
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), bc="cavity", h=h, nu=1e-3,
                              fields=workloads.ldc_noise(n, seed=1))
    for step, tol_p in ((1, 1e-5), (2, 1e-4)):
        grid.step(dt, 1)
        o.rk2_step(u, p, dt, 50)
        errs = {c: rel_err(grid.download(a), o.interior(u[k]))
                for k, (c, a) in enumerate(zip("uv", (0, 1)))}
        assert max(errs.values()) < 1e-5, (step, errs)
        pmax = np.abs(o.interior(p)).max()
        floor = 4 * np.spacing(np.float32(pmax)) * dt / h[2] / np.abs(o.interior(u[2])).max()
        ew = rel_err(grid.download(W), o.interior(u[2]))
        assert ew < max(1e-5, floor), (step, ew, floor)
        assert rel_err(grid.download(P), o.interior(p), remove_mean=True) < tol_p
        print("ldc256 step", step, errs, "w", ew, "w floor", floor)


def test_cavity_512_first_step_bench_configuration():
    """The bench's own workload and launch configuration: the 512^3 cavity
    with the Jacobi sweeps two per launch (9, 4, 16, 64, 6) and the RHS ring
    (8, 64, 1), one step against the oracle's 512^3 step, cell by cell, with
    the bars of the 256^3 case (w's FP32 pressure floor as there)."""
    from paper_1201_2118_gb300 import P, W
    n = 512
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    o, grid, u, p = make_pair((n, n, n), bc="cavity", h=h, nu=1e-3,
                              fields=workloads.ldc_noise(n, seed=1))
    grid.set_kernel_config(jacobi=(9, 4, 16, 64, 6), stencil=(8, 64, 1))
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, 50)
    errs = {c: rel_err(grid.download(a), o.interior(u[k]))
            for k, (c, a) in enumerate(zip("uv", (0, 1)))}
    assert max(errs.values()) < 1e-5, errs
    pmax = np.abs(o.interior(p)).max()
    floor = 4 * np.spacing(np.float32(pmax)) * dt / h[2] / np.abs(o.interior(u[2])).max()
    ew = rel_err(grid.download(W), o.interior(u[2]))
    assert ew < max(1e-5, floor), (ew, floor)
    assert rel_err(grid.download(P), o.interior(p), remove_mean=True) < 1e-5
    print("ldc512 step 1", errs, "w", ew, "w floor", floor)


def test_tg512_against_oracle_plane():
    """The reduced-precision workload's FP32 run: 512^3 periodic
    Taylor-Green, nu = 0.005, two ghost layers (two Jacobi sweeps per launch,
    periodic form), against the oracle on the 512 x 512 x 1 plane, whose
    arithmetic is that of every z-plane (the flow has no z dependence and the
    scheme keeps it so bit for bit).  e <= 1e-5 after one step and after
    five; w stays 0 and every z-plane of the device run is the same."""
    import torch
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    from oracle import Oracle
    n = 512
    h = (2 * math.pi / n,) * 3
    dt = workloads.cfl_dt(h)
    nu = workloads.WORKLOADS["tg512"]["nu"]
    plane = rounded(workloads.taylor_green((n, n, 1), h=h))
    o = Oracle((n, n, 1), ghost=1, h=h, nu=nu)
    u, p = o.state(plane)
    grid = Grid((n, n, n), ghost=2, h=h)
    grid.set_params(nu, 50, 1.0, 2)
    grid.set_kernel_config(jacobi=(9, 4, 16, 64, 6))
    with torch.cuda.stream(grid.stream):
        for arr, c in ((U, "u"), (V, "v"), (W, "w"), (P, "p")):
            src = torch.from_numpy(plane[c][0]).float().cuda()
            grid.interior(arr).copy_(src.expand(n, n, n))
    grid.ghost_fill(0b1111)
    done = 0
    for upto in (1, 5):
        grid.step(dt, upto - done)
        o.run(u, p, dt, 50, upto - done)
        done = upto
        torch.cuda.synchronize()
        for arr in (U, V, P):
            full = grid.interior(arr)
            assert torch.equal(full, full[:1].expand_as(full)), (upto, arr)
        assert float(grid.interior(W).abs().max()) == 0.0
        errs = {c: rel_err(grid.interior(a)[n // 3].double().cpu().numpy(),
                           o.interior(f)[0], remove_mean=(c == "p"))
                for c, a, f in (("u", U, u[0]), ("v", V, u[1]), ("p", P, p))}
        assert max(errs.values()) <= 1e-5, (upto, errs)
        print("tg512 step", upto, errs)


@pytest.mark.parametrize("solver,jacobi,stencil", [("jacobi", (9, 4, 16, 64, 6), (8, 64, 1)),
                                                   ("jacobi", (7, 4, 16, 64, 8), (4, 32, 3)),
                                                   ("mg", (9, 4, 16, 64, 6), (8, 32, 1))])
def test_steps_are_deterministic(solver, jacobi, stencil):
    """The same steps on two grids give the same bits: no kernel of the step
    (mbarrier rings, persistent tile walks, the one-CTA multigrid bottom,
    fixed-order reductions) depends on timing."""
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    n = 192
    h = (1.0 / n,) * 3
    dt = workloads.cfl_dt(h)
    res = []
    for _ in range(2):
        g = Grid((n, n, n), ghost=1, h=h)
        g.set_cavity(1.0)
        g.set_params(1e-3, 30, 1.0, 2)
        g.set_kernel_config(jacobi=jacobi, stencil=stencil)
        if solver == "mg":
            g.set_pressure_solver("mg", 2)
        g.upload(workloads.ldc_noise(n, seed=1))
        g.step(dt, 5)
        ke = g.reduce(0)
        res.append(([g.interior(a).clone() for a in (U, V, W, P)], ke))
        g.check()
    for a, b in zip(res[0][0], res[1][0]):
        assert grid_equal(a, b)
    assert res[0][1] == res[1][1]


def grid_equal(a, b):
    import torch
    return bool(torch.equal(a, b))


def test_largest_grid_1024():
    """A 1024^3 cavity (17 G elements in the arena, offsets far past 2^32):
    ten sweeps as five two-sweep launches equal ten single sweeps bit for
    bit, and one full step stays finite with its wall-normal faces exactly
    zero and finite FP64 reductions."""
    import torch
    from paper_1201_2118_gb300 import Grid, P, R, U, V, W, mask
    n = 1024
    h = (1.0 / n,) * 3
    res = []
    for cfg in ((9, 4, 16, 64, 6), (0, 4, 8, 32, 4)):
        g = Grid((n, n, n), ghost=1, h=h)
        g.set_cavity(1.0)
        g.set_params(1e-3, 10, 1.0, 2)
        g.set_kernel_config(jacobi=cfg, stencil=(8, 64, 1))
        gen = torch.Generator(device="cuda").manual_seed(41)
        g.interior(P).copy_(torch.rand((n, n, n), generator=gen, device="cuda") - 0.5)
        g.interior(R).copy_(torch.rand((n, n, n), generator=gen, device="cuda") - 0.5)
        g.ghost_fill(mask(P, R))
        g.jacobi(10)
        res.append(g.interior(P)[::37, ::41, ::43].clone())
        if cfg[0] == 9:
            full = g.interior(P).clone()
        else:
            assert torch.equal(full, g.interior(P))
            del full
            for a in (U, V, W):
                g.interior(a).copy_(1e-3 * (torch.rand((n, n, n), generator=gen, device="cuda") - 0.5))
            g.interior(P).zero_()
            g.ghost_fill(mask(U, V, W, P))
            g.step(workloads.cfl_dt(h), 1)
            ke, umax, divmax = g.reduce(0)
            assert math.isfinite(ke) and math.isfinite(divmax) and 0 < umax < 2
            assert not bool((g.interior(U)[:, :, -1] != 0).any())
            assert not bool((g.interior(V)[:, -1, :] != 0).any())
            assert not bool((g.interior(W)[-1, :, :] != 0).any())
        g.check()
        del g
        torch.cuda.empty_cache()
    assert torch.equal(res[0], res[1])
