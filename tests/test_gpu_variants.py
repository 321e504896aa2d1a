"""Kernel variants (register/shuffle and TMA-staged Jacobi sweeps, tile
shapes), the autotuner, and reduced-precision storage, against the oracle.

Reduced precision: with BF16 (FP16) storage every stored value is rounded to
nearest with 8 (11) significant bits, so one kernel call fed the device's
own rounded inputs may differ from the FP64 oracle by half an ulp of its
output, 2^-8 (2^-11) relative, plus the FP32 arithmetic error; that is the
bound checked here.
"""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import make_pair, rel_err, rounded

pytestmark = pytest.mark.gpu

JACOBI_CONFIGS = [
    (0, 4, 8, 32, 4), (0, 4, 4, 16, 4), (0, 4, 16, 64, 4), (0, 2, 8, 32, 4), (0, 1, 8, 16, 4),
    (1, 4, 8, 32, 4), (1, 4, 8, 64, 6), (1, 4, 16, 32, 4), (1, 4, 16, 128, 6), (1, 2, 8, 16, 4),
    (1, 2, 16, 32, 4), (1, 4, 4, 16, 6), (1, 4, 4, 32, 4), (2, 4, 4, 1, 0), (2, 4, 4, 2, 0),
    (2, 4, 8, 1, 0), (2, 4, 2, 4, 0), (2, 2, 4, 2, 0), (2, 1, 8, 1, 0),
    (3, 4, 4, 32, 5), (3, 4, 8, 16, 6), (3, 4, 2, 32, 6), (3, 4, 4, 64, 6),
    (5, 4, 4, 16, 0), (5, 4, 8, 32, 0),
    (7, 4, 4, 16, 6), (7, 4, 8, 32, 8), (7, 4, 16, 128, 6), (7, 4, 4, 7, 8),
    (7, 2, 8, 32, 6), (7, 2, 16, 9, 6),
]
SIZES = [(45, 37, 21), (150, 77, 40)]


def cfg_id(c):
    return "k" + "_".join(map(str, c))


def rand(dims, seed):
    rng = np.random.default_rng(seed)
    return {c: rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}


@pytest.mark.parametrize("cfg", JACOBI_CONFIGS, ids=cfg_id)
@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_jacobi_variant_matches_oracle(cfg, dims, bc):
    from paper_1201_2118_gb300 import P, R, WU, WV, WW, mask
    o, g, u, p = make_pair(dims, bc=bc, fields=rand(dims, 1))
    g.set_kernel_config(jacobi=cfg)
    assert g.kernel_config()[0] == cfg
    w = rounded(rand(dims, 2))
    for k, a in enumerate((WU, WV, WW)):
        g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    g.pressure_solve(0.05, 7)
    r = o.divergence(wo, 0.05)
    o.jacobi(p, r, 7)
    assert rel_err(g.download(P), o.interior(p)) < 1e-5
    # ghost-on-write: the first ghost layer of P equals the oracle's fill on
    # the faces (edges and corners are never read by 7-point operators)
    gp = g.download(P, ghosts=True)
    for ax in range(3):
        for side in (0, -1):
            sl = [slice(1, -1)] * 3
            sl[2 - ax] = side
            assert rel_err(gp[tuple(sl)], p[tuple(sl)]) < 1e-5
    g.check()


@pytest.mark.parametrize("cfg", [(1, 4, 8, 32, 4), (1, 2, 8, 16, 4), (0, 1, 8, 16, 4),
                                 (2, 4, 4, 2, 0), (2, 1, 8, 1, 0), (3, 4, 4, 32, 5),
                                 (7, 4, 8, 32, 6), (7, 2, 8, 32, 6), (7, 2, 16, 64, 6)], ids=cfg_id)
def test_jacobi_variant_on_block_set(cfg):
    from oracle import Oracle
    from paper_1201_2118_gb300 import Grid, P, R, WU, WV, WW, mask
    gd, blocks = workloads.block_tiling(seed=2, lo=16, hi=40)
    h = (0.11, 0.13, 0.17)
    rng = np.random.default_rng(3)
    w = rounded({c: rng.uniform(-1, 1, gd[::-1]) for c in "uvw"})
    p0 = rounded({"p": rng.uniform(-1, 1, gd[::-1])})["p"]
    g = Grid(ghost=1, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
    g.fill(float("nan"))
    g.set_kernel_config(jacobi=cfg)
    per = workloads.split_blocks({"u": w["u"], "v": w["v"], "w": w["w"], "p": p0}, blocks)
    for b, f in enumerate(per):
        g.upload({"p": f["p"]}, block=b, fill_ghosts=False)
        for k, a in enumerate((WU, WV, WW)):
            g.interior(a, b).copy_(g.torch.from_numpy(f["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW, P))
    g.pressure_solve(0.03, 6)
    o = Oracle(gd, ghost=1, h=h)
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    po = o.ghost_fill(o.embed(p0), 3)
    r = o.divergence(wo, 0.03)
    o.jacobi(po, r, 6)
    ref = o.interior(po)
    got = np.full(gd[::-1], np.nan)
    for b, blk in enumerate(blocks):
        (nx, ny, nz), (ox, oy, oz) = blk["dims"], blk["origin"]
        got[oz:oz + nz, oy:oy + ny, ox:ox + nx] = g.download(P, block=b)
    assert rel_err(got, ref) < 1e-5
    g.check()


def test_autotune_keeps_state_and_caches(tmp_path):
    from paper_1201_2118_gb300 import Grid, P, U
    n = (96, 80, 64)
    h = tuple(2 * math.pi / d for d in n)
    fl = workloads.random_div_free(n, h, seed=7)
    g = Grid(n, ghost=1, h=h)
    g.upload(fl)
    before_p, before_u = g.download(P), g.download(U)
    cache = str(tmp_path / "tune.txt")
    us = g.autotune(cache)
    assert us > 0
    j, s = g.kernel_config()
    np.testing.assert_array_equal(g.download(P), before_p)
    np.testing.assert_array_equal(g.download(U), before_u)
    text = open(cache).read()
    assert "jacobi=%d,%d,%d,%d,%d" % j in text
    g2 = Grid(n, ghost=1, h=h)
    g2.upload(fl)
    assert g2.autotune(cache) == pytest.approx(us, rel=1e-3)
    assert g2.kernel_config() == (j, s)
    # results do not depend on the chosen variant
    dt = workloads.cfl_dt(h)
    g.step(dt, 2)
    g3 = Grid(n, ghost=1, h=h)
    g3.upload(fl)
    g3.step(dt, 2)
    assert rel_err(g.download(U), g3.download(U)) < 1e-6


@pytest.mark.parametrize("dtype,bits", [("bf16", 8), ("f16", 11)])
def test_reduced_precision_sweep_and_stage(dtype, bits):
    """One Jacobi sweep and one stage-1 update with 16-bit storage, fed the
    device's rounded inputs, within half an ulp of the output."""
    from oracle import Oracle
    from paper_1201_2118_gb300 import P, R, WU, WV, WW
    dims = (150, 77, 40)
    h = (0.11, 0.13, 0.17)
    fl = rand(dims, 4)
    o, g, u, p = make_pair(dims, h=h, fields=fl, dtype=dtype, nu=0.05, iters=1)
    half_ulp = 2.0 ** -bits
    # stage 1 update: W = U + dt F(U)
    g.stage(0.0, 0, 1.0, 0, 0.01, 1)
    ref = o.stage(0.0, None, 1.0, u, 0.01)
    for k, a in enumerate((WU, WV, WW)):
        got, r = g.download(a), o.interior(ref[k])
        assert (np.abs(got - r) <= half_ulp * np.abs(r) + 2e-6 * np.abs(r).max()).all()
    # one sweep from the device's own R (already rounded) and P
    g.ghost_fill(0b1110000)
    g.pressure_solve(0.02, 0)
    r_dev = o.ghost_fill(o.embed(g.download(R)), 3)
    p_dev = o.ghost_fill(o.embed(g.download(P)), 3)
    g.jacobi(1)
    out = o.jacobi_sweep(p_dev, r_dev)
    got, r = g.download(P), o.interior(out)
    assert (np.abs(got - r) <= half_ulp * np.abs(r) + 2e-6 * np.abs(r).max()).all()


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_reduced_precision_taylor_green_error_is_stated(dtype):
    """64^3 Taylor-Green, 20 steps: the 16-bit run stays finite and within
    the storage precision of the FP32 run (error measured, bound loose)."""
    from paper_1201_2118_gb300 import Grid, U, V, P
    n = (64, 64, 64)
    h = tuple(2 * math.pi / d for d in n)
    dt = workloads.cfl_dt(h)
    tg = workloads.taylor_green(n, h=h)
    res = {}
    for dt_name in ("f32", dtype):
        g = Grid(n, ghost=1, h=h, dtype=dt_name)
        g.set_params(0.005, 50, 1.0, 2)
        g.upload(tg)
        g.step(dt, 20)
        res[dt_name] = [g.download(a) for a in (U, V, P)]
        ke, umax, _ = g.reduce(0)
        assert math.isfinite(ke)
    errs = [rel_err(res[dtype][k], res["f32"][k], remove_mean=(k == 2)) for k in range(3)]
    print(dtype, "vs f32 after 20 steps (u, v, p):", errs)
    assert max(errs[:2]) < 0.05


@pytest.mark.parametrize("g", [1, 2])
def test_per_block_launch_mode_is_bitwise_identical(g):
    """The batched form (one persistent launch over the tiles of all 64
    blocks) and the baseline (one launch per block per kernel) compute the
    same cells with the same arithmetic."""
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    gd, blocks = workloads.block_tiling(seed=2, lo=8, hi=24)
    h = (2 * math.pi / 64,) * 3
    fl = workloads.random_div_free(gd, h, seed=3)
    per = workloads.split_blocks(fl, blocks)
    res = []
    for mode in (False, True):
        grid = Grid(ghost=g, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
        grid.set_params(0.01, 10, 1.0, 2 * g)
        grid.set_launch_mode(mode)
        grid.upload_blocks(per)
        grid.step(workloads.cfl_dt(h), 2)
        res.append([grid.download(a, block=b) for b in range(len(blocks)) for a in (U, V, W, P)])
    for x, y in zip(*res):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("cfg", [(9, 4, 16, 16, 6), (9, 2, 8, 16, 6)], ids=cfg_id)
def test_two_sweep_blockset_equals_per_block_single_sweeps(cfg):
    """With two ghost layers the batched form takes the Jacobi sweeps two
    per launch over all blocks; the per-block baseline takes them one per
    launch and block.  Two steps with 11 sweeps per solve (an odd count:
    five two-sweep launches and a single one) agree bit for bit."""
    from paper_1201_2118_gb300 import Grid, U, V, W, P
    gd, blocks = workloads.block_tiling(seed=2, lo=8, hi=24)
    h = (2 * math.pi / 64,) * 3
    fl = workloads.random_div_free(gd, h, seed=3)
    per = workloads.split_blocks(fl, blocks)
    res = []
    for mode in (False, True):
        grid = Grid(ghost=2, h=h, blocks=[(b["dims"], b["origin"]) for b in blocks], global_dims=gd)
        grid.set_params(0.01, 11, 1.0, 4)
        grid.set_kernel_config(jacobi=cfg)
        grid.set_launch_mode(mode)
        grid.upload_blocks(per)
        l0 = grid.launches
        grid.step(workloads.cfl_dt(h), 2)
        res.append([grid.download(a, block=b) for b in range(len(blocks)) for a in (U, V, W, P)])
        if mode:  # single sweeps, one launch per block
            assert grid.launches - l0 >= 2 * 2 * 11 * len(blocks)
        grid.check()
    for x, y in zip(*res):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("cfg", [(3, 8, 4, 32, 5), (3, 8, 8, 16, 6), (3, 8, 2, 64, 6),
                                 (1, 4, 8, 32, 6), (2, 4, 4, 2, 0), (7, 4, 8, 32, 8),
                                 (9, 4, 16, 16, 6), (9, 4, 8, 32, 5), (9, 2, 16, 16, 6)],
                         ids=cfg_id)
def test_16bit_jacobi_variants_agree_with_register_sweep(dtype, cfg):
    """Every 16-bit sweep variant computes the same FP32 expression and
    rounds once, so it matches the register sweep to one rounding step."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    dims = (300, 77, 40)
    half_ulp = 2.0 ** (-8 if dtype == "bf16" else -11)
    res = []
    for c in ((0, 4, 4, 32, 4), cfg):
        o, g, u, p = make_pair(dims, bc="cavity", fields=rand(dims, 5), dtype=dtype)
        g.set_kernel_config(jacobi=c)
        assert g.kernel_config()[0] == c
        w = rand(dims, 6)
        for k, a in enumerate((WU, WV, WW)):
            g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).to(g.tdtype).cuda())
        g.ghost_fill(mask(WU, WV, WW))
        g.pressure_solve(0.05, 5)
        res.append(g.download(P, ghosts=True))
        g.check()
    a, b = res
    inner = (slice(1, -1),) * 3
    assert (np.abs(a[inner] - b[inner]) <= 2 * half_ulp * np.abs(b[inner]) + 1e-30).all()


@pytest.mark.parametrize("stencil", [(8, 16, 2), (4, 8, 4), (8, 32, 0), (8, 32, 1), (4, 16, 1), (8, 7, 1),
                                     (4, 32, 3), (4, 7, 3)])
@pytest.mark.parametrize("order,g,bc", [(2, 1, "periodic"), (4, 2, "periodic"), (2, 1, "cavity")])
def test_stage_variants_match_oracle(stencil, order, g, bc):
    """RHS + stage kernels (L1 neighbours or shared-memory box) against the
    oracle, stage-2 form with distinct inputs, ragged multi-tile grid."""
    from paper_1201_2118_gb300 import WU, WV, WW, U1, V1, W1, SET_U, SET_U1, SET_W, mask
    dims = (70, 37, 21)
    o, grid, u, p = make_pair(dims, ghost=g, order=order, bc=bc, nu=0.03, fields=rand(dims, 7))
    grid.set_kernel_config(stencil=stencil)
    assert grid.kernel_config()[1] == stencil
    f1 = rounded(rand(dims, 8))
    for k, a in enumerate((U1, V1, W1)):
        grid.interior(a).copy_(grid.torch.from_numpy(f1["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(U1, V1, W1))
    u1 = [o.ghost_fill(o.embed(f1["uvw"[k]]), k) for k in range(3)]
    grid.stage(0.5, SET_U, 0.5, SET_U1, 0.013, SET_W)
    ref = o.stage(0.5, u, 0.5, u1, 0.013)
    for k, a in enumerate((WU, WV, WW)):
        assert rel_err(grid.download(a), o.interior(ref[k])) < 1e-5


@pytest.mark.parametrize("cfg", [(5, 4, 4, 16, 0), (5, 4, 8, 7, 0), (5, 4, 4, 64, 0)])
@pytest.mark.parametrize("bc", ["periodic", "cavity"])
@pytest.mark.parametrize("iters", [1, 2, 7, 10])
@pytest.mark.parametrize("dims", [(128, 40, 21), (256, 16, 3)])
def test_fused_two_sweep_launches_match_oracle(cfg, bc, iters, dims):
    """Temporal blocking (two sweeps per launch, boundary-mapped reads) on
    grids it applies to, odd counts included, against the oracle; ghost
    faces of the result as the oracle's fill."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    o, g, u, p = make_pair(dims, bc=bc, fields=rand(dims, 11))
    g.set_kernel_config(jacobi=cfg)
    w = rounded(rand(dims, 12))
    for k, a in enumerate((WU, WV, WW)):
        g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    g.pressure_solve(0.05, iters)
    r = o.divergence(wo, 0.05)
    o.jacobi(p, r, iters)
    assert rel_err(g.download(P), o.interior(p)) < 1e-5
    gp = g.download(P, ghosts=True)
    for ax in range(3):
        for side in (0, -1):
            sl = [slice(1, -1)] * 3
            sl[2 - ax] = side
            assert rel_err(gp[tuple(sl)], p[tuple(sl)]) < 1e-5
    g.check()


@pytest.mark.parametrize("cfg", [(9, 4, 16, 16, 7), (9, 4, 8, 7, 5), (9, 4, 8, 64, 6), (9, 4, 16, 3, 6),
                                 (9, 2, 16, 16, 6), (9, 2, 8, 7, 6)],
                         ids=cfg_id)
@pytest.mark.parametrize("iters", [1, 2, 5, 10])
@pytest.mark.parametrize("dims", [(128, 40, 21), (150, 37, 21), (300, 16, 2), (70, 5, 33)])
def test_two_sweep_ws_launches_match_oracle(cfg, iters, dims):
    """Warp-specialised two-sweep launches (walls on all faces) on full and
    ragged tiles, chunk edges at the walls and inside, odd counts, against
    the oracle; the result's first ghost layer as the oracle's fill."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    o, g, u, p = make_pair(dims, bc="cavity", fields=rand(dims, 13))
    g.set_kernel_config(jacobi=cfg)
    assert g.kernel_config()[0] == cfg
    w = rounded(rand(dims, 14))
    for k, a in enumerate((WU, WV, WW)):
        g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    g.pressure_solve(0.05, iters)
    r = o.divergence(wo, 0.05)
    o.jacobi(p, r, iters)
    assert rel_err(g.download(P), o.interior(p)) < 1e-5
    gp = g.download(P, ghosts=True)
    for ax in range(3):
        for side in (0, -1):
            sl = [slice(1, -1)] * 3
            sl[2 - ax] = side
            assert rel_err(gp[tuple(sl)], p[tuple(sl)]) < 1e-5
    g.check()


@pytest.mark.parametrize("cfg", [(9, 4, 16, 16, 6), (9, 4, 8, 7, 5), (9, 4, 16, 64, 7), (9, 2, 16, 16, 6),
                                 (9, 2, 8, 7, 6)], ids=cfg_id)
@pytest.mark.parametrize("iters", [1, 2, 5, 10])
@pytest.mark.parametrize("dims", [(128, 40, 21), (150, 37, 21), (70, 5, 33)])
def test_two_sweep_ws_periodic_ghost2_matches_oracle(cfg, iters, dims):
    """The periodic form of the two-sweep launch (every face periodic, two
    ghost layers): the first sweep also taken on the ghost layer from the
    wrapped copies, ghost fills between launches; the result and its first
    ghost layer against the oracle."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    o, g, u, p = make_pair(dims, ghost=2, bc="periodic", fields=rand(dims, 17))
    g.set_kernel_config(jacobi=cfg)
    w = rounded(rand(dims, 18))
    for k, a in enumerate((WU, WV, WW)):
        g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    g.pressure_solve(0.05, iters)
    r = o.divergence(wo, 0.05)
    o.jacobi(p, r, iters)
    assert rel_err(g.download(P), o.interior(p)) < 1e-5
    gp = g.download(P, ghosts=True)
    for ax in range(3):
        for side in (1, -2):  # the first ghost layer (ghost width 2)
            sl = [slice(2, -2)] * 3
            sl[2 - ax] = side
            assert rel_err(gp[tuple(sl)], p[tuple(sl)]) < 1e-5, (ax, side)
    g.check()


def test_two_sweep_ws_periodic_steps_match_oracle():
    """Full RK2 steps on a periodic ghost-2 grid with the two-sweep kernel."""
    import workloads
    from gpu_helpers import compare_state
    dims = (64, 48, 40)
    h = tuple(2 * math.pi / d for d in dims)
    o, g, u, p = make_pair(dims, ghost=2, h=h, nu=0.01, iters=9,
                           fields=workloads.random_div_free(dims, h, seed=3))
    g.set_kernel_config(jacobi=(9, 4, 16, 16, 6))
    dt = workloads.cfl_dt(h)
    g.step(dt, 3)
    o.run(u, p, dt, 9, 3)
    compare_state(o, g, u, p, 1e-5, 1e-5, "periodic two-sweep steps")


def test_two_sweep_ws_on_periodic_grid_takes_single_sweeps():
    """On a periodic grid with one ghost layer the two-sweep variant does not
    apply; the solve still matches the oracle (single sweeps)."""
    from paper_1201_2118_gb300 import P, WU, WV, WW, mask
    dims = (128, 40, 21)
    o, g, u, p = make_pair(dims, bc="periodic", fields=rand(dims, 15))
    g.set_kernel_config(jacobi=(9, 4, 16, 16, 6))
    w = rounded(rand(dims, 16))
    for k, a in enumerate((WU, WV, WW)):
        g.interior(a).copy_(g.torch.from_numpy(w["uvw"[k]]).float().cuda())
    g.ghost_fill(mask(WU, WV, WW))
    wo = [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]
    g.pressure_solve(0.05, 6)
    r = o.divergence(wo, 0.05)
    o.jacobi(p, r, 6)
    assert rel_err(g.download(P), o.interior(p)) < 1e-5
    g.check()


def test_fused_sweeps_in_full_steps_match_single_sweeps():
    from paper_1201_2118_gb300 import U, V, W, P
    n = (128, 64, 48)
    h = (1.0 / 128,) * 3
    res = []
    for cfg in ((0, 4, 4, 32, 4), (5, 4, 4, 32, 0), (9, 4, 16, 16, 6)):
        o, g, u, p = make_pair(n, bc="cavity", h=h, nu=1e-3, fields=workloads.ldc_noise(n, seed=1))
        g.set_kernel_config(jacobi=cfg)
        g.step(workloads.cfl_dt(h), 3)
        res.append([g.download(a) for a in (U, V, W, P)])
    for other in res[1:]:
        for a, b in zip(res[0], other):
            assert rel_err(a, b) < 1e-5


@pytest.mark.parametrize("bc,ghost", [("periodic", 2), ("cavity", 1)])
def test_two_sweep_full_size_equals_single_sweeps(bc, ghost):
    """512^3 grid (periodic with two ghost layers, or the cavity the bench
    times): ten sweeps as five two-sweep launches against ten single sweeps
    of the register kernel.  Both take the same FP32 operations in the same
    order on every cell (the first sweep's values are rounded to the storage
    type in shared memory; at walls the face value stands in for the mirror
    ghost, which holds the same value), so the results agree bit for bit."""
    import torch
    from paper_1201_2118_gb300 import Grid, P, R, mask
    n = 512
    h = (2 * math.pi / n, 2 * math.pi / n, 1.7 * math.pi / n)
    res = []
    for cfg in ((9, 4, 16, 64, 6), (0, 4, 8, 32, 4)):
        g = Grid((n, n, n), ghost=ghost, h=h)
        if bc == "cavity":
            g.set_cavity(1.0)
        g.set_kernel_config(jacobi=cfg)
        gen = torch.Generator(device="cuda").manual_seed(31)
        g.interior(P).copy_(torch.rand((n, n, n), generator=gen, device="cuda") - 0.5)
        g.interior(R).copy_(torch.rand((n, n, n), generator=gen, device="cuda") - 0.5)
        g.ghost_fill(mask(P, R))
        g.jacobi(10)
        g.check()
        res.append(g.interior(P).clone())
        del g
        torch.cuda.empty_cache()
    assert torch.equal(res[0], res[1])
