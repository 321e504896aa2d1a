"""Pins of the oracle's geometric multigrid V-cycle (no GPU).

The transfers are checked on fields where they are exact (averages and
trilinear interpolation of linear functions), the cycle against exact
solutions of the discrete problem from library transforms (FFT for periodic
faces, DCT-II for zero-gradient walls), and against two textbook facts:
the convergence factor per cycle does not grow with the grid, and plain
(omega = 1) Jacobi does not smooth, so the cycle then barely converges.
"""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import Oracle, exact_poisson_periodic

H3 = (0.31, 0.23, 0.17)


def centres(o, g):
    """(z, y, x) cell-centre coordinates of every index -g..n+g-1."""
    out = []
    for a in (2, 1, 0):
        i = np.arange(-g, o.dims[a] + g, dtype=np.float64)
        out.append((i + 0.5) * o.h[a])
    z, y, x = out
    return z[:, None, None], y[None, :, None], x[None, None, :]


def exact_poisson_neumann(r_int, h):
    """Exact zero-mean solution of the 7-point problem with zero-gradient
    (mirror) ghosts: the DCT-II basis diagonalises it with eigenvalues
    sum_d (2 cos(pi m_d / N_d) - 2) / h_d^2."""
    nz, ny, nx = r_int.shape
    hx, hy, hz = h
    lam = ((2 * np.cos(np.pi * np.arange(nz) / nz) - 2) / hz**2)[:, None, None] + \
          ((2 * np.cos(np.pi * np.arange(ny) / ny) - 2) / hy**2)[None, :, None] + \
          ((2 * np.cos(np.pi * np.arange(nx) / nx) - 2) / hx**2)[None, None, :]
    c = scipy.fft.dctn(r_int, type=2, norm="ortho")
    lam[0, 0, 0] = 1.0
    c = c / lam
    c[0, 0, 0] = 0.0
    return scipy.fft.idctn(c, type=2, norm="ortho")


def test_levels_and_coarse_grid():
    o = Oracle((32, 16, 8), h=H3)
    assert o.mg_max_levels() == 2  # nz: 8 -> 4 -> 2 (an axis halves while even and >= 4)
    c = o.coarse()
    assert c.dims == (16, 8, 4) and c.h == tuple(2 * x for x in H3)
    assert Oracle((12, 12, 12)).mg_max_levels() == 2  # 12 -> 6 -> 3
    assert Oracle((7, 8, 8)).mg_max_levels() == 0


def test_restriction_averages_the_residual_exactly():
    """p quadratic (ghosts analytic) has L p = 2 (a + b + c) exactly; r linear:
    the mean of r - L p over the 8 children of a coarse cell is the linear
    function at the coarse centre minus that constant."""
    o = Oracle((8, 6, 10), ghost=1, h=H3)
    z, y, x = centres(o, 1)
    a, b, c = 0.7, -0.4, 0.25
    p = np.ascontiguousarray(np.broadcast_to(a * x * x + b * y * y + c * z * z + 0.3 * x * y,
                                             o.shape))
    r = np.ascontiguousarray(np.broadcast_to(1.5 * x - 0.5 * y + 2.0 * z + 0.1, o.shape))
    rc = o.mg_restrict_residual(p, r)
    co = o.coarse()
    Z, Y, X = centres(co, 1)
    exact = 1.5 * X - 0.5 * Y + 2.0 * Z + 0.1 - 2 * (a + b + c)
    np.testing.assert_allclose(co.interior(rc), co.interior(np.broadcast_to(exact, co.shape)),
                               rtol=0, atol=1e-12)


def test_prolongation_is_exact_for_linear_corrections():
    """A linear coarse correction (ghosts analytic) is interpolated exactly at
    every fine centre, including cells next to the faces."""
    o = Oracle((8, 6, 10), ghost=1, h=H3)
    co = o.coarse()
    Z, Y, X = centres(co, 1)
    ec = np.ascontiguousarray(np.broadcast_to(0.9 * X - 1.3 * Y + 0.6 * Z - 0.2, co.shape))
    p = o.zeros()
    o.mg_prolong_add(ec, p)
    z, y, x = centres(o, 1)
    exact = np.broadcast_to(0.9 * x - 1.3 * y + 0.6 * z - 0.2, o.shape)
    np.testing.assert_allclose(o.interior(p), o.interior(exact), rtol=0, atol=1e-12)


def _zero_mean_rhs(dims, seed):
    r = np.random.default_rng(seed).standard_normal(dims[::-1])
    return r - r.mean()


@pytest.mark.parametrize("dims", [(32, 16, 24), (16, 16, 16)])
def test_vcycles_converge_to_exact_periodic_solution(dims):
    o = Oracle(dims, h=H3)
    r = _zero_mean_rhs(dims, 3)
    R = o.embed(r)
    p = o.zeros()
    o.mg_vcycle(p, R, o.mg_max_levels(), cycles=50)
    ex = exact_poisson_periodic(r, H3)
    got = o.interior(p) - o.interior(p).mean()
    assert np.abs(got - ex).max() < 1e-12 * np.abs(ex).max()


def test_vcycles_converge_to_exact_neumann_solution():
    dims = (24, 16, 32)
    o = Oracle(dims, h=H3, bc="cavity")
    r = _zero_mean_rhs(dims, 4)
    R = o.embed(r)
    p = o.ghost_fill(o.zeros(), 3)
    o.mg_vcycle(p, R, o.mg_max_levels(), cycles=50)
    ex = exact_poisson_neumann(r, H3)
    got = o.interior(p) - o.interior(p).mean()
    assert np.abs(got - ex).max() < 1e-12 * np.abs(ex).max()


def _factor(n, bc, omega, cycles=8):
    h = (1.0 / n, 1.1 / n, 0.9 / n)
    o = Oracle((n, n, n), h=h, bc=bc)
    R = o.embed(_zero_mean_rhs((n, n, n), 5))
    p = o.ghost_fill(o.zeros(), 3)
    prev = o.residual(p, R)
    f = 0.0
    for _ in range(cycles):
        o.mg_vcycle(p, R, o.mg_max_levels(), omega=omega)
        cur = o.residual(p, R)
        f, prev = cur / prev, cur
    return f


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_convergence_factor_is_grid_independent(bc):
    f16, f64 = _factor(16, bc, 6.0 / 7.0), _factor(64, bc, 6.0 / 7.0)
    assert f16 < 0.4 and f64 < 0.4, (f16, f64)
    assert abs(f64 - f16) < 0.1 * f16, (f16, f64)


def test_unweighted_jacobi_does_not_smooth():
    """omega = 1 leaves the checkerboard mode undamped (its Jacobi factor is
    -1), so the cycle's factor approaches 1 while omega = 6/7 stays small."""
    assert _factor(32, "periodic", 1.0, cycles=12) > 0.85
    assert _factor(32, "periodic", 6.0 / 7.0, cycles=12) < 0.4


def _exact_projection_step(o, u, dt, solve):
    """Heun step with each stage's pressure equation solved exactly by
    'solve' (FFT or DCT), composed from the pinned stage, divergence and
    projection functions."""
    def ghosts(f):
        return [o.ghost_fill(a, k) for k, a in enumerate(f)]

    def project(w, cdt):
        r = o.divergence(w, cdt)
        p = o.ghost_fill(o.embed(solve(o.interior(r), o.h)), 3)
        return ghosts(o.project(w, p, cdt)), p

    w = ghosts(o.stage(0.0, None, 1.0, u, dt))
    u1, _ = project(w, dt)
    w = ghosts(o.stage(0.5, u, 0.5, u1, 0.5 * dt))
    return project(w, 0.5 * dt)


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_mg_step_converges_to_exact_projection_step(bc):
    """With enough V-cycles per solve the multigrid step equals the step whose
    pressure equations are solved exactly (velocity 1e-10, pressure up to a
    constant), and its velocity is discretely divergence-free."""
    import workloads
    dims = (32, 16, 24)
    if bc == "periodic":
        h = (2 * math.pi / 32, 2 * math.pi / 16, 2 * math.pi / 24)
        fl = workloads.random_div_free(dims, h, seed=3)
        solve = exact_poisson_periodic
    else:
        h = (1 / 32, 1 / 16, 1 / 24)
        rng = np.random.default_rng(8)
        fl = {c: 1e-2 * rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}
        solve = exact_poisson_neumann
    o = Oracle(dims, h=h, bc=bc, nu=0.01)
    u, p = o.state(fl)
    dt = 0.2 * min(h)
    ue, pe = _exact_projection_step(o, [a.copy() for a in u], dt, solve)
    o.rk2_step_mg(u, p, dt, 40)
    for k in range(3):
        scale = np.abs(o.interior(ue[k])).max()
        assert np.abs(o.interior(u[k]) - o.interior(ue[k])).max() < 1e-10 * scale, k
    gp, ep = o.interior(p) - o.interior(p).mean(), o.interior(pe) - o.interior(pe).mean()
    assert np.abs(gp - ep).max() < 1e-9 * np.abs(ep).max()
    assert np.abs(o.interior(o.divergence(u))).max() < 1e-10 * max(
        np.abs(o.interior(a)).max() for a in u) / min(h)
