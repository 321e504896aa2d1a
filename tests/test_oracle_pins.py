"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: a numpy
library routine with an independent definition (np.pad, FFT), a closed form,
an exact-for-polynomials property, or an invariant.  Anisotropic cell sizes
and asymmetric coefficients make a swapped axis, a wrong sign or a shifted
staggered index fail at least one of them.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import Oracle, exact_poisson_periodic, PERIODIC, WALL

H3 = (0.31, 0.23, 0.17)


def coords_ext(dims, g, h, comp):
    """(z, y, x) coordinates of component comp at every index -g..n+g-1."""
    out = []
    for a, name in ((2, "w"), (1, "v"), (0, "u")):
        i = np.arange(-g, dims[a] + g, dtype=np.float64)
        out.append((i + 1.0) * h[a] if comp == name else (i + 0.5) * h[a])
    z, y, x = out
    return z[:, None, None], y[None, :, None], x[None, None, :]


def fill_fn(o, comp, fn):
    z, y, x = coords_ext(o.dims, o.g, o.h, comp)
    return np.ascontiguousarray(np.broadcast_to(fn(x, y, z), o.shape), dtype=np.float64)


# ----------------------------------------------------------------- ghosts

@pytest.mark.parametrize("g", [1, 2])
def test_periodic_ghosts_equal_numpy_wrap(g):
    rng = np.random.default_rng(11)
    o = Oracle((7, 5, 6), ghost=g, h=H3)
    for kind in range(4):
        a = rng.standard_normal((6, 5, 7))
        f = o.ghost_fill(o.embed(a, fill=np.nan), kind)
        np.testing.assert_array_equal(f, np.pad(a, g, mode="wrap"))


def test_cavity_pressure_ghosts_equal_numpy_symmetric():
    rng = np.random.default_rng(12)
    o = Oracle((6, 7, 5), ghost=1, h=H3, bc="cavity")
    a = rng.standard_normal((5, 7, 6))
    f = o.ghost_fill(o.embed(a, fill=np.nan), 3)
    np.testing.assert_array_equal(f, np.pad(a, 1, mode="symmetric"))


@pytest.mark.parametrize("g", [1, 2])
def test_cavity_ghost_layers(g):
    """Every ghost layer: pressure mirrors evenly (np.pad 'symmetric'); a
    tangential component mirrors oddly about the wall velocity (the mean of
    a ghost and its mirror image is U_wall); the wall-normal component is
    zero on every ghost layer (at the low wall the first of them, index -1,
    is the wall face itself)."""
    rng = np.random.default_rng(14)
    n = (6, 7, 5)
    o = Oracle(n, ghost=g, h=H3, bc="cavity", lid=1.0)
    a = rng.standard_normal(n[::-1])
    np.testing.assert_array_equal(o.ghost_fill(o.embed(a, fill=np.nan), 3),
                                  np.pad(a, g, mode="symmetric"))
    u, v, w = [o.ghost_fill(o.embed(rng.standard_normal(n[::-1]), fill=np.nan), c)
               for c in range(3)]
    I = slice(g, -g)
    for m in range(1, g + 1):
        lo, hi = g - m, -g - 1 + m       # ghost m below / above the interior
        mlo, mhi = g + m - 1, -g - m     # its mirror image
        np.testing.assert_allclose(0.5 * (u[I, hi, I] + u[I, mhi, I]), 1.0, atol=1e-15)  # lid
        np.testing.assert_allclose(0.5 * (u[I, lo, I] + u[I, mlo, I]), 0.0, atol=1e-15)
        np.testing.assert_allclose(0.5 * (v[I, I, lo] + v[I, I, mlo]), 0.0, atol=1e-15)
        np.testing.assert_allclose(0.5 * (w[I, hi, I] + w[I, mhi, I]), 0.0, atol=1e-15)
        np.testing.assert_array_equal(u[I, I, lo], 0.0)
        np.testing.assert_array_equal(u[I, I, hi], 0.0)
        np.testing.assert_array_equal(v[I, lo, I], 0.0)
        np.testing.assert_array_equal(v[I, hi, I], 0.0)
        np.testing.assert_array_equal(w[lo, I, I], 0.0)
        np.testing.assert_array_equal(w[hi, I, I], 0.0)


def _wall_fill_numpy(a, comp, g, lid, order=(0, 1, 2)):
    """The cavity ghost fill written with numpy slices: passes over x, then
    y, then z (or the given axis order), each over the whole extent of the
    other two axes, so on edges and corners the later pass wins."""
    f = a.copy()
    for ax in order:
        arr_ax = 2 - ax
        n = f.shape[arr_ax] - 2 * g
        at = lambda i: tuple(i if d == arr_ax else slice(None) for d in range(3))
        u_hi = lid if (comp == 0 and ax == 1) else 0.0
        for m in range(1, g + 1):
            lo, hi = g - m, n + g - 1 + m
            mlo, mhi = g + m - 1, n + g - m
            if comp == 3:
                f[at(lo)], f[at(hi)] = f[at(mlo)], f[at(mhi)]
            elif comp == ax:
                f[at(lo)], f[at(hi)] = 0.0, 0.0
            else:
                f[at(lo)] = 2.0 * 0.0 - f[at(mlo)]
                f[at(hi)] = 2.0 * u_hi - f[at(mhi)]
    return f


@pytest.mark.parametrize("g", [1, 2])
@pytest.mark.parametrize("comp", [0, 1, 2, 3])
def test_cavity_ghost_fill_edges_and_corners(g, comp):
    """The whole padded array after the oracle's cavity fill, edges and
    corners included, equals the numpy passes x -> y -> z bitwise."""
    rng = np.random.default_rng(15 + comp)
    n = (6, 7, 5)
    o = Oracle(n, ghost=g, h=H3, bc="cavity", lid=1.0)
    e = o.embed(rng.standard_normal(n[::-1]), fill=np.nan)
    got = o.ghost_fill(e.copy(), comp)
    ref = _wall_fill_numpy(e, comp, g, 1.0)
    assert np.isfinite(got).all()
    np.testing.assert_array_equal(got, ref)
    if comp == 0:  # the pass order shows where the lid meets a still wall
        rev = _wall_fill_numpy(e, 0, g, 1.0, order=(2, 1, 0))
        edge = (g - 1, -g, slice(g, -g))  # z ghost -1, first y ghost above the lid
        np.testing.assert_allclose(np.abs(got[edge] - rev[edge]), 4.0, rtol=1e-12)


def test_cavity_velocity_ghosts_no_slip_and_lid():
    rng = np.random.default_rng(13)
    n = (6, 7, 5)
    o = Oracle(n, ghost=1, h=H3, bc="cavity", lid=1.0)
    u, v, w = [o.ghost_fill(o.embed(rng.standard_normal(n[::-1]), fill=np.nan), c)
               for c in range(3)]
    I = slice(1, -1)
    # normal component vanishes at the low wall (ghost -1 is the wall face)
    np.testing.assert_array_equal(u[I, I, 0], 0.0)
    np.testing.assert_array_equal(v[I, 0, I], 0.0)
    np.testing.assert_array_equal(w[0, I, I], 0.0)
    # tangential: mean of ghost and first interior equals the wall velocity
    np.testing.assert_allclose(0.5 * (u[I, -1, I] + u[I, -2, I]), 1.0, atol=1e-15)  # lid
    np.testing.assert_allclose(0.5 * (u[I, 0, I] + u[I, 1, I]), 0.0, atol=1e-15)
    np.testing.assert_allclose(0.5 * (w[I, -1, I] + w[I, -2, I]), 0.0, atol=1e-15)
    np.testing.assert_allclose(0.5 * (v[I, I, 0] + v[I, I, 1]), 0.0, atol=1e-15)
    np.testing.assert_allclose(0.5 * (u[0, I, I] + u[1, I, I]), 0.0, atol=1e-15)
    assert np.isfinite(u).all() and np.isfinite(v).all() and np.isfinite(w).all()


# ------------------------------------------------------------- right-hand side

def _linear_field(rng):
    A = rng.uniform(-1, 1, (3, 3))
    b = rng.uniform(-1, 1, 3)
    return A, b


@pytest.mark.parametrize("order,g", [(2, 1), (4, 2)])
def test_advection_exact_for_linear_velocity(order, g):
    """(u.grad)u of a linear field u = A x + b is A(Ax+b) at every point; central
    differences and the (bi)linear / cubic face interpolations are exact."""
    rng = np.random.default_rng(21)
    A, b = _linear_field(rng)
    o = Oracle((6, 5, 7), ghost=g, h=H3, nu=0.0, order=order)
    comps = "uvw"
    f = [fill_fn(o, comps[c], lambda x, y, z, c=c: A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + b[c])
         for c in range(3)]
    F = o.rhs(*f)
    for c in range(3):
        z, y, x = coords_ext(o.dims, g, o.h, comps[c])
        X = [x, y, z]
        vel = [A[d, 0] * x + A[d, 1] * y + A[d, 2] * z + b[d] for d in range(3)]
        exact = -sum(vel[d] * A[c, d] for d in range(3))
        exact = np.broadcast_to(exact, o.shape)
        np.testing.assert_allclose(o.interior(F[c]), o.interior(exact), rtol=0, atol=1e-12)
        del X


@pytest.mark.parametrize("order,g", [(2, 1), (4, 2)])
def test_viscous_term_exact_for_quadratics(order, g):
    """nu * lap(q) of a quadratic q is exact for the 3- and 5-point operators."""
    rng = np.random.default_rng(22)
    C = rng.uniform(-1, 1, (3, 6))
    o = Oracle((5, 6, 7), ghost=g, h=H3, order=order)
    comps = "uvw"

    def q(c):
        return lambda x, y, z: (C[c, 0] * x * x + C[c, 1] * y * y + C[c, 2] * z * z +
                                C[c, 3] * x * y + C[c, 4] * y * z + C[c, 5] * x)

    f = [fill_fn(o, comps[c], q(c)) for c in range(3)]
    o.nu = 0.0
    F0 = o.rhs(*f)
    o.nu = 0.37
    F1 = o.rhs(*f)
    for c in range(3):
        lap = 2 * (C[c, 0] + C[c, 1] + C[c, 2])
        got = (o.interior(F1[c]) - o.interior(F0[c])) / 0.37
        np.testing.assert_allclose(got, lap, rtol=0, atol=1e-9)


def test_order4_advection_exact_for_quadratic_velocity():
    """The 5-point derivative and the 4x4 cubic face interpolation are exact for
    quadratics, so the order-4 advection of a quadratic field is exact."""
    rng = np.random.default_rng(23)
    C = rng.uniform(-1, 1, (3, 7))
    o = Oracle((6, 6, 6), ghost=2, h=H3, order=4, nu=0.0)
    comps = "uvw"

    def qf(c, x, y, z):
        return (C[c, 0] * x * x + C[c, 1] * y * y + C[c, 2] * z * z + C[c, 3] * x * y +
                C[c, 4] * y * z + C[c, 5] * x + C[c, 6])

    def grad(c, x, y, z):
        return (2 * C[c, 0] * x + C[c, 3] * y + C[c, 5], 2 * C[c, 1] * y + C[c, 3] * x +
                C[c, 4] * z, 2 * C[c, 2] * z + C[c, 4] * y)

    f = [fill_fn(o, comps[c], lambda x, y, z, c=c: qf(c, x, y, z)) for c in range(3)]
    F = o.rhs(*f)
    for c in range(3):
        z, y, x = coords_ext(o.dims, 2, o.h, comps[c])
        gr = grad(c, x, y, z)
        exact = -sum(qf(d, x, y, z) * gr[d] for d in range(3))
        np.testing.assert_allclose(o.interior(F[c]), o.interior(np.broadcast_to(exact, o.shape)),
                                   rtol=0, atol=1e-11)


def _tg_rhs_error(n, order):
    g = 1 if order == 2 else 2
    nu = 0.05
    h = (2 * math.pi / n, 2 * math.pi / n, 2 * math.pi / 4)
    o = Oracle((n, n, 4), ghost=g, h=h, nu=nu, order=order)
    tg = workloads.taylor_green((n, n, 4), h=h)
    u, _ = o.state(tg)
    F = o.rhs(*u)
    err = 0.0
    _, y, x = workloads.point_coords((n, n, 4), h, "u")
    ex = -0.5 * np.sin(2 * x) - 2 * nu * np.sin(x) * np.cos(y)
    err = max(err, np.abs(o.interior(F[0]) - ex).max())
    _, y, x = workloads.point_coords((n, n, 4), h, "v")
    ex = -0.5 * np.sin(2 * y) + 2 * nu * np.cos(x) * np.sin(y)
    err = max(err, np.abs(o.interior(F[1]) - ex).max())
    assert np.abs(o.interior(F[2])).max() == 0.0
    return err


@pytest.mark.parametrize("order,rate", [(2, 4.0), (4, 16.0)])
def test_rhs_converges_at_design_order(order, rate):
    """F(Taylor-Green) against the exact -(u.grad)u + nu lap u: the error falls
    by ~2^order per halving of h."""
    e = [_tg_rhs_error(n, order) for n in (16, 32, 64)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 0.8 * rate < r2 < 1.25 * rate, (e, r1, r2)
    assert 0.7 * rate < r1 < 1.3 * rate, (e, r1, r2)


# ------------------------------------------------ conservative (flux) form

def test_flux_form_exact_for_linear_velocity():
    """div(u u_c) of a linear field u = A x + b is tr(A) u_c + sum_d u_d A[c, d].
    The side means of a linear field are exact, their product is a quadratic
    along d and its central difference about the point is exact."""
    rng = np.random.default_rng(24)
    A, b = _linear_field(rng)
    o = Oracle((6, 5, 7), ghost=1, h=H3, nu=0.0, form="flux")
    comps = "uvw"
    f = [fill_fn(o, comps[c], lambda x, y, z, c=c: A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + b[c])
         for c in range(3)]
    F = o.rhs(*f)
    for c in range(3):
        z, y, x = coords_ext(o.dims, 1, o.h, comps[c])
        vel = [A[d, 0] * x + A[d, 1] * y + A[d, 2] * z + b[d] for d in range(3)]
        exact = -(np.trace(A) * vel[c] + sum(vel[d] * A[c, d] for d in range(3)))
        np.testing.assert_allclose(o.interior(F[c]), o.interior(np.broadcast_to(exact, o.shape)),
                                   rtol=0, atol=1e-12)


def _periodic_random_velocity(o, seed):
    rng = np.random.default_rng(seed)
    n = o.dims[::-1]
    return [o.ghost_fill(o.embed(rng.standard_normal(n)), c) for c in range(3)]


def test_flux_form_conserves_momentum_on_periodic_grid():
    """The flux differences telescope: on a periodic grid the advection term
    sums to zero over each component, for any velocity field."""
    o = Oracle((7, 6, 5), ghost=1, h=H3, nu=0.0, form="flux")
    u = _periodic_random_velocity(o, 25)
    F = o.rhs(*u)
    for c in range(3):
        scale = np.abs(o.interior(F[c])).sum()
        assert abs(o.interior(F[c]).sum()) < 1e-13 * scale
    # the advective form does not conserve momentum for such a field
    oa = Oracle((7, 6, 5), ghost=1, h=H3, nu=0.0)
    Fa = oa.rhs(*u)
    assert abs(oa.interior(Fa[0]).sum()) > 1e-3 * np.abs(oa.interior(Fa[0])).sum()


def test_flux_form_energy_identity():
    """Summation by parts on a periodic grid: sum_c sum_p u_c A_c equals
    sum_c sum_p u_c^2 / 2 * (D u(p) + D u(p + e_c)) / 2, with A_c the
    flux-form advection term and D u the cell-centre divergence.  Every
    direction enters through its own divergence term, so a dropped or
    misplaced flux breaks the equality."""
    o = Oracle((7, 6, 5), ghost=1, h=H3, nu=0.0, form="flux")
    u = _periodic_random_velocity(o, 26)
    F = o.rhs(*u)
    D = o.interior(o.divergence(u))
    lhs = sum((o.interior(u[c]) * -o.interior(F[c])).sum() for c in range(3))
    rhs = 0.0
    for c in range(3):
        ax = 2 - c  # numpy axis of direction c in (z, y, x) order
        Dm = 0.5 * (D + np.roll(D, -1, axis=ax))
        rhs += (0.5 * o.interior(u[c]) ** 2 * Dm).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    assert abs(rhs) > 1.0


def test_flux_form_conserves_energy_of_div_free_field():
    """With D u = 0 the identity above makes the advection term do no work:
    sum_c sum_p u_c A_c = 0 (kinetic-energy conservation)."""
    dims = (12, 10, 8)
    fl = workloads.random_div_free(dims, H3, seed=4)
    o = Oracle(dims, ghost=1, h=H3, nu=0.0, form="flux")
    u, _ = o.state(fl)
    F = o.rhs(*u)
    work = sum((o.interior(u[c]) * o.interior(F[c])).sum() for c in range(3))
    scale = sum(np.abs(o.interior(u[c]) * o.interior(F[c])).sum() for c in range(3))
    assert abs(work) < 1e-13 * scale


def _tg_rhs_error_flux(n):
    nu = 0.05
    h = (2 * math.pi / n, 2 * math.pi / n, 2 * math.pi / 4)
    o = Oracle((n, n, 4), ghost=1, h=h, nu=nu, form="flux")
    tg = workloads.taylor_green((n, n, 4), h=h)
    u, _ = o.state(tg)
    F = o.rhs(*u)
    _, y, x = workloads.point_coords((n, n, 4), h, "u")
    err = np.abs(o.interior(F[0]) - (-0.5 * np.sin(2 * x) - 2 * nu * np.sin(x) * np.cos(y))).max()
    _, y, x = workloads.point_coords((n, n, 4), h, "v")
    err = max(err, np.abs(o.interior(F[1]) -
                          (-0.5 * np.sin(2 * y) + 2 * nu * np.cos(x) * np.sin(y))).max())
    assert np.abs(o.interior(F[2])).max() == 0.0
    return err


def test_flux_form_converges_at_second_order():
    """Taylor-Green is divergence-free, so div(u u) = (u.grad)u there and the
    flux-form F approaches the same exact right-hand side at order 2."""
    e = [_tg_rhs_error_flux(n) for n in (16, 32, 64)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.2 < r2 < 5.0 and 2.8 < r1 < 5.2, (e, r1, r2)


def test_flux_form_is_order2_only():
    with pytest.raises(ValueError):
        Oracle((4, 4, 4), ghost=2, order=4, form="flux")


# --------------------------------------------------------- pressure solve

def test_divergence_of_linear_field_is_trace():
    rng = np.random.default_rng(31)
    A, b = _linear_field(rng)
    o = Oracle((5, 6, 7), ghost=1, h=H3)
    f = [fill_fn(o, "uvw"[c], lambda x, y, z, c=c: A[c, 0] * x + A[c, 1] * y + A[c, 2] * z + b[c])
         for c in range(3)]
    r = o.divergence(f, c_dt=0.5)
    np.testing.assert_allclose(o.interior(r), np.trace(A) / 0.5, atol=1e-12)


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_divergence_is_minus_gradient_transpose(bc):
    """Summation by parts on the MAC grid: <D w, p> = -<w, G p> over the
    interior unknowns for any w and p (periodic; or walls, where the
    wall-normal velocity is zero).  G p is read off the projection of a
    zero field, w - G p with w = 0."""
    dims = (7, 6, 5)
    rng = np.random.default_rng(41)
    o = Oracle(dims, ghost=1, h=H3, bc=bc)
    w_int = [rng.uniform(-1, 1, dims[::-1]) for _ in range(3)]
    if bc == "cavity":  # no flow through the walls
        w_int[0][:, :, -1] = 0.0
        w_int[1][:, -1, :] = 0.0
        w_int[2][-1, :, :] = 0.0
    w = [o.ghost_fill(o.embed(w_int[c]), c) for c in range(3)]
    p = o.ghost_fill(o.embed(rng.uniform(-1, 1, dims[::-1])), 3)
    dw = o.interior(o.divergence(w, c_dt=1.0))
    minus_gp = o.project([o.zeros() for _ in range(3)], p, 1.0)
    lhs = float((dw * o.interior(p)).sum())
    rhs = sum(float((w_int[c] * o.interior(minus_gp[c])).sum()) for c in range(3))
    assert abs(lhs) > 1.0
    assert abs(lhs - rhs) < 1e-12 * sum(float(np.abs(w_int[c]).sum()) for c in range(3)) / min(H3)


def test_random_div_free_field_has_zero_discrete_divergence():
    dims, h = (12, 10, 8), H3
    fl = workloads.random_div_free(dims, h, seed=3)
    o = Oracle(dims, ghost=1, h=h)
    u, _ = o.state(fl)
    assert np.abs(o.interior(o.divergence(u))).max() < 1e-12 / min(h)
    assert max(np.abs(fl[c]).max() for c in "uvw") == pytest.approx(1.0)


@pytest.mark.parametrize("g", [1, 2])
@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_jacobi_periodic_eigenmode_closed_form(omega, g):
    """For r an eigenmode e of the periodic operator (L e = lam e) and p0 = 0,
    K weighted Jacobi sweeps give p_K = (1 - rho^K) e / lam with
    rho = 1 - omega (1 - s / diag), s = sum_d 2 cos(theta_d) / h_d^2."""
    n = (8, 6, 10)
    h = H3
    kw = (1, 2, 3)
    th = [2 * math.pi * kw[a] / n[a] for a in range(3)]
    o = Oracle(n, ghost=g, h=h, omega=omega)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    e = np.cos(th[0] * i + th[1] * j + th[2] * k + 0.3)
    s = sum(2 * math.cos(th[a]) / h[a] ** 2 for a in range(3))
    diag = sum(2 / h[a] ** 2 for a in range(3))
    lam = s - diag
    rho = 1 - omega * (1 - s / diag)
    r = o.embed(e)
    p = o.zeros()
    K = 7
    o.jacobi(p, r, K)
    np.testing.assert_allclose(o.interior(p), (1 - rho ** K) * e / lam, rtol=0, atol=1e-12)


@pytest.mark.parametrize("g", [1, 2])
def test_jacobi_neumann_eigenmode_closed_form(g):
    """Zero-gradient ghosts make cos(pi m (i+1/2)/N) eigenvectors with
    eigenvalue (2 cos(pi m / N) - 2) / h^2 per axis (the DCT-II basis)."""
    n = (7, 6, 5)
    h = H3
    mm = (2, 1, 3)
    o = Oracle(n, ghost=g, h=h, bc="cavity")
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = (i, j, k)
    e = np.ones(i.shape)
    for a in range(3):
        e = e * np.cos(math.pi * mm[a] * (idx[a] + 0.5) / n[a])
    s = sum(2 * math.cos(math.pi * mm[a] / n[a]) / h[a] ** 2 for a in range(3))
    diag = sum(2 / h[a] ** 2 for a in range(3))
    lam = s - diag
    rho = s / diag
    p = o.ghost_fill(o.zeros(), 3)
    r = o.embed(e)
    o.jacobi(p, r, 5)
    np.testing.assert_allclose(o.interior(p), (1 - rho ** 5) * e / lam, rtol=0, atol=1e-12)
    # the 7-point operator applied to the mode returns lam * mode
    q = o.ghost_fill(o.embed(e), 3)
    np.testing.assert_allclose(o.interior(o.laplace_p(q)), lam * e, atol=1e-10)


@pytest.mark.parametrize("g,order", [(1, 2), (2, 2), (2, 4)])
def test_exact_solve_projection_is_divergence_free_and_idempotent(g, order):
    """With the exact (FFT) Poisson solve, D G = L, so u = w - G p has D u = 0
    to rounding and projecting u again leaves it unchanged.  The projection
    is the compact second-order one for either order of the right-hand side
    and either ghost width."""
    rng = np.random.default_rng(41)
    n, h = (12, 10, 8), H3
    o = Oracle(n, ghost=g, h=h, order=order)
    w = [o.ghost_fill(o.embed(rng.standard_normal(n[::-1])), c) for c in range(3)]
    r = o.divergence(w)
    p = o.ghost_fill(o.embed(exact_poisson_periodic(o.interior(r), h)), 3)
    assert o.residual(p, r) < 1e-9 * np.abs(r).max() * math.sqrt(r.size)
    u = o.project(w, p, 1.0)
    for c in range(3):
        o.ghost_fill(u[c], c)
    assert np.abs(o.interior(o.divergence(u))).max() < 1e-10
    r2 = o.divergence(u)
    p2 = o.ghost_fill(o.embed(exact_poisson_periodic(o.interior(r2), h)), 3)
    u2 = o.project(u, p2, 1.0)
    for c in range(3):
        np.testing.assert_allclose(o.interior(u2[c]), o.interior(u[c]), atol=1e-12)


# ------------------------------------------------------------- time step

def test_rk2_is_heun_on_pure_diffusion():
    """w = w(x) only and u = v = 0 has zero advection and D u = 0, so the step
    reduces to Heun on dw/dt = nu L w; a sin-mode is multiplied by exactly
    1 + z + z^2/2 with z = dt nu (2 cos(hk) - 2) / h^2."""
    n = (16, 4, 4)
    h = (2 * math.pi / 16, 0.3, 0.4)
    nu, dt = 0.7, 0.05
    o = Oracle(n, ghost=1, h=h, nu=nu)
    x = (np.arange(n[0]) + 0.5) * h[0]
    w0 = np.broadcast_to(np.sin(x), n[::-1]).copy()
    fl = {"u": np.zeros(n[::-1]), "v": np.zeros(n[::-1]), "w": w0, "p": np.zeros(n[::-1])}
    u, p = o.state(fl)
    o.rk2_step(u, p, dt, 10)
    z = dt * nu * (2 * math.cos(h[0]) - 2) / h[0] ** 2
    np.testing.assert_allclose(o.interior(u[2]), (1 + z + z * z / 2) * w0, rtol=0, atol=1e-14)
    assert np.abs(o.interior(u[0])).max() == 0 and np.abs(o.interior(p)).max() == 0


def test_taylor_green_stays_2d_bitwise():
    n = (16, 16, 6)
    h = (2 * math.pi / 16,) * 2 + (0.5,)
    o = Oracle(n, ghost=1, h=h, nu=0.01)
    u, p = o.state(workloads.taylor_green(n, h=h))
    o.run(u, p, 0.04, 20, 5)
    assert np.abs(o.interior(u[2])).max() == 0.0
    for f in (u[0], u[1], p):
        fi = o.interior(f)
        for k in range(1, n[2]):
            np.testing.assert_array_equal(fi[k], fi[0])


def test_taylor_green_kinetic_energy_closed_form():
    """On a full period, sum sin^2 = sum cos^2 = n/2, so KE = (2 pi)^3 / 4; with
    hx = hy the sampled field is also discretely divergence-free."""
    n = (24, 24, 6)
    o = Oracle(n, ghost=1, h=tuple(2 * math.pi / d for d in n))
    u, _ = o.state(workloads.taylor_green(n))
    ke, umax, div = o.reduce(u)
    assert ke == pytest.approx((2 * math.pi) ** 3 / 4, rel=1e-13)
    assert umax <= 1.0
    assert div < 1e-12


def test_taylor_green_decay_32():
    """32^3, nu = 0.01, CFL 0.2, 100 steps, 50 Jacobi sweeps: the amplitude
    follows exp(-2 nu t) up to the O(h^2) semi-discrete viscous factor."""
    n = 32
    h = 2 * math.pi / n
    nu, dt, steps = 0.01, workloads.cfl_dt((h,) * 3), 100
    o = Oracle((n, n, 2), ghost=1, h=(h, h, h), nu=nu)
    tg = workloads.taylor_green((n, n, 2), h=(h, h, h))
    u, p = o.state(tg)
    a0 = np.abs(tg["u"]).max()
    o.run(u, p, dt, 50, steps)
    T = dt * steps
    amp = np.abs(o.interior(u[0])).max() / a0
    exact = math.exp(-2 * nu * T)
    assert T == pytest.approx(3.92699, rel=1e-5)
    assert exact == pytest.approx(0.924465, rel=1e-5)
    assert abs(amp - exact) < 0.01 * (1 - exact) + 5e-4, (amp, exact)
    ex = workloads.taylor_green((n, n, 2), h=(h, h, h), t=T, nu=nu)
    err = max(np.abs(o.interior(u[k]) - ex[c]).max() for k, c in enumerate("uv"))
    assert err < 5e-3


def test_taylor_green_error_second_order():
    """Full RK2 + projection: error against the exact solution at a fixed time
    falls ~4x per halving of h (dt proportional to h)."""
    errs = []
    for n in (16, 32, 64):
        h = 2 * math.pi / n
        o = Oracle((n, n, 1), ghost=1, h=(h, h, h), nu=0.05)
        u, p = o.state(workloads.taylor_green((n, n, 1), h=(h, h, h)))
        dt = workloads.cfl_dt((h,) * 3)
        steps = 2 * n  # T = steps * dt = 0.4 pi for every n
        o.run(u, p, dt, 400, steps)
        ex = workloads.taylor_green((n, n, 1), h=(h, h, h), t=steps * dt, nu=0.05)
        errs.append(max(np.abs(o.interior(u[k]) - ex[c]).max() for k, c in enumerate("uv")))
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
    assert 3.0 < errs[1] / errs[2] < 5.0, errs


def test_cavity_walls_held_and_mass_conserved():
    n = (10, 9, 8)
    o = Oracle(n, ghost=1, h=tuple(1.0 / d for d in n), bc="cavity", nu=0.05)
    u, p = o.state(workloads.ldc_noise(n, seed=1, amp=1e-2))
    o.run(u, p, 0.02, 30, 4)
    ui = [o.interior(a) for a in u]
    assert np.abs(ui[0][:, :, -1]).max() == 0.0
    assert np.abs(ui[1][:, -1, :]).max() == 0.0
    assert np.abs(ui[2][-1, :, :]).max() == 0.0
    # net flux through the closed box is zero: the cell divergences telescope
    div = o.interior(o.divergence(u))
    assert abs(div.sum()) * np.prod(o.h) < 1e-13
    # the lid drives flow: the first interior row under the lid moves with +x
    assert ui[0][:, -1, :-1].mean() > 0.01
