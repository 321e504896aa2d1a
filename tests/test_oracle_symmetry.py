"""Symmetry pins of the FP64 oracle: one RK2 step commutes with the mirror
reflection of each axis and with the exchange of x and y (equal cell
sizes), for both advection forms and both orders, on periodic grids; and
with the reflection of z on the lid-driven cavity (lid in the x-z plane at
y = 1, moving along x), and with the reflection of x there when the lid's
velocity is reversed; a step with multigrid solves on power-of-two
grids; and the adjoint's gradients.  Whole-cell translations of a
periodic grid commute with the step bitwise (for the V-cycle step, shifts
by whole coarsest-level cells, 2^levels fine cells).

On the staggered grid a reflection of axis a maps a cell-centred index i to
n - 1 - i, and the a-face index i (at (i + 1) h_a) to n - 2 - i (mod n on a
periodic axis; on walls the wall face n - 1 maps to the ghost face -1,
both zero), and flips the sign of the a-component of velocity.  A shifted
staggered index, a sign error or a mixed-up axis anywhere in the right-hand
side, the Jacobi solve or the projection breaks the commutation.  The two
sides sum the same terms in different orders, so they agree to rounding.
"""
import numpy as np
import pytest

from oracle import Oracle

AXIS = {"x": 2, "y": 1, "z": 0}      # array axis of each coordinate in (z, y, x)
COMP = {"x": "u", "y": "v", "z": "w"}


def reflect(f, ax):
    """Mirror reflection of coordinate ax of interior fields {u, v, w, p}."""
    a = AXIS[ax]
    out = {}
    for c, arr in f.items():
        n = arr.shape[a]
        if c == COMP[ax]:
            idx = (n - 2 - np.arange(n)) % n
            out[c] = -np.take(arr, idx, axis=a)
        else:
            out[c] = np.flip(arr, axis=a).copy()
    return out


def reflect_wall(f, ax):
    """The same on an axis with walls: the wall-normal unknowns 0..n-2
    permute among themselves and the wall face n-1 stays zero."""
    out = reflect(f, ax)
    a = AXIS[ax]
    c = COMP[ax]
    n = f[c].shape[a]
    arr = np.zeros_like(f[c])
    sl_dst = [slice(None)] * 3
    sl_src = [slice(None)] * 3
    sl_dst[a] = slice(0, n - 1)
    sl_src[a] = slice(n - 2, None, -1) if n > 1 else slice(0, 0)
    arr[tuple(sl_dst)] = -f[c][tuple(sl_src)]
    out[c] = arr
    return out


def swap_xy(f):
    t = lambda arr: np.ascontiguousarray(arr.transpose(0, 2, 1))
    return {"u": t(f["v"]), "v": t(f["u"]), "w": t(f["w"]), "p": t(f["p"])}


def step(dims, h, f, bc, form, ghost, order, iters=6, lid=1.0):
    o = Oracle(dims, ghost=ghost, h=h, bc=bc, nu=0.03, form=form, order=order, lid=lid)
    u, p = o.state(f)
    o.rk2_step(u, p, 0.04 * min(h), iters)
    return {c: o.interior(a).copy() for c, a in zip("uvwp", u + [p])}


def close(a, b):
    for c in "uvwp":
        scale = max(np.abs(b[c]).max(), 1e-300)
        assert np.abs(a[c] - b[c]).max() <= 1e-12 * scale, c


def rand_fields(dims, seed):
    rng = np.random.default_rng(seed)
    return {c: rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}


@pytest.mark.parametrize("form,ghost,order", [("advective", 1, 2), ("flux", 1, 2),
                                              ("advective", 2, 4)])
@pytest.mark.parametrize("ax", ["x", "y", "z"])
def test_periodic_step_commutes_with_reflection(form, ghost, order, ax):
    dims, h = (9, 8, 7), (0.21, 0.17, 0.13)
    f = rand_fields(dims, 5)
    close(step(dims, h, reflect(f, ax), "periodic", form, ghost, order),
          reflect(step(dims, h, f, "periodic", form, ghost, order), ax))


@pytest.mark.parametrize("form,ghost,order", [("advective", 1, 2), ("flux", 1, 2),
                                              ("advective", 2, 4)])
def test_periodic_step_commutes_with_xy_exchange(form, ghost, order):
    dims, h = (8, 8, 6), (0.19, 0.19, 0.11)
    f = rand_fields(dims, 6)
    close(step(dims, h, swap_xy(f), "periodic", form, ghost, order),
          swap_xy(step(dims, h, f, "periodic", form, ghost, order)))


@pytest.mark.parametrize("form", ["advective", "flux"])
def test_cavity_step_commutes_with_z_reflection(form):
    dims, h = (7, 6, 8), (1 / 7, 1 / 6, 1 / 8)
    f = rand_fields(dims, 7)
    f["u"][:, :, -1] = 0.0
    f["v"][:, -1, :] = 0.0
    f["w"][-1, :, :] = 0.0
    close(step(dims, h, reflect_wall(f, "z"), "cavity", form, 1, 2),
          reflect_wall(step(dims, h, f, "cavity", form, 1, 2), "z"))


@pytest.mark.parametrize("form", ["advective", "flux"])
def test_cavity_x_reflection_reverses_the_lid(form):
    """Reflecting x maps the lid moving along +x to one moving along -x."""
    dims, h = (7, 6, 8), (1 / 7, 1 / 6, 1 / 8)
    f = rand_fields(dims, 9)
    f["u"][:, :, -1] = 0.0
    f["v"][:, -1, :] = 0.0
    f["w"][-1, :, :] = 0.0
    close(step(dims, h, reflect_wall(f, "x"), "cavity", form, 1, 2, lid=-1.0),
          reflect_wall(step(dims, h, f, "cavity", form, 1, 2, lid=1.0), "x"))
    a = step(dims, h, reflect_wall(f, "x"), "cavity", form, 1, 2, lid=1.0)
    b = reflect_wall(step(dims, h, f, "cavity", form, 1, 2, lid=1.0), "x")
    assert np.abs(a["u"] - b["u"]).max() > 1e-3 * np.abs(b["u"]).max()


@pytest.mark.parametrize("bc,ax", [("periodic", "x"), ("periodic", "y"), ("periodic", "z"),
                                   ("cavity", "z")])
def test_multigrid_step_commutes_with_reflection(bc, ax):
    """With power-of-two dims a reflection maps the children of each coarse
    cell onto the children of another, so the V-cycle (averaging
    restriction, trilinear prolongation, every level) commutes with it."""
    dims, h = (16, 8, 8), (0.07, 0.11, 0.13)
    f = rand_fields(dims, 10)
    refl = reflect if bc == "periodic" else reflect_wall
    if bc == "cavity":
        f["u"][:, :, -1] = 0.0
        f["v"][:, -1, :] = 0.0
        f["w"][-1, :, :] = 0.0

    def mg_step(fl):
        o = Oracle(dims, ghost=1, h=h, bc=bc, nu=0.03)
        u, p = o.state(fl)
        o.rk2_step_mg(u, p, 0.04 * min(h), 2)
        return {c: o.interior(a).copy() for c, a in zip("uvwp", u + [p])}
    close(mg_step(refl(f, ax)), refl(mg_step(f), ax))


@pytest.mark.parametrize("form", ["advective", "flux"])
@pytest.mark.parametrize("ax", ["x", "z"])
def test_adjoint_gradient_commutes_with_reflection(form, ax):
    """A reflection R is a signed permutation (orthogonal), so for the loss
    L = 1/2 |u_T - t|^2 the gradient at (R u_0, R t) is R applied to the
    gradient at (u_0, t), and dL/dnu is the same."""
    dims, h = (9, 8, 7), (0.21, 0.17, 0.13)
    f = rand_fields(dims, 11)
    t = rand_fields(dims, 12)

    def grad(fl, target):
        o = Oracle(dims, ghost=1, h=h, bc="periodic", nu=0.03, form=form)
        u, p = o.state(fl)
        tt = [target[c] for c in "uvw"]
        loss = lambda ut: (0.5 * sum(float(((a - b) ** 2).sum()) for a, b in zip(ut, tt)),
                           [a - b for a, b in zip(ut, tt)])
        _, du, dp, dnu = o.gradient(u, p, 0.04 * min(h), 6, 2, loss)
        return {"u": du[0], "v": du[1], "w": du[2], "p": dp}, dnu
    ga, na = grad(reflect(f, ax), reflect(t, ax))
    gb, nb = grad(f, t)
    close(ga, reflect(gb, ax))
    assert abs(na - nb) <= 1e-12 * abs(nb)


def shift(f, d):
    """Periodic translation by d = (dx, dy, dz) whole cells."""
    return {c: np.roll(a, (d[2], d[1], d[0]), axis=(0, 1, 2)) for c, a in f.items()}


@pytest.mark.parametrize("form,ghost,order", [("advective", 1, 2), ("flux", 1, 2),
                                              ("advective", 2, 4)])
def test_periodic_step_commutes_with_translation_bitwise(form, ghost, order):
    """Every cell does the same arithmetic in the same order, so a shift by
    whole cells commutes with the step exactly."""
    dims, h = (9, 8, 7), (0.21, 0.17, 0.13)
    f = rand_fields(dims, 13)
    d = (3, 5, 1)
    a = step(dims, h, shift(f, d), "periodic", form, ghost, order)
    b = shift(step(dims, h, f, "periodic", form, ghost, order), d)
    for c in "uvwp":
        assert np.array_equal(a[c], b[c]), c


def test_multigrid_step_commutes_with_coarse_aligned_translation_bitwise():
    """A shift by a multiple of the coarsest level's cell (2^levels fine
    cells, levels = the number of halvings) maps every level's cells onto
    cells of the same level."""
    dims, h = (32, 16, 16), (0.05, 0.07, 0.09)
    f = rand_fields(dims, 14)

    def mg_step(fl):
        o = Oracle(dims, ghost=1, h=h, bc="periodic", nu=0.03)
        u, p = o.state(fl)
        o.rk2_step_mg(u, p, 0.04 * min(h), 2)
        return {c: o.interior(a).copy() for c, a in zip("uvwp", u + [p])}, o.mg_max_levels()
    b, levels = mg_step(f)
    unit = 2 ** levels
    assert levels == 3 and unit == 8
    d = (3 * unit, unit, unit)
    a, _ = mg_step(shift(f, d))
    for c in "uvwp":
        assert np.array_equal(a[c], shift(b, d)[c]), c
    # half a coarsest cell moves the coarse grids against the fine one
    half = (unit // 2,) * 3
    a, _ = mg_step(shift(f, half))
    assert np.abs(a["u"] - shift(b, half)["u"]).max() > 1e-6


def test_reflection_is_an_involution_and_breaks_a_shifted_index():
    """The maps themselves: applying one twice is the identity, and an
    off-by-one staggered map (n - 1 - i for the reflected component) does
    not commute with the step, so the pins above can fail."""
    dims, h = (9, 8, 7), (0.21, 0.17, 0.13)
    f = rand_fields(dims, 8)
    for ax in "xyz":
        g = reflect(reflect(f, ax), ax)
        for c in "uvwp":
            assert np.array_equal(g[c], f[c])

    def bad(fl):
        out = reflect(fl, "x")
        out["u"] = -np.flip(fl["u"], axis=2).copy()
        return out
    a = step(dims, h, bad(f), "periodic", "advective", 1, 2)
    b = bad(step(dims, h, f, "periodic", "advective", 1, 2))
    assert np.abs(a["u"] - b["u"]).max() > 1e-3 * np.abs(b["u"]).max()
