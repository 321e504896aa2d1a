"""Pins of the FP64 oracle adjoint (no GPU).

The adjoint is checked against the forward oracle (itself pinned in
test_oracle_pins.py) through identities that hold for any correct
transpose: <A x, y> = <x, A^T y> for the linear pieces, and for the
nonlinear step <dS(u; v), w> = <v, dS(u)^T w> with the tangent dS(u; v)
taken by central differences (the step is a polynomial of low degree in u,
so the central difference is exact up to O(eps^2) and rounding).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import Oracle

H3 = (0.31, 0.23, 0.17)


def rnd(o, rng, kind=None, ghosts=False):
    a = o.embed(rng.standard_normal(o.dims[::-1]))
    if ghosts:
        a = rng.standard_normal(o.shape)
    return a


@pytest.mark.parametrize("bc,g", [("periodic", 1), ("periodic", 2), ("cavity", 1)])
def test_ghost_fold_is_transpose_of_fill(bc, g):
    rng = np.random.default_rng(1)
    o = Oracle((7, 6, 5), ghost=g, h=H3, bc=bc, lid=0.0)  # lid 0: the fill is linear
    for kind in range(4):
        f = o.embed(rng.standard_normal(o.dims[::-1]))
        y = rng.standard_normal(o.shape)
        lhs = np.sum(o.ghost_fill(f.copy(), kind) * y)
        rhs = np.sum(f * o.ghost_fold(y.copy(), kind))
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("order,g,bc,form", [(2, 1, "periodic", "advective"),
                                             (4, 2, "periodic", "advective"),
                                             (2, 1, "cavity", "advective"),
                                             (2, 1, "periodic", "flux"), (2, 2, "periodic", "flux"),
                                             (2, 1, "cavity", "flux")])
def test_adj_stage_matches_central_difference(order, g, bc, form):
    """Stage map out(y) = a x + b y + c F(y): its tangent by central
    differences (exact: F is quadratic) against the adjoint."""
    rng = np.random.default_rng(2)
    o = Oracle((7, 6, 5), ghost=g, h=H3, bc=bc, nu=0.07, order=order, lid=0.0, form=form)
    y = [rng.standard_normal(o.shape) for _ in range(3)]
    v = [rng.standard_normal(o.shape) for _ in range(3)]
    w = [o.embed(rng.standard_normal(o.dims[::-1])) for _ in range(3)]
    eps = 1e-3
    yp = [a + eps * b for a, b in zip(y, v)]
    ym = [a - eps * b for a, b in zip(y, v)]
    op, om = o.stage(0.0, None, 0.7, yp, 0.3), o.stage(0.0, None, 0.7, ym, 0.3)
    lhs = sum(np.sum(o.interior((a - b) / (2 * eps)) * o.interior(c)) for a, b, c in zip(op, om, w))
    ybar = [o.zeros() for _ in range(3)]
    o.adj_stage(0.0, None, 0.7, y, 0.3, ybar, [c.copy() for c in w])
    rhs = sum(np.sum(a * b) for a, b in zip(v, ybar))
    assert lhs == pytest.approx(rhs, rel=1e-9)


@pytest.mark.parametrize("order,g,bc,iters,form", [(2, 1, "periodic", 6, "advective"),
                                                   (2, 1, "periodic", 5, "advective"),
                                                   (4, 2, "periodic", 4, "advective"),
                                                   (2, 1, "cavity", 6, "advective"),
                                                   (2, 2, "periodic", 5, "flux"),
                                                   (2, 1, "cavity", 6, "flux")])
def test_adj_step_dot_product(order, g, bc, iters, form):
    """Full RK2 step S(u, p) -> (u', p'): <dS (v, q), (w, s)> by central
    differences equals <(v, q), dS^T (w, s)> from the adjoint step."""
    rng = np.random.default_rng(3)
    n = (8, 7, 6)
    h = (0.35, 0.3, 0.25)
    o = Oracle(n, ghost=g, h=h, bc=bc, nu=0.05, order=order, lid=0.7, form=form)
    dt = 0.02
    base = {c: 0.5 * rng.standard_normal(n[::-1]) for c in "uvwp"}
    if bc == "cavity":
        base = {k: v.copy() for k, v in base.items()}
        base["u"][:, :, -1] = 0
        base["v"][:, -1, :] = 0
        base["w"][-1, :, :] = 0
    dv = {c: rng.standard_normal(n[::-1]) for c in "uvwp"}
    if bc == "cavity":
        dv["u"][:, :, -1] = 0
        dv["v"][:, -1, :] = 0
        dv["w"][-1, :, :] = 0
    wbar = {c: rng.standard_normal(n[::-1]) for c in "uvwp"}

    def step(eps):
        f = {c: base[c] + eps * dv[c] for c in "uvwp"}
        u, p = o.state(f)
        o.rk2_step(u, p, dt, iters)
        return [o.interior(a).copy() for a in u] + [o.interior(p).copy()]

    eps = 1e-4
    sp, sm = step(eps), step(-eps)
    lhs = sum(np.sum((a - b) / (2 * eps) * wbar[c]) for a, b, c in zip(sp, sm, "uvwp"))
    u, p = o.state(base)
    states = o.forward_record(u, p, dt, iters, 1)
    ubar = [o.embed(wbar[c]) for c in "uvw"]
    pbar = o.embed(wbar["p"])
    o.adj_rk2_step(states[0][0], states[0][1], dt, iters, ubar, pbar)
    rhs = sum(np.sum(o.interior(a) * dv[c]) for a, c in zip(ubar, "uvw"))
    rhs += np.sum(o.interior(pbar) * dv["p"])
    assert lhs == pytest.approx(rhs, rel=1e-8)
    # the adjoint leaves nothing in the ghost layers
    for a in ubar + [pbar]:
        assert np.abs(a).sum() == pytest.approx(np.abs(o.interior(a)).sum())


def _loss(target):
    def f(ui):
        d = [a - t for a, t in zip(ui, target)]
        return 0.5 * sum(np.sum(x * x) for x in d), d
    return f


def test_gradient_wrt_nu_and_u0_matches_finite_differences():
    """Three steps of the periodic flow from a divergence-free start;
    L = 1/2 |u_T - u*|^2.  dL/dnu and the directional derivative along a
    random direction of u0 against central differences."""
    n = (10, 8, 6)
    h = (0.4, 0.45, 0.5)
    dt, iters, steps = 0.05, 8, 3
    u0f = workloads.random_div_free(n, h, seed=4)
    tgt = workloads.random_div_free(n, h, seed=5)
    target = [tgt[c] * 0.8 for c in "uvw"]
    rng = np.random.default_rng(6)
    dirn = [rng.standard_normal(n[::-1]) for _ in range(3)]

    def run(nu, shift=0.0):
        o = Oracle(n, ghost=1, h=h, nu=nu)
        f = {c: u0f[c] + shift * dirn[k] for k, c in enumerate("uvw")}
        f["p"] = u0f["p"]
        u, p = o.state(f)
        o.run(u, p, dt, iters, steps)
        return _loss(target)([o.interior(a) for a in u])[0]

    nu = 0.03
    o = Oracle(n, ghost=1, h=h, nu=nu)
    u, p = o.state(u0f)
    L, gu, gp, gnu = o.gradient(u, p, dt, iters, steps, _loss(target))
    assert L == pytest.approx(run(nu), rel=1e-12)
    e = 1e-5
    fd_nu = (run(nu + e) - run(nu - e)) / (2 * e)
    assert gnu == pytest.approx(fd_nu, rel=1e-6)
    fd_u = (run(nu, e) - run(nu, -e)) / (2 * e)
    ad_u = sum(np.sum(a * b) for a, b in zip(gu, dirn))
    assert ad_u == pytest.approx(fd_u, rel=1e-6)
