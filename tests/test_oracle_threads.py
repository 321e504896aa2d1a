"""The oracle's results do not depend on its host thread count: its
parallel loops write disjoint cells, and its reductions sum per-plane
partials in plane order.  One RK2 step (both advection forms), a multigrid
step, the FP64 reductions and an adjoint step on a ragged cavity grid, on
one thread and on four, compared bitwise."""
import numpy as np
import pytest

import workloads
from oracle import Oracle, set_threads

DIMS = (13, 10, 7)


def _state(o, seed):
    rng = np.random.default_rng(seed)
    f = workloads.ldc_noise(DIMS, seed=seed, amp=0.3)
    f["p"] = rng.uniform(-1, 1, DIMS[::-1])
    return o.state(f)


def _run(threads, form):
    set_threads(threads)
    try:
        h = (1.0 / 13, 1.0 / 10, 1.0 / 7)
        o = Oracle(DIMS, ghost=1, h=h, bc="cavity", nu=0.02, form=form)
        dt = 0.3 * min(h)
        u, p = _state(o, 3)
        un = [a.copy() for a in u]
        o.rk2_step(u, p, dt, 20)
        red = o.reduce(u)
        r = o.divergence(u, dt)
        res = o.residual(p, r)
        um, pm = _state(o, 4)
        o.rk2_step_mg(um, pm, dt, 2)
        states = o.forward_record([a.copy() for a in un], o.zeros(), dt, 20, 1)
        ubar = [o.embed(np.ones(DIMS[::-1])) for _ in range(3)]
        pbar = o.zeros()
        dnu = o.adj_rk2_step(states[0][0], states[0][1], dt, 20, ubar, pbar)
        return [*u, p, *um, pm, *ubar, pbar], (*red, res, dnu)
    finally:
        set_threads(0)


@pytest.mark.parametrize("form", ["advective", "flux"])
def test_one_thread_and_four_agree_bitwise(form):
    a1, s1 = _run(1, form)
    a4, s4 = _run(4, form)
    assert s1 == s4
    for x, y in zip(a1, a4):
        assert np.array_equal(x, y)
    assert all(np.isfinite(v) for v in s1)
