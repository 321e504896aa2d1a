"""Seeded random parity cases: ragged dims (2..70 cells per axis), periodic,
cavity or channel faces, ghost width 1 (order 2, advective or flux form) or
2 (order 4), any Jacobi variant and RHS + stage variant the library accepts
(variants that do not apply to a grid fall back to single sweeps), one RK2
step against the oracle at the one-step bar (1e-5)."""
import numpy as np
import pytest

from gpu_helpers import channel_faces, compare_state, make_pair

pytestmark = pytest.mark.gpu

JACOBI = [(0, 4, 8, 32, 4), (0, 2, 4, 16, 4), (0, 1, 8, 7, 4), (1, 4, 16, 16, 4), (1, 4, 8, 32, 6),
          (1, 2, 8, 16, 4), (2, 4, 4, 2, 0), (3, 4, 4, 32, 5), (5, 4, 4, 16, 0), (7, 4, 16, 64, 8),
          (7, 2, 8, 32, 6), (9, 4, 16, 16, 6), (9, 4, 8, 7, 5)]
STENCIL = [(8, 32, 0), (4, 16, 0), (8, 32, 1), (4, 16, 1), (8, 7, 1), (8, 16, 2), (4, 8, 4),
           (4, 32, 3), (4, 9, 3)]


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    ghost = int(rng.integers(1, 3))
    dims = tuple(int(rng.integers(2 * ghost, 71)) for _ in range(3))
    bc = ["periodic", "cavity", "channel"][int(rng.integers(0, 3))]
    form = "flux" if ghost == 1 and rng.random() < 0.5 else "advective"
    jac = JACOBI[int(rng.integers(0, len(JACOBI)))]
    if jac[0] == 3:  # the cp.async sweep takes 4-wide vectors of FP32
        jac = (3, 4, jac[2], jac[3], jac[4])
    st = STENCIL[int(rng.integers(0, len(STENCIL)))]
    iters = int(rng.integers(1, 12))
    return dims, ghost, bc, form, jac, st, iters


@pytest.mark.parametrize("seed", range(24))
def test_random_case_one_step(seed):
    dims, ghost, bc, form, jac, st, iters = _case(seed)
    faces = channel_faces() if bc == "channel" else bc
    h = tuple(1.0 / d for d in dims)
    rng = np.random.default_rng(seed)
    fl = {c: rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}
    o, grid, u, p = make_pair(dims, ghost=ghost, h=h, bc=faces, nu=0.02, fields=fl, iters=iters,
                              order=2 * ghost, form=form)
    grid.set_kernel_config(jacobi=jac, stencil=st)
    dt = 0.05 * min(h)
    grid.step(dt, 1)
    o.rk2_step(u, p, dt, iters)
    compare_state(o, grid, u, p, 1e-5, 1e-5, "case %d %s" % (seed, (dims, ghost, bc, form, jac, st,
                                                                    iters)))
