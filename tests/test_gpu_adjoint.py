"""Hand-written GPU adjoint against the FP64 oracle adjoint and against
central finite differences of the GPU forward model.

Tolerances: the GPU adjoint runs in FP32 on FP32 forward states, the oracle
in FP64, so normwise agreement to 1e-4 is expected at 32^3; the 128^3
finite-difference check (eps = 1e-3, FP32 forward) is held to 1e-2.
"""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import rounded

pytestmark = pytest.mark.gpu


def norm_rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_case(dims, h, nsteps, seg, iters, nu, seed=4, tseed=5, form="advective"):
    import torch
    from oracle import Oracle
    from paper_1201_2118_gb300 import Rollout
    dt = workloads.cfl_dt(h)
    u0 = rounded(workloads.random_div_free(dims, h, seed=seed))
    tgt = workloads.random_div_free(dims, h, seed=tseed)
    target = [0.5 * tgt[c] for c in "uvw"]
    ro = Rollout(dims, h, nsteps, dt, jacobi_iters=iters, seg=seg, form=form)
    t = [torch.tensor(u0[c], dtype=torch.float32, device="cuda", requires_grad=True) for c in "uvw"]
    nut = torch.tensor(nu, dtype=torch.float64, requires_grad=True)
    out = ro(t[0], t[1], t[2], nut)
    tg = [torch.tensor(x, device="cuda") for x in target]
    loss = sum(((o.double() - x) ** 2).sum() for o, x in zip(out, tg)) * 0.5
    loss.backward()
    gpu_grad = [x.grad.double().cpu().numpy() for x in t]
    gpu_gnu = nut.grad.item()
    o = Oracle(dims, ghost=2, h=h, nu=nu, form=form)
    u, p = o.state(u0)

    def lg(ui):
        d = [a - b for a, b in zip(ui, target)]
        return 0.5 * sum(np.sum(x * x) for x in d), d
    L, gu, gp, gnu = o.gradient(u, p, dt, iters, nsteps, lg)
    return loss.item(), gpu_grad, gpu_gnu, L, gu, gnu


@pytest.mark.parametrize("dims,nsteps,seg,iters,form", [((32, 32, 32), 1, 1, 50, "advective"),
                                                        ((36, 28, 20), 6, 2, 10, "advective"),
                                                        ((32, 32, 32), 5, 3, 50, "advective"),
                                                        ((32, 32, 32), 1, 1, 50, "flux"),
                                                        ((36, 28, 20), 6, 2, 10, "flux")])
def test_gpu_adjoint_matches_oracle_adjoint(dims, nsteps, seg, iters, form):
    h = tuple(2 * math.pi / d for d in dims)
    L, gg, ggnu, Lo, go, gonu = run_case(dims, h, nsteps, seg, iters, 0.01, form=form)
    assert L == pytest.approx(Lo, rel=1e-5)
    assert norm_rel(gg, go) < 1e-4
    assert ggnu == pytest.approx(gonu, rel=1e-4)


def test_gpu_gradient_matches_central_differences_128():
    """The 128^3 differentiation workload: curl-noise start (seed 4), 200 RK2
    steps, target from nu = 0.012 and a perturbed start; dL/dnu and dL/du0
    along a divergence-free direction against central differences
    (eps = 1e-3) of the FP32 forward model."""
    import torch
    from paper_1201_2118_gb300 import Rollout
    n = (128, 128, 128)
    h = tuple(2 * math.pi / d for d in n)
    dt = workloads.cfl_dt(h)
    steps = 200
    u0 = workloads.random_div_free(n, h, seed=4)
    dlt = workloads.random_div_free(n, h, seed=5)
    ro = Rollout(n, h, steps, dt, jacobi_iters=50, seg=15)
    cu = lambda f: [torch.tensor(f[c], dtype=torch.float32, device="cuda") for c in "uvw"]
    start = cu(u0)
    pert = cu({c: u0[c] + 0.1 * dlt[c] for c in "uvw"})
    target = [x.double() for x in ro.forward_only(*pert, 0.012)]

    def loss_of(fields, nu):
        out = ro.forward_only(*fields, nu)
        return sum(((o.double() - x) ** 2).sum() for o, x in zip(out, target)).item()

    t = [x.clone().requires_grad_(True) for x in start]
    nut = torch.tensor(0.01, dtype=torch.float64, requires_grad=True)
    out = ro(*t, nut)
    loss = sum(((o.double() - x) ** 2).sum() for o, x in zip(out, target))
    loss.backward()
    # eps = 1e-3 is 10 % of nu, so the central difference carries an O(eps^2)
    # truncation error of about a percent; Richardson extrapolation of the
    # eps and eps/2 differences removes that term.
    def fd(f, e):
        return (f(e) - f(-e)) / (2 * e)

    f_nu = lambda e: loss_of(start, 0.01 + e)
    fd1, fd2 = fd(f_nu, 1e-3), fd(f_nu, 5e-4)
    fd_nu = (4 * fd2 - fd1) / 3
    assert nut.grad.item() == pytest.approx(fd_nu, rel=1e-2)
    dirn = cu(workloads.random_div_free(n, h, seed=9))
    f_u = lambda e: loss_of([a + e * d for a, d in zip(start, dirn)], 0.01)
    fu1, fu2 = fd(f_u, 1e-3), fd(f_u, 5e-4)
    fd_u = (4 * fu2 - fu1) / 3
    ad_u = sum((x.grad.double() * d.double()).sum().item() for x, d in zip(t, dirn))
    assert ad_u == pytest.approx(fd_u, rel=1e-2)
    assert ad_u == pytest.approx(fu1, rel=1e-2)
    print("128^3 dL/dnu %.6e (central eps=1e-3: %.6e, Richardson: %.6e), "
          "dL/du0.d %.6e (central eps=1e-3: %.6e, Richardson: %.6e)"
          % (nut.grad.item(), fd1, fd_nu, ad_u, fu1, fd_u))
