"""Shared helpers of the GPU parity tests: set up the same seeded case on the
oracle (FP64) and on the CUDA path, and compare element by element."""
import math

import numpy as np

import workloads
from oracle import Oracle


def rounded(fields, dtype="f32"):
    """The initial values as the device stores them (round to nearest)."""
    import torch
    td = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    return {k: torch.from_numpy(np.asarray(v, dtype=np.float64)).to(td).to(torch.float64).numpy()
            for k, v in fields.items()}


def rel_err(got, ref, remove_mean=False):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if remove_mean:
        got = got - got.mean()
        ref = ref - ref.mean()
    scale = np.abs(ref).max()
    return np.abs(got - ref).max() / (scale if scale > 0 else 1.0)


def make_pair(dims, ghost=1, h=None, bc="periodic", nu=0.01, order=2, iters=50, omega=1.0,
              fields=None, dtype="f32", lid=1.0, form="advective"):
    """Oracle and GPU grid holding the same (device-rounded) state."""
    from paper_1201_2118_gb300 import Grid
    if h is None:
        h = tuple(2 * math.pi / d for d in dims) if bc == "periodic" else tuple(1.0 / d for d in dims)
    # (a face table gets h = 1 / n as well)
    o = Oracle(dims, ghost=ghost, h=h, bc=bc, nu=nu, order=order, omega=omega, lid=lid, form=form)
    g = Grid(dims, ghost=ghost, h=h, dtype=dtype)
    g.fill(float("nan"))
    if isinstance(bc, str):
        if bc == "cavity":
            g.set_cavity(lid)
    else:  # a face table [(kind, wall velocity), ...] for faces -x, +x, -y, +y, -z, +z
        for f, (kind, vel) in enumerate(bc):
            g.set_bc(f, kind, vel)
    g.set_params(nu, iters, omega, order)
    g.set_advection(form)
    f = rounded(fields, dtype)
    g.upload(f)
    u, p = o.state(f)
    return o, g, u, p


def compare_state(o, g, u, p, tol_u, tol_p=None, tag=""):
    from paper_1201_2118_gb300 import U, V, W, P
    errs = {}
    for k, a in enumerate((U, V, W)):
        got = g.download(a)
        assert np.isfinite(got).all(), "%s non-finite %s" % (tag, "uvw"[k])
        errs["uvw"[k]] = rel_err(got, o.interior(u[k]))
    gp = g.download(P)
    assert np.isfinite(gp).all()
    errs["p"] = rel_err(gp, o.interior(p), remove_mean=True)
    for k in "uvw":
        assert errs[k] <= tol_u, (tag, errs)
    if tol_p is not None:
        assert errs["p"] <= tol_p, (tag, errs)
    return errs


def channel_faces(lid=1.0):
    """Periodic in x and z, walls at the y faces, the +y wall moving in x."""
    from oracle import PERIODIC, WALL
    return [(PERIODIC, (0.0, 0.0, 0.0))] * 2 + [(WALL, (0.0, 0.0, 0.0)), (WALL, (lid, 0.0, 0.0))] + \
        [(PERIODIC, (0.0, 0.0, 0.0))] * 2


def tg_fields(dims, h=None):
    return workloads.taylor_green(dims, h=h)
