"""Seeded synthetic inputs shared by the FP64 oracle tests and the CUDA path.

This module only draws and lays out input data; it holds none of the time
step's arithmetic (no advection, Laplacian, divergence, Jacobi or projection).
Every array is float64, interior only, shaped (nz, ny, nx) with x fastest.

Staggered (MAC) positions, cell size h = (hx, hy, hz), interior index i,j,k:

  p[k,j,i] at ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz)   cell centre
  u[k,j,i] at ((i+1)hx,   (j+1/2)hy, (k+1/2)hz)   right x-face
  v[k,j,i] at ((i+1/2)hx, (j+1)hy,   (k+1/2)hz)   top y-face
  w[k,j,i] at ((i+1/2)hx, (j+1/2)hy, (k+1)hz)     front z-face

The paper only says the grid is regular, rectangular and staggered (Sec. 4.1);
this placement is the usual marker-and-cell one.

Workloads (the paper's lid-driven cavity of Sec. 4.2, plus periodic test flows):

  taylor_green     2D Taylor-Green vortex embedded in 3D (periodic, L = 2 pi)
  ldc_noise        zero velocity plus seeded uniform noise on non-wall unknowns
  random_div_free  discrete MAC curl of a low-pass Gaussian vector potential
  block_tiling     rectilinear 4x4x4 tiling with seeded slab widths
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _axis_coords(n: int, h: float, staggered: bool) -> np.ndarray:
    """Cell-centre ((i+1/2)h) or face ((i+1)h) positions along one axis."""
    i = np.arange(n, dtype=np.float64)
    return (i + 1.0) * h if staggered else (i + 0.5) * h


def point_coords(dims, h, comp: str):
    """Broadcastable (z, y, x) coordinate arrays of component comp in 'uvwp'."""
    nx, ny, nz = dims
    hx, hy, hz = h
    x = _axis_coords(nx, hx, comp == "u")
    y = _axis_coords(ny, hy, comp == "v")
    z = _axis_coords(nz, hz, comp == "w")
    return z[:, None, None], y[None, :, None], x[None, None, :]


def cfl_dt(h, u_ref: float = 1.0, cfl: float = 0.2) -> float:
    """Fixed time step dt = cfl * min(h) / u_ref."""
    return cfl * min(h) / u_ref


def taylor_green(dims, h=None, amp: float = 1.0, t: float = 0.0, nu: float = 0.0):
    """Exact 2D Taylor-Green solution of the incompressible Navier-Stokes
    equations (Eq. 1-2 with f = 0) sampled at the MAC points:

      u =  A sin x cos y e^{-2 nu t},  v = -A cos x sin y e^{-2 nu t},  w = 0,
      p =  A^2/4 (cos 2x + cos 2y) e^{-4 nu t}.

    dims = (nx, ny, nz); h defaults to 2 pi / n per axis (one period).
    """
    nx, ny, nz = dims
    if h is None:
        h = (TWO_PI / nx, TWO_PI / ny, TWO_PI / nz)
    decay = math.exp(-2.0 * nu * t)
    out = {}
    _, y, x = point_coords(dims, h, "u")
    out["u"] = np.broadcast_to(amp * decay * np.sin(x) * np.cos(y), (nz, ny, nx)).copy()
    _, y, x = point_coords(dims, h, "v")
    out["v"] = np.broadcast_to(-amp * decay * np.cos(x) * np.sin(y), (nz, ny, nx)).copy()
    out["w"] = np.zeros((nz, ny, nx))
    _, y, x = point_coords(dims, h, "p")
    out["p"] = np.broadcast_to(0.25 * amp * amp * decay * decay * (np.cos(2 * x) + np.cos(2 * y)),
                               (nz, ny, nx)).copy()
    return out


def ldc_noise(n, seed: int = 1, amp: float = 1e-3):
    """Lid-driven cavity start: u = v = w = 0 plus U(-amp, amp) noise on every
    interior unknown that is not a wall-normal face, p = 0.

    n is an int (cube) or (nx, ny, nz).  Walls sit at x,y,z in {0, 1}; the
    wall-normal faces are u[:, :, nx-1], v[:, ny-1, :], w[nz-1, :, :].
    Draw order: u, v, w, each a full (nz, ny, nx) block from PCG64(seed).
    """
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for c in "uvw":
        out[c] = rng.uniform(-amp, amp, size=(nz, ny, nx))
    out["u"][:, :, nx - 1] = 0.0
    out["v"][:, ny - 1, :] = 0.0
    out["w"][nz - 1, :, :] = 0.0
    out["p"] = np.zeros((nz, ny, nx))
    return out


def _lowpass_gaussian(rng, shape, kcut: float) -> np.ndarray:
    """One N(0,1) periodic field, Fourier-filtered by exp(-(|k|/kcut)^2),
    |k| in integer wavenumbers of the periodic box."""
    a = rng.standard_normal(size=shape)
    kz = np.fft.fftfreq(shape[0]) * shape[0]
    ky = np.fft.fftfreq(shape[1]) * shape[1]
    kx = np.fft.rfftfreq(shape[2]) * shape[2]
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    spec = np.fft.rfftn(a) * np.exp(-k2 / (kcut * kcut))
    return np.fft.irfftn(spec, s=shape, axes=(0, 1, 2))


def random_div_free(dims, h, seed: int, kcut: float = 4.0):
    """Seeded divergence-free periodic velocity: u = curl A on the MAC grid.

    A_x, A_y, A_z are i.i.d. N(0,1) on the periodic lattice (PCG64(seed), drawn
    in that order), low-pass filtered, and placed on the cell edges:
      A_x at ((i+1/2)hx, (j+1)hy, (k+1)hz), A_y at ((i+1)hx, (j+1/2)hy, (k+1)hz),
      A_z at ((i+1)hx, (j+1)hy, (k+1/2)hz).
    The one-sided edge differences below make the discrete divergence of
    (u, v, w) vanish identically.  The field is scaled to max |u_d| = 1.
    p = 0.
    """
    nx, ny, nz = dims
    hx, hy, hz = h
    shape = (nz, ny, nx)
    rng = np.random.Generator(np.random.PCG64(seed))
    ax = _lowpass_gaussian(rng, shape, kcut)
    ay = _lowpass_gaussian(rng, shape, kcut)
    az = _lowpass_gaussian(rng, shape, kcut)

    def back(a, axis):  # a[idx] - a[idx - 1] along one axis, periodic
        return a - np.roll(a, 1, axis=axis)

    u = back(az, 1) / hy - back(ay, 0) / hz
    v = back(ax, 0) / hz - back(az, 2) / hx
    w = back(ay, 2) / hx - back(ax, 1) / hy
    s = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    return {"u": u / s, "v": v / s, "w": w / s, "p": np.zeros(shape)}


def block_tiling(seed: int = 2, nb: int = 4, lo: int = 16, hi: int = 96):
    """Carpet-style rectilinear tiling of a periodic box by nb^3 blocks.

    Per axis, nb slab widths are drawn from U{lo..hi} (PCG64(seed), one
    (3, nb) draw, rows x, y, z).  Returns (global_dims, blocks) with blocks a
    list of dicts {dims: (nx,ny,nz), origin: (ox,oy,oz), index: (bx,by,bz)},
    ordered x fastest.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    widths = rng.integers(lo, hi + 1, size=(3, nb))
    starts = [np.concatenate([[0], np.cumsum(widths[a])[:-1]]) for a in range(3)]
    gdims = tuple(int(widths[a].sum()) for a in range(3))
    blocks = []
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                blocks.append({
                    "dims": (int(widths[0, bx]), int(widths[1, by]), int(widths[2, bz])),
                    "origin": (int(starts[0][bx]), int(starts[1][by]), int(starts[2][bz])),
                    "index": (bx, by, bz),
                })
    return gdims, blocks


def split_blocks(fields: dict, blocks) -> list:
    """Cut global interior arrays (nz, ny, nx) into per-block interior copies."""
    out = []
    for b in blocks:
        (nx, ny, nz), (ox, oy, oz) = b["dims"], b["origin"]
        out.append({c: np.ascontiguousarray(a[oz:oz + nz, oy:oy + ny, ox:ox + nx])
                    for c, a in fields.items()})
    return out


# Workload definitions (grid, physics, time step).  Names say what they are.
WORKLOADS = {
    "tg32": dict(desc="32^3 periodic Taylor-Green, nu=0.01, 100 RK2 steps, FP32",
                 dims=(32, 32, 32), ghost=1, nu=0.01, steps=100, order=2,
                 jacobi_iters=50, bc="periodic", ic="taylor_green"),
    "ldc256": dict(desc="256^3 lid-driven cavity Re=1000, 1000 RK2 steps, FP32",
                   dims=(256, 256, 256), ghost=1, nu=1e-3, steps=1000, order=2,
                   jacobi_iters=50, bc="cavity", ic="ldc_noise", seed=1),
    "ldc512": dict(desc="512^3 lid-driven cavity Re=1000, 1000 RK2 steps, FP32",
                   dims=(512, 512, 512), ghost=1, nu=1e-3, steps=1000, order=2,
                   jacobi_iters=50, bc="cavity", ic="ldc_noise", seed=1),
    "blocks64": dict(desc="64 uneven periodic blocks (4x4x4, widths U{16..96}), "
                          "curl-noise start, nu=0.01, 100 RK2 steps",
                     tiling_seed=2, ic_seed=3, nu=0.01, steps=100, jacobi_iters=50,
                     bc="periodic", ic="random_div_free"),
    "tg512": dict(desc="512^3 periodic Taylor-Green, nu=0.005, 500 RK2 steps, "
                       "BF16/FP16 storage", dims=(512, 512, 512), ghost=1, nu=0.005,
                  steps=500, order=2, jacobi_iters=50, bc="periodic", ic="taylor_green"),
    "adj128": dict(desc="128^3 periodic curl-noise start, 200 RK2 steps, adjoint "
                        "gradient wrt u0 and nu", dims=(128, 128, 128), ghost=1,
                   nu=0.01, nu_target=0.012, steps=200, order=2, jacobi_iters=50,
                   bc="periodic", ic="random_div_free", seed=4, target_seed=5),
}


def workload_h(name: str, dims=None):
    """Cell size of a workload: 2 pi / n for periodic flows (one period over
    a 2 pi box; 2 pi / 128 per cell for the block tiling), 1 / n for the unit
    cavity."""
    w = WORKLOADS[name]
    dims = dims or w.get("dims")
    if w["bc"] == "cavity":
        return tuple(1.0 / d for d in dims)
    if name == "blocks64":
        return (TWO_PI / 128,) * 3
    return tuple(TWO_PI / d for d in dims)
