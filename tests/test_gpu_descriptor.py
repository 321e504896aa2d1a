"""Kernels generated from descriptors against the oracle (or, for a stencil
the oracle does not have, a float64 numpy evaluation of the descriptor's own
formula on the same inputs), element by element, on ragged multi-tile grids.
FP32 storage and arithmetic: e <= 1e-5 (the same bar as the library's own
kernels)."""
import math

import numpy as np
import pytest

from gpu_helpers import make_pair, rel_err, rounded

pytestmark = pytest.mark.gpu

DIMS = (45, 37, 21)


def rand(dims, seed):
    rng = np.random.default_rng(seed)
    return {c: rng.uniform(-1, 1, dims[::-1]) for c in "uvwp"}


def _update_velocity(ty=8, zc=32, mode="cached"):
    from paper_1201_2118_gb300 import Descriptor
    return Descriptor(
        name="update_velocity_%s_%d_%d" % (mode, ty, zc),
        inputs={"wu": mode, "wv": mode, "ww": mode, "p": mode},
        outputs=["u", "v", "w"], params=["cdt"], stencil=(0, 1, 0, 1, 0, 1), ty=ty, zc=zc,
        body="""
          const float pc = at(p, 0, 0, 0);
          out(u) = at(wu, 0, 0, 0) - cdt * ((at(p, 1, 0, 0) - pc) * idx);
          out(v) = at(wv, 0, 0, 0) - cdt * ((at(p, 0, 1, 0) - pc) * idy);
          out(w) = at(ww, 0, 0, 0) - cdt * ((at(p, 0, 0, 1) - pc) * idz);
        """)


def _load_w(grid, o, seed):
    from paper_1201_2118_gb300 import WU, WV, WW, mask
    w = rounded(rand(DIMS, seed))
    for k, a in enumerate((WU, WV, WW)):
        grid.interior(a).copy_(grid.torch.from_numpy(w["uvw"[k]]).float().cuda())
    grid.ghost_fill(mask(WU, WV, WW))
    return [o.ghost_fill(o.embed(w["uvw"[k]]), k) for k in range(3)]


@pytest.mark.parametrize("g", [1, 2])
@pytest.mark.parametrize("ty,zc,mode", [(8, 32, "cached"), (4, 7, "cached"), (16, 5, "direct")])
def test_update_velocity_descriptor_matches_oracle_projection(g, ty, zc, mode):
    """The projection written as a descriptor (the paper's sample kernel:
    velocity in and out as separate arrays, pressure in, one parameter)."""
    from paper_1201_2118_gb300 import GeneratedKernel, P, U, V, W, U1, V1, W1, WU, WV, WW
    o, grid, u, p = make_pair(DIMS, ghost=g, fields=rand(DIMS, 1))
    wo = _load_w(grid, o, 2)
    kern = GeneratedKernel(_update_velocity(ty, zc, mode))
    kern(grid, {"wu": WU, "wv": WV, "ww": WW, "p": P, "u": U1, "v": V1, "w": W1}, cdt=0.037)
    ref = o.project(wo, p, 0.037)
    for k, a in enumerate((U1, V1, W1)):
        assert rel_err(grid.download(a), o.interior(ref[k])) < 1e-5, k


def test_divergence_descriptor_matches_oracle():
    from paper_1201_2118_gb300 import Descriptor, GeneratedKernel, R, WU, WV, WW
    o, grid, u, p = make_pair(DIMS, fields=rand(DIMS, 3))
    wo = _load_w(grid, o, 4)
    d = Descriptor(name="divergence", inputs={"wu": "direct", "wv": "direct", "ww": "direct"},
                   outputs=["r"], params=["inv_cdt"], stencil=(1, 0, 1, 0, 1, 0),
                   body="""
                     out(r) = ((at(wu, 0, 0, 0) - at(wu, -1, 0, 0)) * idx +
                               (at(wv, 0, 0, 0) - at(wv, 0, -1, 0)) * idy +
                               (at(ww, 0, 0, 0) - at(ww, 0, 0, -1)) * idz) * inv_cdt;
                   """)
    GeneratedKernel(d)(grid, {"wu": WU, "wv": WV, "ww": WW, "r": R}, inv_cdt=1.0 / 0.02)
    assert rel_err(grid.download(R), o.interior(o.divergence(wo, 0.02))) < 1e-5


@pytest.mark.parametrize("bc", ["periodic", "cavity"])
def test_jacobi_descriptor_matches_oracle_sweep(bc):
    """One weighted Jacobi sweep (cached p, direct r) on a grid whose ghosts
    the library filled (periodic wrap or zero-gradient walls)."""
    from paper_1201_2118_gb300 import Descriptor, GeneratedKernel, P, P2, R, mask
    o, grid, u, p = make_pair(DIMS, bc=bc, fields=rand(DIMS, 5), omega=0.8)
    r = rounded({"r": np.random.default_rng(6).uniform(-1, 1, DIMS[::-1])})["r"]
    grid.interior(R).copy_(grid.torch.from_numpy(r).float().cuda())
    grid.ghost_fill(mask(P))
    d = Descriptor(name="jacobi_sweep", inputs={"p": "cached", "r": "direct"}, outputs=["q"],
                   params=["omega"], ty=4, zc=6,
                   body="""
                     const float c = at(p, 0, 0, 0);
                     const float nb = (at(p, -1, 0, 0) + at(p, 1, 0, 0)) * idx2 +
                                      (at(p, 0, -1, 0) + at(p, 0, 1, 0)) * idy2 +
                                      (at(p, 0, 0, -1) + at(p, 0, 0, 1)) * idz2;
                     out(q) = c + omega * ((nb - at(r, 0, 0, 0)) / (2.f * (idx2 + idy2 + idz2)) - c);
                   """)
    GeneratedKernel(d)(grid, {"p": P, "r": R, "q": P2}, omega=0.8)
    ref = o.jacobi_sweep(p, o.embed(r))
    assert rel_err(grid.download(P2), o.interior(ref)) < 1e-5


def test_wide_stencil_descriptor_matches_numpy():
    """A fourth-order Laplacian (stencil width 2, ghost width 2) of a periodic
    field against the same five-point formula evaluated in float64 with
    numpy on the device's stored values."""
    from paper_1201_2118_gb300 import Descriptor, GeneratedKernel, U, WU
    h = (0.3, 0.25, 0.2)
    o, grid, u, p = make_pair(DIMS, ghost=2, h=h, fields=rand(DIMS, 7))
    d = Descriptor(name="lap4", inputs={"f": "cached"}, outputs=["g"], stencil=(2,) * 6, ty=4,
                   body="""
                     float s = -90.f * at(f, 0, 0, 0) * (idx2 + idy2 + idz2);
                     s += (16.f * (at(f, -1, 0, 0) + at(f, 1, 0, 0)) - (at(f, -2, 0, 0) + at(f, 2, 0, 0))) * idx2;
                     s += (16.f * (at(f, 0, -1, 0) + at(f, 0, 1, 0)) - (at(f, 0, -2, 0) + at(f, 0, 2, 0))) * idy2;
                     s += (16.f * (at(f, 0, 0, -1) + at(f, 0, 0, 1)) - (at(f, 0, 0, -2) + at(f, 0, 0, 2))) * idz2;
                     out(g) = s * (1.f / 12.f);
                   """)
    GeneratedKernel(d)(grid, {"f": U, "g": WU})
    f = grid.download(U)
    ref = -90.0 * f * sum(1.0 / x ** 2 for x in h)
    for ax, hh in ((2, h[0]), (1, h[1]), (0, h[2])):
        r1 = np.roll(f, 1, ax) + np.roll(f, -1, ax)
        r2 = np.roll(f, 2, ax) + np.roll(f, -2, ax)
        ref = ref + (16.0 * r1 - r2) / hh ** 2
    ref /= 12.0
    assert rel_err(grid.download(WU), ref) < 1e-5


def test_launch_errors():
    from paper_1201_2118_gb300 import GeneratedKernel, Grid, P, U, V, W, WU, WV, WW
    kern = GeneratedKernel(_update_velocity())
    g = Grid(DIMS, ghost=1, h=(0.1,) * 3)
    with pytest.raises(ValueError, match="unbound"):
        kern(g, {"wu": WU}, cdt=0.1)
    with pytest.raises(ValueError, match="own"):
        kern(g, {"wu": WU, "wv": WV, "ww": WW, "p": P, "u": WU, "v": V, "w": W}, cdt=0.1)
    with pytest.raises(ValueError, match="parameters"):
        kern(g, {"wu": WU, "wv": WV, "ww": WW, "p": P, "u": U, "v": V, "w": W})
    g16 = Grid(DIMS, ghost=1, h=(0.1,) * 3, dtype="bf16")
    with pytest.raises(ValueError, match="FP32"):
        kern(g16, {"wu": WU, "wv": WV, "ww": WW, "p": P, "u": U, "v": V, "w": W}, cdt=0.1)
