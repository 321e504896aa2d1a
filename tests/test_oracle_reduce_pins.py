"""Pins of the oracle's global reductions max |u_d| and max |D u| (and the
kinetic energy beside them) to values fixed by the sampled fields themselves.

The diagnostics are those the configs ask for in FP64 (CFL speed, non-finite
watchdog, discrete mass balance of Eq. 2).  Each expected value here comes
from a closed form of the input, not from the reduction's own formula:

* the sampled Taylor-Green field on one period of n = 24 cells: u peaks at
  sin(pi/2) cos(h/2) (the MAC sample nearest the crest), so max |u_d| is
  cos(pi/24);
* planted spikes of known sign in v and w over a field bounded by 1/2, and a
  larger value in a ghost cell that no interior cell reads: max |u_d| is the
  largest interior spike;
* a linear velocity u = a x, v = b y, w = c z sampled at the faces, with a
  different dyadic cell size per axis: D u = a + b + c exactly in every cell;
* the same field with the low x wall face raised by delta: only cell
  (0, j0, k0) changes, by -delta/hx.

The last test plants mistakes in altered copies of the oracle's reduction
(compiled from the same sources) and checks that each one breaks a pin.
"""
import math
import os
import tempfile

import numpy as np
import pytest

import workloads
from oracle import Oracle, compile_sources, load_library, source_paths

DIMS = (10, 7, 6)
H = (0.5, 0.25, 2.0)
A, B, C = 0.75, -2.5, 1.25   # trace -0.5
DELTA_OVER_HX = 3.0


def _face_coords(o, comp):
    """Coordinates of component comp's points on o's padded array: faces of
    the staggered grid along their own axis, cell centres across."""
    g = o.g
    nx, ny, nz = o.dims
    ax = [(np.arange(-g, n + g) + (1.0 if d == comp else 0.5)) * o.h[d]
          for d, n in enumerate((nx, ny, nz))]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _linear(o):
    """u = A x, v = B y, w = C z on every point of the padded arrays."""
    return [A * _face_coords(o, 0)[0], B * _face_coords(o, 1)[1], C * _face_coords(o, 2)[2]]


def check_tg_max(make):
    n = (24, 24, 6)
    o = make(n, (2 * math.pi / 24, 2 * math.pi / 24, 2 * math.pi / 6), "periodic")
    u, _ = o.state(workloads.taylor_green(n))
    ke, umax, _ = o.reduce(u)
    return (ke == pytest.approx((2 * math.pi) ** 3 / 4, rel=1e-13)
            and umax == pytest.approx(math.cos(math.pi / 24), abs=1e-15))


def check_spikes(make, bc):
    o = make(DIMS, H, bc)
    rng = np.random.default_rng(7)
    u = [rng.uniform(-0.5, 0.5, o.shape) for _ in range(3)]
    g = o.g
    u[1][g + 2, g + 5, g + 3] = 3.5
    u[2][g + 4, g + 1, g + 8] = -4.25
    u[0][g + 1, g - 1, g + 2] = 100.0   # a y ghost of u: no interior cell reads it
    _, umax, _ = o.reduce(u)
    return umax == 4.25


def check_linear_divergence(make, bc):
    o = make(DIMS, H, bc)
    _, _, dmax = o.reduce(_linear(o))
    return dmax == abs(A + B + C)


def check_low_face_spike(make, bc):
    o = make(DIMS, H, bc)
    u = _linear(o)
    g = o.g
    u[0][g + 3, g + 4, g - 1] += DELTA_OVER_HX * o.h[0]   # face x = 0 of cell (0, 4, 3)
    _, _, dmax = o.reduce(u)
    return dmax == abs(A + B + C - DELTA_OVER_HX)


def _pins(make):
    out = {"tg_max": check_tg_max(make)}
    for bc in ("periodic", "cavity"):
        out["spikes_" + bc] = check_spikes(make, bc)
        out["linear_div_" + bc] = check_linear_divergence(make, bc)
        out["face_spike_" + bc] = check_low_face_spike(make, bc)
    return out


def _make_with(lib=None):
    def make(dims, h, bc):
        return Oracle(dims, ghost=1, h=h, bc=bc, lib=lib)
    return make


def test_reduction_pins_hold_for_the_oracle():
    failed = [k for k, ok in _pins(_make_with()).items() if not ok]
    assert not failed, failed


def test_linear_field_divergence_is_the_trace_in_every_cell():
    """Cross-check of the input itself: the face differences of the sampled
    linear field, taken with numpy, are A, B and C exactly."""
    o = Oracle(DIMS, ghost=1, h=H)
    u = _linear(o)
    for d, (a, ax) in enumerate(((A, 2), (B, 1), (C, 0))):
        diff = np.diff(u[d], axis=ax) / H[d]
        assert np.all(diff == a)


# the reduction's body in the oracle source, and mistakes planted in it
MUTATIONS = {
    "max_velocity_never_updated": ("if (fabs(x) > m) m = fabs(x);", "(void)x;"),
    "max_velocity_signed": ("if (fabs(x) > m) m = fabs(x);", "if (x > m) m = x;"),
    "w_component_dropped": ("for (int d = 0; d < 3; ++d) {", "for (int d = 0; d < 2; ++d) {"),
    "forward_neighbour": ("val(G, u[d], q, d, -1, d, 0)", "val(G, u[d], q, d, 1, d, 0)"),
    "x_cell_size_on_every_axis": ("/ G->h[d];", "/ G->h[0];"),
    "divergence_signed": ("if (fabs(div) > dm) dm = fabs(div);", "if (div > dm) dm = div;"),
    "max_divergence_zero": ("if (part[3 * k + 2] > dm) dm = part[3 * k + 2];", "(void)dm;"),
}


def _mutated_library(tmp, name, old, new):
    srcs = source_paths()
    main = [s for s in srcs if s.endswith("cfd_oracle.c")][0]
    text = open(main).read()
    start = text.index("void ora_reduce(")
    end = text.index("\n}\n", start)
    body = text[start:end]
    assert body.count(old) == 1, (name, old)
    text = text[:start] + body.replace(old, new) + text[end:]
    path = os.path.join(tmp, "cfd_oracle.c")
    with open(path, "w") as f:
        f.write(text)
    others = [s for s in srcs if s is not main]
    return load_library(compile_sources([path] + others, os.path.join(tmp, "lib_%s.so" % name)))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_reduction_mistake_breaks_a_pin(name):
    old, new = MUTATIONS[name]
    with tempfile.TemporaryDirectory() as tmp:
        lib = _mutated_library(tmp, name, old, new)
        results = _pins(_make_with(lib))
    assert not all(results.values()), (name, results)
