"""ctypes wrapper of the FP64 C oracle, plus test-only exact solvers.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py; the CUDA library never uses it.

Arrays are float64, shape (nz+2g, ny+2g, nx+2g), x fastest; `interior(a)`
is the (nz, ny, nx) view of cells 0..n-1.  Component kinds: 0 u, 1 v, 2 w,
3 p.  Faces: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["cfd_oracle.c", "cfd_oracle_adjoint.c", "cfd_oracle_mg.c"]
_lock = threading.Lock()
_lib = None

PERIODIC, WALL = 0, 1
FORMS = {"advective": 0, "flux": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -O2, OpenMP over rows (k, j))."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "cfd_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    compile_sources(srcs, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("g", ctypes.c_int), ("h", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 6), ("wall", (ctypes.c_double * 3) * 6),
                ("nu", ctypes.c_double), ("omega", ctypes.c_double), ("order", ctypes.c_int),
                ("form", ctypes.c_int)]


class _Mg(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("ncoarse", ctypes.c_int), ("omega", ctypes.c_double)]


_D = ctypes.POINTER(ctypes.c_double)


def _configure(lib):
    """Argument and result types of every oracle entry point on a loaded
    library."""
    G = ctypes.POINTER(_Grid)
    P3 = _D * 3
    sig = {
        "ora_ghost_fill": [G, _D, ctypes.c_int],
        "ora_rhs": [G, _D, _D, _D, _D, _D, _D],
        "ora_stage": [G, ctypes.c_double, P3, ctypes.c_double, P3, ctypes.c_double, P3],
        "ora_divergence": [G, P3, ctypes.c_double, _D],
        "ora_jacobi_sweep": [G, _D, _D, _D],
        "ora_jacobi": [G, _D, _D, _D, ctypes.c_int],
        "ora_project": [G, P3, _D, ctypes.c_double, P3],
        "ora_rk2_step": [G, P3, _D, ctypes.c_double, ctypes.c_int, _D * 8],
        "ora_reduce": [G, P3, _D, _D, _D],
        "ora_residual": [G, _D, _D],
        "ora_laplace_p": [G, _D, _D],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_double if name == "ora_residual" else None
    adj = {
        "ora_ghost_fold": [G, _D, ctypes.c_int],
        "ora_adj_stage": [G, ctypes.c_double, P3, ctypes.c_double, P3, ctypes.c_double,
                          P3, P3, _D],
        "ora_adj_rk2_step": [G, P3, P3, ctypes.c_double, ctypes.c_int, P3, _D, _D,
                             _D * 11],
    }
    for name, args in adj.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None
    mg = {
        "ora_mg_restrict_residual": [G, _D, _D, _D],
        "ora_mg_prolong_add": [G, _D, _D],
        "ora_mg_vcycle": [G, ctypes.POINTER(_Mg), _D, _D],
        "ora_rk2_step_mg": [G, P3, _D, ctypes.c_double, ctypes.POINTER(_Mg), ctypes.c_int,
                            _D * 8],
    }
    for name, args in mg.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None
    lib.ora_mg_max_levels.argtypes = [G]
    lib.ora_mg_max_levels.restype = ctypes.c_int
    lib.ora_set_threads.argtypes = [ctypes.c_int]
    lib.ora_set_threads.restype = ctypes.c_int
    return lib


def load_library(path: str):
    """A configured ctypes handle of an oracle build at `path` (the tests'
    planted-error checks load altered builds of the same sources this way)."""
    return _configure(ctypes.CDLL(path))


def compile_sources(sources, out_path: str) -> str:
    """gcc the given C files (plain C99, -O2, OpenMP) into a shared library."""
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-I", _HERE, "-o",
           out_path] + list(sources) + ["-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def source_paths():
    return [os.path.join(_HERE, s) for s in _SOURCES]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _p3(arrs):
    return (_D * 3)(*[_ptr(a) for a in arrs])


def bc_faces(kind: str, lid: float = 1.0):
    """Face boundary table: 'periodic' (all faces) or 'cavity' (unit box,
    walls on every face, the +y lid moving with velocity (lid, 0, 0))."""
    if kind == "periodic":
        return [(PERIODIC, (0.0, 0.0, 0.0))] * 6
    if kind == "cavity":
        faces = [(WALL, (0.0, 0.0, 0.0))] * 6
        faces[3] = (WALL, (lid, 0.0, 0.0))
        return faces
    raise ValueError(kind)


class Oracle:
    """One block of the FP64 scheme with its boundary table and parameters."""

    def __init__(self, dims, ghost=1, h=(1.0, 1.0, 1.0), bc="periodic", nu=0.0, omega=1.0,
                 order=2, lid=1.0, form="advective", lib=None):
        if form not in FORMS:
            raise ValueError(f"form must be one of {sorted(FORMS)}")
        if form == "flux" and int(order) != 2:
            raise ValueError("the flux form is order 2")
        self.lib = _load() if lib is None else lib
        self.form = form
        self.dims = tuple(int(d) for d in dims)
        self.g = int(ghost)
        faces = bc_faces(bc, lid) if isinstance(bc, str) else list(bc)
        self.faces = faces
        gr = _Grid()
        gr.n[:] = self.dims
        gr.g = self.g
        gr.h[:] = tuple(float(x) for x in h)
        for f, (kind, vel) in enumerate(faces):
            gr.bc[f] = kind
            gr.wall[f][:] = tuple(float(x) for x in vel)
        gr.nu, gr.omega, gr.order = float(nu), float(omega), int(order)
        gr.form = FORMS[form]
        self._g = gr
        self.h = tuple(float(x) for x in h)
        self.shape = tuple(d + 2 * self.g for d in self.dims[::-1])

    @property
    def nu(self):
        return self._g.nu

    @nu.setter
    def nu(self, value):
        self._g.nu = float(value)

    def _G(self):
        return ctypes.byref(self._g)

    # -- arrays
    def zeros(self):
        return np.zeros(self.shape)

    def interior(self, a):
        g = self.g
        nx, ny, nz = self.dims
        return a[g:g + nz, g:g + ny, g:g + nx]

    def embed(self, interior_arr, fill=0.0):
        a = np.full(self.shape, fill, dtype=np.float64)
        self.interior(a)[...] = interior_arr
        return a

    # -- the scheme's steps
    def ghost_fill(self, f, kind):
        self.lib.ora_ghost_fill(self._G(), _ptr(f), int(kind))
        return f

    def rhs(self, u, v, w):
        out = [self.zeros() for _ in range(3)]
        self.lib.ora_rhs(self._G(), _ptr(u), _ptr(v), _ptr(w), *[_ptr(o) for o in out])
        return out

    def stage(self, a, x, b, y, c):
        out = [self.zeros() for _ in range(3)]
        xs = _p3(x) if x is not None else (_D * 3)()
        self.lib.ora_stage(self._G(), float(a), xs, float(b), _p3(y), float(c), _p3(out))
        return out

    def divergence(self, w, c_dt=1.0):
        r = self.zeros()
        self.lib.ora_divergence(self._G(), _p3(w), float(c_dt), _ptr(r))
        return r

    def jacobi_sweep(self, p, r):
        out = self.zeros()
        self.lib.ora_jacobi_sweep(self._G(), _ptr(p), _ptr(r), _ptr(out))
        return out

    def jacobi(self, p, r, iters):
        tmp = self.zeros()
        self.lib.ora_jacobi(self._G(), _ptr(p), _ptr(r), _ptr(tmp), int(iters))
        return p

    def project(self, w, p, c_dt):
        out = [self.zeros() for _ in range(3)]
        self.lib.ora_project(self._G(), _p3(w), _ptr(p), float(c_dt), _p3(out))
        return out

    def rk2_step(self, u, p, dt, iters, scratch=None):
        if scratch is None:
            scratch = [self.zeros() for _ in range(8)]
        self.lib.ora_rk2_step(self._G(), _p3(u), _ptr(p), float(dt), int(iters),
                              (_D * 8)(*[_ptr(s) for s in scratch]))
        return u, p

    def run(self, u, p, dt, iters, steps):
        scratch = [self.zeros() for _ in range(8)]
        for _ in range(steps):
            self.rk2_step(u, p, dt, iters, scratch)
        return u, p

    def reduce(self, u):
        ke, um, dm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self.lib.ora_reduce(self._G(), _p3(u), ctypes.byref(ke), ctypes.byref(um),
                            ctypes.byref(dm))
        return ke.value, um.value, dm.value

    def residual(self, p, r):
        return self.lib.ora_residual(self._G(), _ptr(p), _ptr(r))

    def laplace_p(self, p):
        out = self.zeros()
        self.lib.ora_laplace_p(self._G(), _ptr(p), _ptr(out))
        return out

    # -- geometric multigrid
    def mg_max_levels(self):
        return int(self.lib.ora_mg_max_levels(self._G()))

    def coarse(self):
        """Oracle of the next coarser level (n / 2, 2 h, same faces)."""
        if any(d % 2 for d in self.dims):
            raise ValueError("every dimension must be even")
        c = Oracle.__new__(Oracle)
        c.__dict__.update(self.__dict__)
        gr = _Grid()
        ctypes.pointer(gr)[0] = self._g
        gr.n[:] = tuple(d // 2 for d in self.dims)
        gr.h[:] = tuple(2 * x for x in self.h)
        c._g = gr
        c.dims = tuple(d // 2 for d in self.dims)
        c.h = tuple(2 * x for x in self.h)
        c.shape = tuple(d + 2 * self.g for d in c.dims[::-1])
        return c

    def mg_restrict_residual(self, p, r):
        rc = self.coarse().zeros()
        self.lib.ora_mg_restrict_residual(self._G(), _ptr(p), _ptr(r), _ptr(rc))
        return rc

    def mg_prolong_add(self, ec, p):
        self.lib.ora_mg_prolong_add(self._G(), _ptr(ec), _ptr(p))
        return p

    def mg_vcycle(self, p, r, levels, nu1=2, nu2=2, ncoarse=30, omega=6.0 / 7.0, cycles=1):
        """cycles V-cycles in place on p (ghosts filled)."""
        m = _Mg(int(levels), int(nu1), int(nu2), int(ncoarse), float(omega))
        for _ in range(cycles):
            self.lib.ora_mg_vcycle(self._G(), ctypes.byref(m), _ptr(p), _ptr(r))
        return p

    def rk2_step_mg(self, u, p, dt, cycles, levels=0, nu1=2, nu2=2, ncoarse=30,
                    omega=6.0 / 7.0, steps=1):
        """steps RK2 steps in place, each pressure solve 'cycles' V-cycles
        (levels 0: all available)."""
        m = _Mg(int(levels or self.mg_max_levels()), int(nu1), int(nu2), int(ncoarse),
                float(omega))
        scratch = [self.zeros() for _ in range(8)]
        for _ in range(steps):
            self.lib.ora_rk2_step_mg(self._G(), _p3(u), _ptr(p), float(dt), ctypes.byref(m),
                                     int(cycles), (_D * 8)(*[_ptr(s) for s in scratch]))
        return u, p

    # -- discrete adjoint
    def ghost_fold(self, f, kind):
        self.lib.ora_ghost_fold(self._G(), _ptr(f), int(kind))
        return f

    def adj_stage(self, a, xbar, b, y, c, ybar, outbar):
        nb = ctypes.c_double(0.0)
        xs = _p3(xbar) if xbar is not None else (_D * 3)()
        self.lib.ora_adj_stage(self._G(), float(a), xs, float(b), _p3(y), float(c), _p3(ybar),
                               _p3(outbar), ctypes.byref(nb))
        return nb.value

    def forward_record(self, u, p, dt, iters, steps):
        """Runs steps RK2 steps in place and returns the per-step stored
        states [(u^n, u1), ...] (copies, ghosts filled)."""
        scratch = [self.zeros() for _ in range(8)]
        states = []
        for _ in range(steps):
            un = [a.copy() for a in u]
            self.rk2_step(u, p, dt, iters, scratch)
            states.append((un, [scratch[3].copy(), scratch[4].copy(), scratch[5].copy()]))
        return states

    def adj_rk2_step(self, un, u1, dt, iters, ubar, pbar, scratch=None):
        """One adjoint step in place on ubar, pbar; returns dL/dnu of it."""
        if scratch is None:
            scratch = [self.zeros() for _ in range(11)]
        nb = ctypes.c_double(0.0)
        self.lib.ora_adj_rk2_step(self._G(), _p3(un), _p3(u1), float(dt), int(iters), _p3(ubar),
                                  _ptr(pbar), ctypes.byref(nb),
                                  (_D * 11)(*[_ptr(s) for s in scratch]))
        return nb.value

    def gradient(self, u0, p0, dt, iters, steps, loss_grad):
        """dL/du0 (interior, 3 arrays), dL/dp0 and dL/dnu of a loss of the
        final velocity: loss_grad(u_T interiors) -> (L, [dL/du_T interiors])."""
        u = [a.copy() for a in u0]
        p = p0.copy()
        states = self.forward_record(u, p, dt, iters, steps)
        L, g = loss_grad([self.interior(a) for a in u])
        ubar = [self.embed(gc) for gc in g]
        pbar = self.zeros()
        nubar = 0.0
        scratch = [self.zeros() for _ in range(11)]
        for un, u1 in reversed(states):
            nubar += self.adj_rk2_step(un, u1, dt, iters, ubar, pbar, scratch)
        return L, [self.interior(a).copy() for a in ubar], self.interior(pbar).copy(), nubar

    # -- set-up helper: padded state from interior arrays, ghosts filled
    def state(self, fields):
        u = [self.ghost_fill(self.embed(fields[c]), k) for k, c in enumerate("uvw")]
        p = self.ghost_fill(self.embed(fields["p"]), 3)
        return u, p


def exact_poisson_periodic(r_int: np.ndarray, h) -> np.ndarray:
    """Exact solution of the periodic 7-point problem L p = r (mean-free),
    test-only: separable DFT (numpy FFT as the library primitive) with the
    operator's eigenvalues sum_d (2 cos(2 pi k_d / N_d) - 2) / h_d^2."""
    nz, ny, nx = r_int.shape
    hx, hy, hz = h
    lam = ((2 * np.cos(2 * np.pi * np.fft.fftfreq(nz)) - 2) / hz**2)[:, None, None] + \
          ((2 * np.cos(2 * np.pi * np.fft.fftfreq(ny)) - 2) / hy**2)[None, :, None] + \
          ((2 * np.cos(2 * np.pi * np.fft.fftfreq(nx)) - 2) / hx**2)[None, None, :]
    rh = np.fft.fftn(r_int)
    lam[0, 0, 0] = 1.0
    ph = rh / lam
    ph[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(ph))


def set_threads(n: int) -> int:
    """Host threads of the oracle's OpenMP loops (n <= 0: the default);
    returns the count in effect.  Results do not depend on it."""
    return int(_load().ora_set_threads(int(n)))
