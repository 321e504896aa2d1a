"""Python face of the C ABI: a grid (one block or a block set) whose device
memory is one torch allocation bound to the library.

Every step of the time step runs in the CUDA library; this module only
marshals arguments, owns the torch allocation and moves host arrays in and
out.  Array ids and set ids follow include/gb300cfd.h.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import call, ints, doubles, c_void_p, c_size_t, c_ll, c_int, c_double

U, V, W, P, WU, WV, WW, U1, V1, W1, P2, R, LU, LV, LW, LP = range(16)
NUM_ARRAYS = 16
SET_U, SET_W, SET_U1 = 0, 1, 2
PERIODIC, WALL = 0, 1
DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
NAMES = {"u": U, "v": V, "w": W, "p": P}


def mask(*arrays) -> int:
    m = 0
    for a in arrays:
        m |= 1 << a
    return m


class Grid:
    """dims = (nx, ny, nz) for one block, or blocks = [(dims, origin), ...] with
    global_dims for a periodic rectilinear block set."""

    def __init__(self, dims=None, ghost=1, h=(1.0, 1.0, 1.0), dtype="f32", stream=None,
                 blocks=None, global_dims=None):
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("gb300cfd needs a CUDA device")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.dtype = dtype
        self.tdtype = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
        self.ghost = int(ghost)
        self.h = tuple(float(x) for x in h)
        handle = c_void_p()
        sp = c_void_p(self.stream.cuda_stream)
        if blocks is None:
            call("cfd_grid_create", ints(*dims), self.ghost, doubles(*self.h), DTYPES[dtype], sp,
                 ctypes.byref(handle))
            self.nblocks = 1
        else:
            nb = len(blocks)
            flat_d = [x for d, _ in blocks for x in d]
            flat_o = [x for _, o in blocks for x in o]
            call("cfd_blockset_create", nb, ints(*flat_d), ints(*flat_o), ints(*global_dims),
                 self.ghost, doubles(*self.h), DTYPES[dtype], sp, ctypes.byref(handle))
            self.nblocks = nb
        self.handle = handle
        nbytes = c_size_t()
        call("cfd_memory_bytes", handle, ctypes.byref(nbytes))
        self.nbytes = nbytes.value
        with torch.cuda.stream(self.stream):
            self.mem = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = self.mem.data_ptr()
        self._shift = (-ptr) % 256
        call("cfd_bind_memory", handle, c_void_p(ptr + self._shift), self.nbytes)
        self._views = {}

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            call("cfd_grid_destroy", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- layout
    def block_info(self, block=0):
        d, o, g = (c_int * 3)(), (c_int * 3)(), c_int()
        call("cfd_block_info", self.handle, block, d, o, ctypes.byref(g))
        return tuple(d), tuple(o)

    def array(self, array_id: int, block: int = 0):
        """Full ghosted (z, y, x) torch view of one array of one block."""
        key = (array_id, block)
        if key not in self._views:
            off, shape, strides, es = c_ll(), (c_ll * 3)(), (c_ll * 3)(), c_int()
            call("cfd_array_layout", self.handle, block, array_id, ctypes.byref(off), shape,
                 strides, ctypes.byref(es))
            n = (shape[0] - 1) * strides[0] + (shape[1] - 1) * strides[1] + shape[2]
            start = self._shift + off.value
            flat = self.mem[start:start + n * es.value].view(self.tdtype)
            self._views[key] = flat.as_strided(tuple(shape), tuple(strides))
        return self._views[key]

    def interior(self, array_id: int, block: int = 0):
        a = self.array(array_id, block)
        g = self.ghost
        return a[g:a.shape[0] - g, g:a.shape[1] - g, g:a.shape[2] - g]

    # ---------------------------------------------------------- host <-> dev
    def upload(self, fields: dict, block: int = 0, fill_ghosts: bool = True):
        """fields: {'u','v','w','p'} -> float64 (nz, ny, nx) numpy arrays."""
        t = self.torch
        with t.cuda.stream(self.stream):
            for name, arr in fields.items():
                src = t.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(self.tdtype)
                self.interior(NAMES[name] if isinstance(name, str) else name, block).copy_(
                    src.to("cuda", non_blocking=False))
        if fill_ghosts:
            self.ghost_fill(mask(U, V, W, P))

    def upload_blocks(self, per_block: list):
        for b, f in enumerate(per_block):
            self.upload(f, block=b, fill_ghosts=False)
        self.ghost_fill(mask(U, V, W, P))

    def download(self, array_id: int, block: int = 0, ghosts: bool = False) -> np.ndarray:
        t = self.torch
        with t.cuda.stream(self.stream):
            src = self.array(array_id, block) if ghosts else self.interior(array_id, block)
            out = src.to(t.float64).cpu().numpy()
        return out

    def fill(self, value: float):
        """Sets every byte of every array to one value (NaN canaries in tests)."""
        with self.torch.cuda.stream(self.stream):
            for b in range(self.nblocks):
                for a in range(NUM_ARRAYS):
                    self.array(a, b).fill_(value)

    # --------------------------------------------------------------- setup
    def set_bc(self, face: int, kind: int, wall_velocity=(0.0, 0.0, 0.0)):
        call("cfd_set_bc", self.handle, face, kind, doubles(*wall_velocity))

    def set_cavity(self, lid: float = 1.0):
        for f in range(6):
            self.set_bc(f, WALL, (lid, 0.0, 0.0) if f == 3 else (0.0, 0.0, 0.0))

    def set_params(self, nu: float, jacobi_iters: int = 50, omega: float = 1.0, order: int = 2):
        call("cfd_set_params", self.handle, float(nu), int(jacobi_iters), float(omega), int(order))

    ADVECTION_FORMS = {"advective": 0, "flux": 1}

    def set_advection(self, form: str):
        """Advection term of the momentum equation: 'advective', (u . grad) u_c
        (the default), or 'flux', the conservative div(u u_c) (order 2)."""
        if form not in self.ADVECTION_FORMS:
            raise ValueError(f"form must be one of {sorted(self.ADVECTION_FORMS)}")
        call("cfd_set_advection", self.handle, self.ADVECTION_FORMS[form])

    # -------------------------------------------------------- path steps
    def ghost_fill(self, m: int):
        call("cfd_ghost_fill", self.handle, int(m))

    def stage(self, a, x_set, b, y_set, c, out_set):
        call("cfd_stage", self.handle, float(a), int(x_set), float(b), int(y_set), float(c),
             int(out_set))

    def rhs_eval(self, out=None):
        """F(U) into WU, WV, WW; with out = three device tensors, also their
        compact interiors (blocks in order) into those."""
        ptrs = None if out is None else (c_void_p * 3)(*[c_void_p(t.data_ptr()) for t in out])
        call("cfd_rhs_eval", self.handle, ptrs)

    def pressure_solve(self, c_dt: float, iters: int, residual: bool = False):
        r = c_double()
        call("cfd_pressure_solve", self.handle, float(c_dt), int(iters),
             ctypes.byref(r) if residual else None)
        return r.value if residual else None

    def pressure_solve_converged(self, c_dt: float, rtol: float, max_iters: int,
                                 check_every: int = 10):
        """Sweeps until ||L P - R|| <= rtol ||R|| (checked every check_every
        sweeps) or max_iters; returns (sweeps taken, final residual)."""
        n = ctypes.c_int()
        r = c_double()
        call("cfd_pressure_solve_converged", self.handle, float(c_dt), float(rtol), int(max_iters),
             int(check_every), ctypes.byref(n), ctypes.byref(r))
        return n.value, r.value

    def jacobi(self, iters: int):
        call("cfd_jacobi", self.handle, int(iters))

    # ------------------------------------------------------------ multigrid
    def multigrid_levels(self) -> int:
        n = ctypes.c_int()
        call("cfd_multigrid_levels", self.handle, ctypes.byref(n))
        return n.value

    def set_multigrid(self, levels: int = 0, nu1: int = 2, nu2: int = 2, ncoarse: int = 30,
                      omega: float = 6.0 / 7.0):
        call("cfd_set_multigrid", self.handle, int(levels), int(nu1), int(nu2), int(ncoarse),
             float(omega))

    def set_pressure_solver(self, solver: str = "jacobi", cycles: int = 2):
        """Pressure solve of the steps' stages: 'jacobi' (jacobi_iters sweeps)
        or 'mg' (cycles V-cycles)."""
        kinds = {"jacobi": 0, "mg": 1}
        if solver not in kinds:
            raise ValueError("solver must be 'jacobi' or 'mg'")
        call("cfd_set_pressure_solver", self.handle, kinds[solver], int(cycles))

    def mg_vcycles(self, cycles: int):
        call("cfd_mg_vcycles", self.handle, int(cycles))

    def pressure_solve_mg(self, c_dt: float, rtol: float, max_cycles: int):
        """V-cycles until ||L P - R|| <= rtol ||R|| or max_cycles; returns
        (cycles taken, final residual)."""
        n = ctypes.c_int()
        r = c_double()
        call("cfd_pressure_solve_mg", self.handle, float(c_dt), float(rtol), int(max_cycles),
             ctypes.byref(n), ctypes.byref(r))
        return n.value, r.value

    @property
    def launches(self) -> int:
        n = c_ll()
        call("cfd_stats", self.handle, ctypes.byref(n))
        return n.value

    def set_kernel_config(self, jacobi=None, stencil=None):
        call("cfd_set_kernel_config", self.handle, ints(*jacobi) if jacobi else None,
             ints(*stencil) if stencil else None)

    def set_launch_mode(self, per_block: bool):
        call("cfd_set_launch_mode", self.handle, 1 if per_block else 0)

    def kernel_config(self):
        j, s = (c_int * 5)(), (c_int * 3)()
        call("cfd_get_kernel_config", self.handle, j, s)
        return tuple(j), tuple(s)

    def autotune(self, cache_path=None) -> float:
        us = c_double()
        call("cfd_autotune", self.handle, cache_path.encode() if cache_path else None,
             ctypes.byref(us))
        return us.value

    def project(self, c_dt: float, out_set: int):
        call("cfd_project", self.handle, float(c_dt), int(out_set))

    def rk_step(self, stage: int, dt: float):
        call("cfd_rk_step", self.handle, int(stage), float(dt))

    def step(self, dt: float, n: int = 1):
        call("cfd_step", self.handle, float(dt), int(n))

    def reduce(self, vset: int = SET_U):
        ke, um, dm = c_double(), c_double(), c_double()
        call("cfd_reduce", self.handle, int(vset), ctypes.byref(ke), ctypes.byref(um),
             ctypes.byref(dm))
        return ke.value, um.value, dm.value

    def residual(self) -> float:
        r = c_double()
        call("cfd_residual", self.handle, ctypes.byref(r))
        return r.value

    def copy_interior(self, array_id: int, host_ptr: int, to_device: bool, block: int = 0):
        call("cfd_copy_interior", self.handle, int(block), int(array_id), c_void_p(host_ptr),
             1 if to_device else 0)

    def set_host_copy(self, mode: str = "kernel"):
        """Route of copy_interior for page-locked host memory: 'kernel' (the
        pack kernel over the host link), 'engine' (a copy engine through
        the staging region, leaving the SMs to other streams) or 'narrow'
        (the pack kernel on one CTA per eight SMs, many transfers in flight
        per thread)."""
        modes = {"kernel": 0, "engine": 1, "narrow": 2}
        if mode not in modes:
            raise ValueError("mode must be 'kernel', 'engine' or 'narrow'")
        call("cfd_set_host_copy", self.handle, modes[mode])

    def adjoint_step(self, dt: float, un_ptrs, u1_ptrs, dnu_dev_ptr: int):
        call("cfd_adjoint_step", self.handle, float(dt), (c_void_p * 3)(*un_ptrs),
             (c_void_p * 3)(*u1_ptrs), ctypes.cast(c_void_p(dnu_dev_ptr), ctypes.POINTER(c_double)))

    def rollout_bytes(self, nsteps: int, seg: int) -> int:
        n = c_size_t()
        call("cfd_rollout_bytes", self.handle, int(nsteps), int(seg), ctypes.byref(n))
        return n.value

    def rollout_forward(self, dt, nsteps, seg, store_ptr, nbytes):
        call("cfd_rollout_forward", self.handle, float(dt), int(nsteps), int(seg),
             c_void_p(store_ptr), int(nbytes))

    def rollout_backward(self, dt, nsteps, seg, store_ptr, nbytes) -> float:
        d = c_double()
        call("cfd_rollout_backward", self.handle, float(dt), int(nsteps), int(seg),
             c_void_p(store_ptr), int(nbytes), ctypes.byref(d))
        return d.value

    def check(self):
        call("cfd_check", self.handle)

    def selftest_wait_timeout(self, form: int = 0):
        """Enqueues the library's bounded-wait self-test (cfd_check then
        reports CFD_ETIMEOUT)."""
        call("cfd_selftest_wait_timeout", self.handle, int(form))

    @property
    def time(self):
        t, s = c_double(), c_ll()
        call("cfd_get_state", self.handle, ctypes.byref(t), ctypes.byref(s))
        return t.value, s.value

    def set_time(self, t: float, step: int):
        call("cfd_set_state", self.handle, float(t), int(step))
