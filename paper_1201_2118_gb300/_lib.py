"""ctypes declarations of libgb300cfd.so (argument marshalling only).

Loading fails loudly when the library is missing and cannot be built: there is
no CPU fallback for any step of the time step.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_uint, c_double, c_void_p, c_size_t, c_ll = (ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                                                    ctypes.c_void_p, ctypes.c_size_t,
                                                    ctypes.c_longlong)
P = ctypes.POINTER

# name -> argument types (all return cfd_status as int unless listed below)
SIGNATURES = {
    "cfd_grid_create": [P(c_int), c_int, P(c_double), c_int, c_void_p, P(c_void_p)],
    "cfd_blockset_create": [c_int, P(c_int), P(c_int), P(c_int), c_int, P(c_double), c_int,
                            c_void_p, P(c_void_p)],
    "cfd_grid_destroy": [c_void_p],
    "cfd_memory_bytes": [c_void_p, P(c_size_t)],
    "cfd_bind_memory": [c_void_p, c_void_p, c_size_t],
    "cfd_alloc_memory": [c_void_p],
    "cfd_array_layout": [c_void_p, c_int, c_int, P(c_ll), P(c_ll), P(c_ll), P(c_int)],
    "cfd_block_info": [c_void_p, c_int, P(c_int), P(c_int), P(c_int)],
    "cfd_set_bc": [c_void_p, c_int, c_int, P(c_double)],
    "cfd_set_params": [c_void_p, c_double, c_int, c_double, c_int],
    "cfd_set_advection": [c_void_p, c_int],
    "cfd_multigrid_levels": [c_void_p, P(c_int)],
    "cfd_set_multigrid": [c_void_p, c_int, c_int, c_int, c_int, c_double],
    "cfd_mg_vcycles": [c_void_p, c_int],
    "cfd_set_pressure_solver": [c_void_p, c_int, c_int],
    "cfd_pressure_solve_mg": [c_void_p, c_double, c_double, c_int, P(c_int), P(c_double)],
    "cfd_ghost_fill": [c_void_p, c_uint],
    "cfd_stage": [c_void_p, c_double, c_int, c_double, c_int, c_double, c_int],
    "cfd_rhs_eval": [c_void_p, P(c_void_p)],
    "cfd_pressure_solve": [c_void_p, c_double, c_int, P(c_double)],
    "cfd_pressure_solve_converged": [c_void_p, c_double, c_double, c_int, c_int, P(c_int),
                                     P(c_double)],
    "cfd_project": [c_void_p, c_double, c_int],
    "cfd_jacobi": [c_void_p, c_int],
    "cfd_stats": [c_void_p, P(c_ll)],
    "cfd_set_launch_mode": [c_void_p, c_int],
    "cfd_set_kernel_config": [c_void_p, P(c_int), P(c_int)],
    "cfd_get_kernel_config": [c_void_p, P(c_int), P(c_int)],
    "cfd_autotune": [c_void_p, ctypes.c_char_p, P(c_double)],
    "cfd_adjoint_step": [c_void_p, c_double, P(c_void_p), P(c_void_p), P(c_double)],
    "cfd_rollout_bytes": [c_void_p, c_int, c_int, P(c_size_t)],
    "cfd_rollout_forward": [c_void_p, c_double, c_int, c_int, c_void_p, c_size_t],
    "cfd_rollout_backward": [c_void_p, c_double, c_int, c_int, c_void_p, c_size_t, P(c_double)],
    "cfd_rk_step": [c_void_p, c_int, c_double],
    "cfd_step": [c_void_p, c_double, c_int],
    "cfd_reduce": [c_void_p, c_int, P(c_double), P(c_double), P(c_double)],
    "cfd_residual": [c_void_p, P(c_double)],
    "cfd_get_state": [c_void_p, P(c_double), P(c_ll)],
    "cfd_set_state": [c_void_p, c_double, c_ll],
    "cfd_copy_interior": [c_void_p, c_int, c_int, c_void_p, c_int],
    "cfd_set_host_copy": [c_void_p, c_int],
    "cfd_check": [c_void_p],
    "cfd_selftest_wait_timeout": [c_void_p, c_int],
    "cfd_last_error": [],
    "cfd_reduce_velocity_noalloc": [c_void_p, c_void_p, c_void_p, c_int, P(c_int), c_ll, c_ll,
                                    P(c_double), c_void_p, c_void_p],
    "cfd_noalloc_last_error": [],
}
RESTYPES = {"cfd_last_error": ctypes.c_char_p, "cfd_noalloc_last_error": ctypes.c_char_p}

STATUS = {0: "CFD_OK", 1: "CFD_EINVAL", 2: "CFD_ENOMEM", 3: "CFD_ECUDA", 4: "CFD_ESTATE",
          5: "CFD_EUNSUPPORTED", 6: "CFD_ENONFINITE", 7: "CFD_ETIMEOUT"}


class CfdError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__("%s returned %s: %s" % (fn, STATUS.get(status, status), msg))
        self.status = status
        self.fn = fn


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded library (built in-tree on first use if nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libgb300cfd.so missing at %s" % path)
            L = ctypes.CDLL(path)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = RESTYPES.get(name, c_int)
            _lib = L
    return _lib


def call(name: str, *args) -> None:
    """Calls an entry point and raises CfdError on a non-zero status."""
    L = lib()
    st = getattr(L, name)(*args)
    if st != 0:
        raise CfdError(st, name, L.cfd_last_error().decode())


def ints(*v):
    return (c_int * len(v))(*v)


def doubles(*v):
    return (c_double * len(v))(*v)
