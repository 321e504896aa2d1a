"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point the public header declares (no compute calls without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cfd_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_path_entry_points():
    names = declared_symbols()
    for need in ("cfd_grid_create", "cfd_set_bc", "cfd_rhs_eval", "cfd_pressure_solve",
                 "cfd_rk_step", "cfd_ghost_fill", "cfd_step"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_1201_2118_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1201_2118_gb300 import _lib
    assert declared_symbols() <= set(_lib.SIGNATURES)


def test_errors_without_gpu_are_status_codes():
    """Argument validation happens before any device call."""
    import ctypes
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    out = ctypes.c_void_p()
    st = L.cfd_grid_create(_lib.ints(1, 8, 8), 1, _lib.doubles(1, 1, 1), 0, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"dims" in L.cfd_last_error()
    st = L.cfd_grid_create(_lib.ints(8, 8, 8), 3, _lib.doubles(1, 1, 1), 0, None, ctypes.byref(out))
    assert st == 1
    st = L.cfd_blockset_create(2, _lib.ints(4, 4, 4, 4, 4, 4), _lib.ints(0, 0, 0, 2, 0, 0),
                               _lib.ints(8, 4, 4), 1, _lib.doubles(1, 1, 1), 0, None,
                               ctypes.byref(out))
    assert st == 1  # overlapping slabs are not a rectilinear tiling
    assert L.cfd_step(None, ctypes.c_double(0.1), 1) == 1


def test_graft_entry_build_runs():
    import __graft_entry__
    __graft_entry__.build()


def test_library_has_no_unresolved_internal_symbols():
    """Every kernel launcher the runtime calls is defined in the library."""
    import shutil
    import subprocess
    from paper_1201_2118_gb300 import build
    path = build.build()
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "-C", path], capture_output=True, text=True).stdout
    undefined = [l for l in out.splitlines() if " U " in l and "cfd::" in l]
    assert not undefined, undefined
