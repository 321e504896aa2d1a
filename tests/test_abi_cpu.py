"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point the public header declares; argument errors (a null grid, bad
sizes, cell sizes or storage types, block sets that are not rectilinear
tilings) come back as status codes before any device call (no compute
calls without a GPU)."""
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


def test_every_grid_entry_point_rejects_a_null_grid():
    """Each call that takes a grid returns CFD_EINVAL for a null one (other
    arguments zero or null) before any device call; destroying a null grid
    is a no-op that succeeds."""
    import ctypes
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    ints = (ctypes.c_int, ctypes.c_uint, ctypes.c_longlong, ctypes.c_size_t, ctypes.c_long)
    checked = []
    for name, args in sorted(_lib.SIGNATURES.items()):
        if not args or args[0] is not ctypes.c_void_p or name.endswith("_create"):
            continue
        if "noalloc" in name:  # takes device pointers, not a grid
            continue
        vals = [None] + [0 if t in ints else 0.0 if t in (ctypes.c_double, ctypes.c_float)
                         else None for t in args[1:]]
        st = getattr(L, name)(*vals)
        assert st == (0 if name == "cfd_grid_destroy" else 1), (name, st)
        checked.append(name)
    assert "cfd_set_host_copy" in checked and "cfd_step" in checked and len(checked) > 30


@pytest.mark.parametrize("case,blocks,gd,ghost,msg", [
    ("no blocks", [], (8, 4, 4), 1, b"nblocks"),
    ("thin block", [((1, 4, 4), (0, 0, 0))], (1, 4, 4), 1, b"2*ghost"),
    ("thin for g=2", [((3, 4, 4), (0, 0, 0))], (3, 4, 4), 2, b"2*ghost"),
    ("outside", [((4, 4, 4), (6, 0, 0))], (8, 4, 4), 1, b"outside"),
    ("negative origin", [((4, 4, 4), (-1, 0, 0))], (8, 4, 4), 1, b"outside"),
    ("gap", [((4, 4, 4), (0, 0, 0)), ((3, 4, 4), (5, 0, 0))], (8, 4, 4), 1, b"rectilinear"),
    ("short", [((4, 4, 4), (0, 0, 0)), ((3, 4, 4), (4, 0, 0))], (8, 4, 4), 1, b"cover"),
    ("missing combination", [((4, 4, 4), (0, 0, 0)), ((4, 4, 4), (4, 0, 0)),
                             ((4, 4, 4), (0, 4, 0))], (8, 8, 4), 1, b"slab combination"),
    ("coincide", [((4, 4, 4), (0, 0, 0)), ((4, 4, 4), (0, 0, 0)), ((4, 4, 4), (4, 4, 0)),
                  ((4, 4, 4), (0, 4, 0))], (8, 8, 4), 1, b"coincide"),
    ("ghost 0", [((4, 4, 4), (0, 0, 0))], (4, 4, 4), 0, b"ghost width"),
])
def test_blockset_tiling_errors_on_the_host(case, blocks, gd, ghost, msg):
    """cfd_blockset_create checks the tiling (every block inside the domain
    and at least 2*ghost wide, per axis slabs that partition [0, G), one
    block per slab combination) before any device call."""
    import ctypes
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    out = ctypes.c_void_p()
    dims = [x for b in blocks for x in b[0]] or [4, 4, 4]
    origin = [x for b in blocks for x in b[1]] or [0, 0, 0]
    st = L.cfd_blockset_create(len(blocks), _lib.ints(*dims), _lib.ints(*origin), _lib.ints(*gd),
                               ghost, _lib.doubles(1, 1, 1), 0, None, ctypes.byref(out))
    assert st == 1 and out.value is None, case
    assert msg in L.cfd_last_error(), (case, L.cfd_last_error())


@pytest.mark.parametrize("h,storage,msg", [((1, 0, 1), 0, b"h[1]"), ((1, 1, float("inf")), 0, b"h[2]"),
                                           ((1, 1, 1), 3, b"storage")])
def test_grid_argument_errors_on_the_host(h, storage, msg):
    import ctypes
    from paper_1201_2118_gb300 import _lib
    L = _lib.lib()
    out = ctypes.c_void_p()
    st = L.cfd_grid_create(_lib.ints(8, 8, 8), 1, _lib.doubles(*h), storage, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert msg in L.cfd_last_error()
