"""Kernel descriptors: new stencil kernels generated from a declaration.

The paper's kernel abstraction (Sec. 3, Listing 1) has three parts: a
descriptor that declares a kernel's variables (whether each is cached and
whether it is read, written, or read and written to a separate copy), its
stencil width per face, its tile and its parameters; optimised templates;
and a generator that joins the two.  Here the descriptor is a Python object,
the template is the z-streaming tile of this library's own stencil kernels
(a CTA of 32 x ty threads owns a 32 x ty column of the grid and walks it
along z; cached inputs are staged plane by plane, halo included, in a
shared-memory ring; the other inputs are read through the read-only path),
and the generator emits CUDA C for sm_103a, checks every neighbour access
against the declared stencil, builds a shared library with nvcc (cached by
the source's hash) and loads its ``extern "C"`` launcher.

The point computation is C with these names:

  ``at(v, di, dj, dk)``  input v at offset (di, dj, dk), integer literals
                         within the stencil;
  ``out(v) = ...;``      the output v at the point;
  ``i, j, k``            the point; ``nx, ny, nz`` the interior size;
  ``idx, idy, idz``      1/h per axis; ``idx2, idy2, idz2`` 1/h^2;
  each parameter by its name (float).

Every array is FP32 storage of one single-block Grid; the caller fills the
inputs' ghosts before a launch (the stencil may not exceed the ghost width)
and the generated kernel writes interior points only.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import re
import subprocess
from dataclasses import dataclass, field

from . import build as _build

GEN_DIR = os.path.join(_build.BUILD, "generated")
MAX_ARRAYS = 16
MAX_PARAMS = 16
_AT = re.compile(r"\bat\s*\(\s*([A-Za-z_]\w*)\s*,\s*(-?\d+)\s*,\s*(-?\d+)\s*,\s*(-?\d+)\s*\)")
_AT_ANY = re.compile(r"\bat\s*\(")
_OUT = re.compile(r"\bout\s*\(\s*([A-Za-z_]\w*)\s*\)\s*=")
_NAME = re.compile(r"^[A-Za-z_]\w*$")
_RESERVED = {"i", "j", "k", "nx", "ny", "nz", "idx", "idy", "idz", "idx2", "idy2", "idz2", "at",
             "out", "a", "e", "k0", "k1", "i0", "j0", "pt", "ga", "ring", "tid", "mine", "lx", "ly",
             "lz", "load_plane"}


@dataclass
class Descriptor:
    """A stencil kernel: inputs {name: "cached" | "direct"}, outputs [names]
    (written to arrays of their own), parameters [names], stencil width per
    face (-x, +x, -y, +y, -z, +z), tile rows ty (threads 32 x ty), z chunk,
    and the point computation."""
    name: str
    inputs: dict
    outputs: list
    body: str
    params: list = field(default_factory=list)
    stencil: tuple = (1, 1, 1, 1, 1, 1)
    ty: int = 8
    zc: int = 32

    def validate(self):
        if not _NAME.match(self.name):
            raise ValueError("kernel name must be an identifier")
        names = list(self.inputs) + list(self.outputs) + list(self.params)
        for nm in names:
            if not _NAME.match(nm) or nm in _RESERVED:
                raise ValueError("bad or reserved name %r" % nm)
        if len(set(names)) != len(names):
            raise ValueError("names must be distinct across inputs, outputs and parameters")
        if not self.outputs:
            raise ValueError("a kernel needs at least one output")
        if len(self.inputs) + len(self.outputs) > MAX_ARRAYS or len(self.params) > MAX_PARAMS:
            raise ValueError("at most %d arrays and %d parameters" % (MAX_ARRAYS, MAX_PARAMS))
        for nm, mode in self.inputs.items():
            if mode not in ("cached", "direct"):
                raise ValueError("input %r: mode must be 'cached' or 'direct'" % nm)
        if len(self.stencil) != 6 or any(int(w) < 0 or int(w) > 2 for w in self.stencil):
            raise ValueError("stencil: six widths in 0..2 (-x, +x, -y, +y, -z, +z)")
        if self.ty not in (1, 2, 4, 8, 16) or not 1 <= self.zc <= 1024:
            raise ValueError("ty must be 1, 2, 4, 8 or 16 and zc in 1..1024")
        cached = sum(1 for m in self.inputs.values() if m == "cached")
        st = [int(x) for x in self.stencil]
        smem = 4 * cached * _ring(st[4] + st[5] + 2) * (32 + st[0] + st[1]) * (self.ty + st[2] + st[3])
        if smem > 48 * 1024:
            raise ValueError("cached planes need %d bytes of shared memory (> 48 KB): "
                             "use fewer cached inputs, a smaller ty or a narrower stencil" % smem)
        uses = _AT.findall(self.body)
        if len(uses) != len(_AT_ANY.findall(self.body)):
            raise ValueError("every at() needs a declared input and three integer literals")
        lo = [-int(self.stencil[0]), -int(self.stencil[2]), -int(self.stencil[4])]
        hi = [int(self.stencil[1]), int(self.stencil[3]), int(self.stencil[5])]
        for v, *off in uses:
            if v not in self.inputs:
                raise ValueError("at(%s, ...): %r is not an input" % (v, v))
            for a in range(3):
                o = int(off[a])
                if not lo[a] <= o <= hi[a]:
                    raise ValueError("at(%s, %s): offset outside the declared stencil" %
                                     (v, ", ".join(off)))
        assigned = _OUT.findall(self.body)
        for o in self.outputs:
            if o not in assigned:
                raise ValueError("output %r is never assigned" % o)
        for o in assigned:
            if o not in self.outputs:
                raise ValueError("out(%s): %r is not an output" % (o, o))
        return self


def _ring(depth: int) -> int:
    r = 1
    while r < depth:
        r *= 2
    return r


def generate(d: Descriptor) -> str:
    """CUDA source of the kernel and its extern "C" launcher."""
    d.validate()
    xm, xp, ym, yp, zm, zp = (int(w) for w in d.stencil)
    cached = [v for v, m in d.inputs.items() if m == "cached"]
    arrays = list(d.inputs) + list(d.outputs)
    slot = {v: n for n, v in enumerate(arrays)}
    sx, sy = 32 + xm + xp, d.ty + ym + yp
    ring = _ring(zm + zp + 2)
    L = []
    w = L.append
    w("// generated from kernel descriptor %s" % d.name)
    w("#include <cuda_runtime.h>")
    w("#include <stdint.h>")
    w("struct GenArgs {")
    w("  float* a[%d];  // interior origin of each array" % MAX_ARRAYS)
    w("  int py; long long pz; int n[3]; int ghost;")
    w("  float ih[3], ih2[3];")
    w("  float prm[%d];" % MAX_PARAMS)
    w("};")
    w("#define SX %d" % sx)
    w("#define SY %d" % sy)
    w("#define PL (SX * SY)")
    w("#define RING %d" % ring)
    w("#define TY %d" % d.ty)
    w("#define ZC %d" % d.zc)
    w("#define NC %d" % max(1, len(cached)))
    w("#define XM %d" % xm)
    w("#define YM %d" % ym)
    w("#define ZM %d" % zm)
    w("#define ZP %d" % zp)
    # at least 4 CTAs per SM: the register budget that leaves keeps enough
    # warps resident to hide the loads' latency
    w("extern \"C\" __global__ void __launch_bounds__(32 * TY, 4) gen_%s(GenArgs ga) {" % d.name)
    if cached:
        w("  __shared__ float ring[NC][RING][PL];")
    w("  const int nx = ga.n[0], ny = ga.n[1], nz = ga.n[2];")
    w("  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY;")
    w("  const int k0 = blockIdx.z * ZC, k1 = min(k0 + ZC, nz);")
    w("  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;")
    w("  const int tid = threadIdx.y * 32 + threadIdx.x;")
    w("  const float idx = ga.ih[0], idy = ga.ih[1], idz = ga.ih[2];")
    w("  const float idx2 = ga.ih2[0], idy2 = ga.ih2[1], idz2 = ga.ih2[2];")
    w("  (void)idx; (void)idy; (void)idz; (void)idx2; (void)idy2; (void)idz2;")
    for n, p in enumerate(d.params):
        w("  const float %s = ga.prm[%d];" % (p, n))
    w("  const int lx = nx + ga.ghost - 1, ly = ny + ga.ghost - 1, lz = nz + ga.ghost - 1;")
    if cached:
        # one plane (halo included) of every cached input into its ring slot;
        # cells beyond the allocated extent (partial tiles) are not read
        w("  auto load_plane = [&](int kk) {")
        w("    if (kk > lz) return;")
        w("    for (int e = tid; e < PL; e += 32 * TY) {")
        w("      const int xx = e % SX, yy = e / SX;")
        w("      const int gi = i0 - XM + xx, gj = j0 - YM + yy;")
        w("      if (gi > lx || gj > ly) continue;")
        w("      const long long o = (long long)kk * ga.pz + (long long)gj * ga.py + gi;")
        for c, v in enumerate(cached):
            w("      ring[%d][kk & (RING - 1)][e] = ga.a[%d][o];" % (c, slot[v]))
        w("    }")
        w("  };")
        w("  for (int kk = k0 - ZM; kk <= k0 + ZP; ++kk) load_plane(kk);")
    w("  const bool mine = i < nx && j < ny;")
    if not cached:
        # no plane ring: an unrolled z loop would only hold more addresses
        w("#pragma unroll 1")
    w("  for (int k = k0; k < k1; ++k) {")
    if cached:
        w("    __syncthreads();")
    w("    if (mine) {")
    w("      const long long pt = (long long)k * ga.pz + (long long)j * ga.py + i;")
    w("      (void)pt;")
    body = d.body

    def at_sub(m):
        v, di, dj, dk = m.group(1), int(m.group(2)), int(m.group(3)), int(m.group(4))
        if d.inputs[v] == "cached":
            c = cached.index(v)
            return ("ring[%d][(k + (%d)) & (RING - 1)][(threadIdx.y + YM + (%d)) * SX + "
                    "(threadIdx.x + XM + (%d))]" % (c, dk, dj, di))
        return "__ldg(ga.a[%d] + pt + (%d) * ga.pz + (%d) * (long long)ga.py + (%d))" % (
            slot[v], dk, dj, di)

    body = _AT.sub(at_sub, body)
    body = _OUT.sub(lambda m: "ga.a[%d][pt] =" % slot[m.group(1)], body)
    for line in body.strip().splitlines():
        w("      " + line.strip())
    w("    }")
    if cached:
        w("    __syncthreads();")
        w("    load_plane(k + ZP + 1);")
    w("  }")
    w("}")
    w("extern \"C\" int gen_%s_launch(const GenArgs* a, void* stream) {" % d.name)
    w("  dim3 grid((a->n[0] + 31) / 32, (a->n[1] + TY - 1) / TY, (a->n[2] + ZC - 1) / ZC);")
    w("  gen_%s<<<grid, dim3(32, TY), 0, (cudaStream_t)stream>>>(*a);" % d.name)
    w("  return (int)cudaGetLastError();")
    w("}")
    return "\n".join(L) + "\n"


class _GenArgs(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p * MAX_ARRAYS), ("py", ctypes.c_int),
                ("pz", ctypes.c_longlong), ("n", ctypes.c_int * 3), ("ghost", ctypes.c_int),
                ("ih", ctypes.c_float * 3), ("ih2", ctypes.c_float * 3),
                ("prm", ctypes.c_float * MAX_PARAMS)]


def compile_source(src: str, name: str) -> str:
    """nvcc -shared for sm_103a into the generated-kernel cache; returns the
    library path (reused when the same source was built before)."""
    tag = hashlib.sha256(src.encode()).hexdigest()[:16]
    os.makedirs(GEN_DIR, exist_ok=True)
    lib = os.path.join(GEN_DIR, "%s_%s.so" % (name, tag))
    if os.path.exists(lib):
        return lib
    cu = lib[:-3] + ".cu"
    with open(cu, "w") as f:
        f.write(src)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [_build.nvcc()] + _build.ARCH + ["-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                                          "-o", tmp, cu]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("generated kernel %s failed to build:\n%s" %
                           (name, r.stdout.decode(errors="replace")))
    os.replace(tmp, lib)
    return lib


class GeneratedKernel:
    """A built descriptor; call it on a Grid with {name: array id} bindings."""

    def __init__(self, d: Descriptor):
        self.d = d.validate()
        self.source = generate(d)
        self.path = compile_source(self.source, d.name)
        self._lib = ctypes.CDLL(self.path)
        self._fn = getattr(self._lib, "gen_%s_launch" % d.name)
        self._fn.argtypes = [ctypes.POINTER(_GenArgs), ctypes.c_void_p]
        self._fn.restype = ctypes.c_int

    def __call__(self, grid, bind: dict, **params):
        d = self.d
        if grid.nblocks != 1 or grid.dtype != "f32":
            raise ValueError("generated kernels run on single-block FP32 grids")
        if max(d.stencil) > grid.ghost:
            raise ValueError("the stencil is wider than the grid's ghost layer")
        names = list(d.inputs) + list(d.outputs)
        missing = [nm for nm in names if nm not in bind]
        if missing:
            raise ValueError("unbound arrays: %s" % ", ".join(missing))
        outs = [bind[o] for o in d.outputs]
        if any(bind[v] in outs for v in d.inputs) or len(set(outs)) != len(outs):
            raise ValueError("outputs must be arrays of their own (not inputs, not shared)")
        if set(params) != set(d.params):
            raise ValueError("parameters: expected %s" % sorted(d.params))
        ga = _GenArgs()
        view = grid.interior(bind[names[0]])
        for n, nm in enumerate(names):
            ga.a[n] = grid.interior(bind[nm]).data_ptr()
        ga.pz, ga.py = view.stride(0), view.stride(1)
        ga.n[:] = (view.shape[2], view.shape[1], view.shape[0])
        ga.ghost = grid.ghost
        ga.ih[:] = tuple(1.0 / x for x in grid.h)
        ga.ih2[:] = tuple(1.0 / (x * x) for x in grid.h)
        for n, p in enumerate(d.params):
            ga.prm[n] = float(params[p])
        st = self._fn(ctypes.byref(ga), ctypes.c_void_p(grid.stream.cuda_stream))
        if st != 0:
            raise RuntimeError("generated kernel %s: CUDA error %d" % (d.name, st))
