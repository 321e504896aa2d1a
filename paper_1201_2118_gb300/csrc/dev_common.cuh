// Device helpers shared by the stencil translation units: storage-type
// conversion (fields are stored as FP32, BF16 or FP16 and always computed in
// FP32), VX-wide vector access, and the ghost-on-write images of pressure
// face cells.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cfd_internal.h"

namespace cfd {
namespace {

// ------------------------------------------------------------ storage types

template <typename T> __device__ __forceinline__ float ldf(const T* p);
template <> __device__ __forceinline__ float ldf<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ldf<__half>(const __half* p) {
  return __half2float(__ldg(p));
}

template <typename T> __device__ __forceinline__ T cvt(float x);
template <> __device__ __forceinline__ float cvt<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <> __device__ __forceinline__ __half cvt<__half>(float x) { return __float2half_rn(x); }

// VX consecutive elements as one aligned vector load / store.
template <typename T, int VX> struct alignas(sizeof(T) * VX) Vec { T v[VX]; };

__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float tof(__half x) { return __half2float(x); }

template <int VX, typename T>
__device__ __forceinline__ void ldv(const T* p, float (&out)[VX]) {
  const Vec<T, VX> x = *reinterpret_cast<const Vec<T, VX>*>(p);
#pragma unroll
  for (int e = 0; e < VX; ++e) out[e] = tof(x.v[e]);
}

template <typename T, int VX>
__device__ __forceinline__ void stv(T* p, const float (&in)[VX]) {
  Vec<T, VX> x;
#pragma unroll
  for (int e = 0; e < VX; ++e) x.v[e] = cvt<T>(in[e]);
  *reinterpret_cast<Vec<T, VX>*>(p) = x;
}

template <typename T>
struct Fld {
  const T* p;
  int py;
  long long pz;
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    return ldf<T>(p + (long long)k * pz + (long long)j * py + i);
  }
};

template <typename T>
__device__ __forceinline__ Fld<T> fld(const Launch& L, const BlockDev& B, int arr) {
  return Fld<T>{reinterpret_cast<const T*>(L.base) + B.org[arr], B.py, B.pz};
}

template <typename T>
__device__ __forceinline__ T* wptr(const Launch& L, const BlockDev& B, int arr) {
  return reinterpret_cast<T*>(L.base) + B.org[arr];
}

// ------------------------------------------------------- Jacobi update
//
// One weighted Jacobi update of the 7-point operator, p' = p + w((N p - r)
// / diag - p), N p = sum over axes of (p_- + p_+) / h^2, with every rounding
// spelled out, so that every sweep kernel (scalar or packed pairs) computes
// the same bits: nb = fma(zm + zp, cz, fma(ym + yp, cy, (xm + xp) cx)),
// p' = fma(w, fma(nb - r, 1/diag, -p), p).
__device__ __forceinline__ float jacobi_update(float c, float xm, float xp, float ym, float yp,
                                               float zm, float zp, float r, float cx, float cy,
                                               float cz, float omega, float inv_diag) {
  const float nb = __fmaf_rn(__fadd_rn(zm, zp), cz,
                             __fmaf_rn(__fadd_rn(ym, yp), cy, __fmul_rn(__fadd_rn(xm, xp), cx)));
  return __fmaf_rn(omega, __fmaf_rn(__fsub_rn(nb, r), inv_diag, -c), c);
}

// Packed FP32 pairs (two floats in a 64-bit register) for the sm_100-family
// f32x2 instructions: one issue slot computes the same IEEE round-to-nearest
// operation on two cells.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpk2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// jacobi_update on two cells at once with the same roundings.  The x terms
// arrive summed (xs = xm + xp, one scalar add per cell, written straight into
// the pair).  nb = fma(zm+zp, cz, fma(ym+yp, cy, xs cx)); the update
// fma(w, fma(nb - r, 1/diag, -c), c) is taken as fma(-w, fma(r - nb, 1/diag,
// c), c): r - nb = -(nb - r) and fma(-a, b, c) = -fma(a, b, -c) exactly
// (round-to-nearest is symmetric), and -w times -x is w times x, so this is
// the same value without forming -c (an exact zero may change its sign).
struct Jac2 {
  unsigned long long cx, cy, cz, mom, inv;
  __device__ __forceinline__ Jac2(float cx_, float cy_, float cz_, float om_, float inv_)
      : cx(pk2(cx_, cx_)), cy(pk2(cy_, cy_)), cz(pk2(cz_, cz_)), mom(pk2(-om_, -om_)),
        inv(pk2(inv_, inv_)) {}
  __device__ __forceinline__ unsigned long long operator()(
      unsigned long long c, unsigned long long xs, unsigned long long ym, unsigned long long yp,
      unsigned long long zm, unsigned long long zp, unsigned long long r) const {
    const unsigned long long nb =
        fma2(add2(zm, zp), cz, fma2(add2(ym, yp), cy, mul2(xs, cx)));
    return fma2(mom, fma2(sub2(r, nb), inv, c), c);
  }
};

// four cells of a row (VX = 4) with their x neighbours left/right
__device__ __forceinline__ void jac_row4(const Jac2& J, const float (&c)[4], float left,
                                         float right, const float (&ym)[4], const float (&yp)[4],
                                         const float (&zm)[4], const float (&zp)[4],
                                         const float (&r)[4], float (&out)[4]) {
  const unsigned long long c01 = pk2(c[0], c[1]), c23 = pk2(c[2], c[3]);
  const unsigned long long x01 = pk2(__fadd_rn(left, c[1]), __fadd_rn(c[0], c[2]));
  const unsigned long long x23 = pk2(__fadd_rn(c[1], c[3]), __fadd_rn(c[2], right));
  const unsigned long long o01 = J(c01, x01, pk2(ym[0], ym[1]), pk2(yp[0], yp[1]),
                                   pk2(zm[0], zm[1]), pk2(zp[0], zp[1]), pk2(r[0], r[1]));
  const unsigned long long o23 = J(c23, x23, pk2(ym[2], ym[3]), pk2(yp[2], yp[3]),
                                   pk2(zm[2], zm[3]), pk2(zp[2], zp[3]), pk2(r[2], r[3]));
  unpk2(o01, out[0], out[1]);
  unpk2(o23, out[2], out[3]);
}

// two cells of a row (VX = 2) with their x neighbours left/right
__device__ __forceinline__ void jac_row2(const Jac2& J, const float (&c)[2], float left,
                                         float right, const float (&ym)[2], const float (&yp)[2],
                                         const float (&zm)[2], const float (&zp)[2],
                                         const float (&r)[2], float (&out)[2]) {
  const unsigned long long x01 = pk2(__fadd_rn(left, c[1]), __fadd_rn(c[0], right));
  const unsigned long long o01 = J(pk2(c[0], c[1]), x01, pk2(ym[0], ym[1]), pk2(yp[0], yp[1]),
                                   pk2(zm[0], zm[1]), pk2(zp[0], zp[1]), pk2(r[0], r[1]));
  unpk2(o01, out[0], out[1]);
}
template <int VX>
__device__ __forceinline__ void jac_row(const Jac2& J, const float (&c)[VX], float left,
                                        float right, const float (&ym)[VX], const float (&yp)[VX],
                                        const float (&zm)[VX], const float (&zp)[VX],
                                        const float (&r)[VX], float (&out)[VX]) {
  if constexpr (VX == 4) jac_row4(J, c, left, right, ym, yp, zm, zp, r, out);
  else jac_row2(J, c, left, right, ym, yp, zm, zp, r, out);
}

// ------------------------------------------------------- ghost-on-write
//
// A Jacobi sweep writes each new face value of p also into the first ghost
// layer where the next sweep reads it: across a periodic or block-to-block
// face into the neighbour block's ghost cell, at a wall into the own ghost
// cell (homogeneous Neumann, p_ghost = p_face).  Edges and corners of the
// ghost layer are never read by the 7-point operator and are not written.

template <typename T>
__device__ __forceinline__ void p_ghost_images(const Launch& L, const BlockDev& B, int dst,
                                               int i, int j, int k, T val) {
  const int q[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int face = 2 * d + side;
      if (q[d] != (side == 0 ? 0 : B.n[d] - 1)) continue;
      int t[3] = {q[0], q[1], q[2]};
      const BlockDev* D = &B;
      if (B.bc[face] == BC_PERIODIC) {
        D = &L.blocks[B.nbr[face]];
        t[d] = side == 0 ? D->n[d] : -1;
      } else {
        t[d] = side == 0 ? -1 : B.n[d];
      }
      wptr<T>(L, *D, dst)[(long long)t[2] * D->pz + (long long)t[1] * D->py + t[0]] = val;
    }
  }
}

// The x- and y-face images of one x-row of a z-column are found once per
// tile and kept in shared memory: entry f of a row (0: x low, 1: x high,
// 2: y low, 3: y high) holds the address of the image of cell (x_f, j, 0)
// and the z pitch of the block it lies in, so the per-plane work is one
// store per image.  z-face images (first and last plane of a block) use
// p_ghost_images.
template <typename T>
struct RowImage {
  T* p;
  long long pz;
};

template <typename T, int FACE>
__device__ __forceinline__ void face_image(const Launch& L, const BlockDev& B, int dst, int ti,
                                           int tj, RowImage<T>& out) {
  constexpr bool hi = FACE & 1;
  const BlockDev* D = &B;
  int t;
  if (B.bc[FACE] == BC_PERIODIC) {
    D = &L.blocks[B.nbr[FACE]];
    t = hi ? -1 : D->n[FACE >> 1];
  } else {
    t = hi ? B.n[FACE >> 1] : -1;
  }
  if (FACE < 2) ti = t; else tj = t;
  out.p = wptr<T>(L, *D, dst) + (long long)tj * D->py + ti;
  out.pz = D->pz;
}

// Fills the four entries of row j for x-row cells x0 .. x0 + w - 1 (the
// x-tile of the calling warp) and returns the mask of those that exist.
template <typename T>
__device__ __forceinline__ unsigned row_images(const Launch& L, const BlockDev& B, int dst,
                                               int x0, int w, int j, RowImage<T>* e) {
  const int nx = B.n[0], ny = B.n[1];
  unsigned m = 0;
  if (j >= ny || x0 >= nx) return 0;
  if (x0 == 0) { face_image<T, 0>(L, B, dst, 0, j, e[0]); m |= 1u; }
  if (x0 + w > nx - 1) { face_image<T, 1>(L, B, dst, nx - 1, j, e[1]); m |= 2u; }
  if (j == 0) { face_image<T, 2>(L, B, dst, x0, j, e[2]); m |= 4u; }
  if (j == ny - 1) { face_image<T, 3>(L, B, dst, x0, j, e[3]); m |= 8u; }
  return m;
}

// z-face images of cell (i, j, k) for k == 0 or k == n_z - 1.
template <typename T>
__device__ __forceinline__ void p_ghost_z(const Launch& L, const BlockDev& B, int dst, int i,
                                          int j, int k, T val) {
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int face = 4 + side;
    if (k != (side == 0 ? 0 : B.n[2] - 1)) continue;
    const BlockDev* D = &B;
    int t;
    if (B.bc[face] == BC_PERIODIC) {
      D = &L.blocks[B.nbr[face]];
      t = side == 0 ? D->n[2] : -1;
    } else {
      t = side == 0 ? -1 : B.n[2];
    }
    wptr<T>(L, *D, dst)[(long long)t * D->pz + (long long)j * D->py + i] = val;
  }
}

// Per-thread share of a row's images: bit f of the result says that the
// thread writes image f (the x images belong to the lanes holding x = 0 and
// x = n_x - 1, the y images to every lane with cells in the row).  i is the
// thread's first cell, VX cells per thread.
template <int VX>
__device__ __forceinline__ unsigned thread_images(unsigned row_mask, int lane, int i, int nx) {
  if (i >= nx) return 0;
  unsigned m = row_mask & 12u;
  if ((row_mask & 1u) && lane == 0) m |= 1u;
  if ((row_mask & 2u) && nx - 1 < i + VX) m |= 2u;
  return m;
}

// v[idx] for a register array, as a chain of predicated selects (a C++
// select chain over a runtime index becomes an indexed load from a
// local-memory copy of the array)
template <int VX>
__device__ __forceinline__ float pick(const float (&v)[VX], int idx) {
  float r = v[0];
#pragma unroll
  for (int q = 1; q < VX; ++q)
    asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, %3;\n\tselp.f32 %0, %1, %0, p;\n\t}"
        : "+f"(r)
        : "f"(v[q]), "r"(idx), "r"(q));
  return r;
}

// Writes the images the thread owns for plane k; xl = i - x0 is the
// thread's offset in the row tile, nv its number of cells inside the block.
template <typename T, int VX>
__device__ __forceinline__ void put_row_images(const RowImage<T>* e, unsigned tm, int k, int xl,
                                               int nv, const float (&out)[VX]) {
  if (tm & 1u) e[0].p[k * e[0].pz] = cvt<T>(out[0]);
  if (tm & 2u) e[1].p[k * e[1].pz] = cvt<T>(pick<VX>(out, nv - 1));
#pragma unroll
  for (int f = 2; f < 4; ++f)
    if (tm & (1u << f)) {
      T* p = e[f].p + k * e[f].pz + xl;
      if (nv >= VX) {
        stv<T, VX>(p, out);
      } else {
#pragma unroll
        for (int q = 0; q < VX; ++q)
          if (q < nv) p[q] = cvt<T>(out[q]);
      }
    }
}

}  // namespace
}  // namespace cfd
