// Stencil kernels of the staggered-grid projection step (sm_103a).
//
// All kernels walk a flattened list of tiles over all blocks of the grid
// (one persistent launch covers every block; tiles are numbered block by
// block, x fastest, then y, then z chunks), read fields in their storage
// type, compute in FP32 and store with round-to-nearest.  Fields are
// addressed as base + org[array] + k*pz + j*py + i with i,j,k relative to the
// interior origin, so ghost cells have negative or >= n indices.
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_fp16.h>

#include "cfd_internal.h"
#include "dev_common.cuh"
#include "ffloat.cuh"
#include "tiles.cuh"

namespace cfd {
namespace {

// ------------------------------------------------------------------ ghosts
//
struct GhostArrays { int arr[kNumArrays]; int n; };

// Ghost fill of the arrays in ga.  A block's ghost shell is 26 disjoint
// boxes, one per direction (dx, dy, dz) in {-1, 0, 1}^3 other than 0; each
// is the image of one box of cells, found on the host axis by axis (x, then
// y, then z): a periodic or block-to-block face moves the source into the
// neighbouring block, a wall mirrors it within the block and composes the
// wall rule v -> A + S v (zero normal velocity, tangential 2 U_wall - v,
// pressure v).  The result is that of ghost passes x, y, z over the full
// extent, each reading the previous pass's ghosts, with nothing but copies
// between blocks.  Every source is an interior cell and every destination a
// ghost cell, so no load of a launch reads what the launch stores.
//
// The host cuts the boxes into pieces (GhostItem): an inner-axis range of
// at most kGhostItemCells cells over some rows of one plane.  Warp w of CTA
// b copies piece 8 b + w: its lanes form 2^sh columns by 32 >> sh rows, and
// in up to eight steps they pass over the range (passes steps per row
// group) and then on to the next rows, so every step is one contiguous run
// per row and no lane divides.  NA arrays are copied at a time (1, 2 or 4:
// the fewest that cover the call's arrays in one group, up to four), all
// their loads issued before any store.  One launch is about one wave of
// short-lived warps, so the piece -> block -> data chain of loads is paid
// once per warp, side by side.
constexpr int kGhostWarps = 8;
constexpr int kGhostU = 8;  // steps per piece
template <typename T, int NA>
__global__ void __launch_bounds__(32 * kGhostWarps) k_ghost(Launch L, const GhostItem* items,
                                                            int nitems,
                                                            const __grid_constant__ GhostArrays ga) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * kGhostWarps + (threadIdx.x >> 5);
  if (item >= nitems) return;
  const GhostItem it = items[item];
  const BlockDev& B = L.blocks[it.dst];
  const BlockDev& Sd = L.blocks[it.src];
  auto pick3 = [](int i, long long v0, long long v1, long long v2) {
    return i == 0 ? v0 : (i == 1 ? v1 : v2);
  };
  const long long dsi = pick3(it.ax[0], 1, B.py, B.pz), dsj = pick3(it.ax[1], 1, B.py, B.pz);
  const long long dsk = pick3(it.ax[2], 1, B.py, B.pz);
  const long long ssi = pick3(it.ax[0], 1, Sd.py, Sd.pz), ssj = pick3(it.ax[1], 1, Sd.py, Sd.pz);
  const long long ssk = pick3(it.ax[2], 1, Sd.py, Sd.pz);
  // this lane: column col of each pass, row rs of each row group
  const int W = 1 << it.sh, RPI = 32 >> it.sh;
  const int col = lane & (W - 1), rs = lane >> it.sh;
  const int i = it.i0 + col, rj = it.rj0 + rs;
  const long long sbase = (long long)(it.s0[0] + it.st[0] * i) * ssi +
                          (long long)(it.s0[1] + it.st[1] * rj) * ssj +
                          (long long)(it.s0[2] + it.st[2] * it.rk) * ssk;
  const long long dbase = (long long)(it.d0[0] + i) * dsi + (long long)(it.d0[1] + rj) * dsj +
                          (long long)(it.d0[2] + it.rk) * dsk;
  const long long sp_step = (long long)(it.st[0] * W) * ssi, st_step = (long long)(it.st[1] * RPI) * ssj;
  const long long dp_step = (long long)W * dsi, dt_step = (long long)RPI * dsj;
  // step u is pass p, row group t (u = t * passes + p); valid while the
  // column and the row are inside the piece
  unsigned valid = 0;
  {
    int p = 0, t = 0;
#pragma unroll
    for (int u = 0; u < kGhostU; ++u) {
      if (col + W * p < it.ni && rs + RPI * t < it.nrows) valid |= 1u << u;
      if (++p == it.passes) {
        p = 0;
        ++t;
      }
    }
  }
  T* const base = reinterpret_cast<T*>(L.base);
  for (int a0 = 0; a0 < ga.n; a0 += NA) {
    float v[NA][kGhostU];
    // both sides' array origins are read before any store: the block table
    // sits in global memory, so a read after a store would wait for it
    const T* sp[NA];
    T* dp[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int arr = ga.arr[a0 + q < ga.n ? a0 + q : a0];
      sp[q] = base + Sd.org[arr] + sbase;
      dp[q] = base + B.org[arr] + dbase;
    }
    {
      int p = 0, t = 0;
#pragma unroll
      for (int u = 0; u < kGhostU; ++u) {
        if (valid & (1u << u)) {
          const long long so = p * sp_step + t * st_step;
#pragma unroll
          for (int q = 0; q < NA; ++q)
            if (a0 + q < ga.n) v[q][u] = ldf<T>(sp[q] + so);
        }
        if (++p == it.passes) {
          p = 0;
          ++t;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      if (a0 + q >= ga.n) continue;
      const int arr = ga.arr[a0 + q];
      // the array's wall rule v -> A + S v, composed over the axes in order
      const int kind = array_kind(arr);
      float A = 0.f, S = 1.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (it.wface[d] < 0) continue;
        float a, s1;
        if (kind == 3) { a = 0.f; s1 = 1.f; }
        else if (kind == d) { a = 0.f; s1 = 0.f; }
        else { a = 2.f * B.wall[it.wface[d]][kind]; s1 = -1.f; }
        A = a + s1 * A;
        S = s1 * S;
      }
#pragma unroll
      for (int u = 0; u < kGhostU; ++u) v[q][u] = S != 0.f ? A + S * v[q][u] : A;
    }
    int p = 0, t = 0;
#pragma unroll
    for (int u = 0; u < kGhostU; ++u) {
      if (valid & (1u << u)) {
        const long long d = p * dp_step + t * dt_step;
#pragma unroll
        for (int q = 0; q < NA; ++q)
          if (a0 + q < ga.n) dp[q][d] = cvt<T>(v[q][u]);
      }
      if (++p == it.passes) {
        p = 0;
        ++t;
      }
    }
  }
}

// ------------------------------------------------------- RHS + stage combine

// F_C = nu lap u_C - A_C at the point (i, j, k) of component C.  Advective
// form (kSchemeAdv2/4): A_C = sum_d vel_d * du_C/dx_d with the transverse
// velocity interpolated to the point.  Conservative form (kSchemeFlux2,
// Eq. 1 rewritten with Eq. 2): A_C = sum_d (E_d(p) - E_d(p - e_d)) / h_d,
// E_d(q) the C-momentum flux through the side between the points q and
// q + e_d, the product of the means (u_C(q) + u_C(q + e_d)) / 2 and
// (u_d(q) + u_d(q + e_C)) / 2.
template <typename F, int SCH, int C>
__device__ __forceinline__ float rhs_comp(const F (&f)[3], int i, int j, int k,
                                          const float (&ih)[3], const float (&ih2)[3],
                                          float nu) {
  auto at = [&](int comp, int d1, int o1, int d2, int o2) -> float {
    int q[3] = {i, j, k};
    q[d1] += o1;
    q[d2] += o2;
    return f[comp](q[0], q[1], q[2]);
  };
  const float f0 = f[C](i, j, k);
  if constexpr (SCH == kSchemeFlux2) {
    float adv = 0.f, lap = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float p1 = at(C, d, 1, d, 0), m1 = at(C, d, -1, d, 0);
      const float ch = f0 + p1, cl = m1 + f0;  // 2 x the u_C side means
      float dh, dl;                            // 2 x the u_d side means
      if (d == C) {
        dh = ch;
        dl = cl;
      } else {
        dh = at(d, C, 0, d, 0) + at(d, C, 1, d, 0);
        dl = at(d, C, 0, d, -1) + at(d, C, 1, d, -1);
      }
      adv += (ch * dh - cl * dl) * (0.25f * ih[d]);
      lap += (p1 - 2.f * f0 + m1) * ih2[d];
    }
    return nu * lap - adv;
  } else {
    float adv = 0.f, lap = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float p1 = at(C, d, 1, d, 0), m1 = at(C, d, -1, d, 0);
      float deriv, second;
      if (SCH == kSchemeAdv2) {
        deriv = (p1 - m1) * (0.5f * ih[d]);
        second = (p1 - 2.f * f0 + m1) * ih2[d];
      } else {
        const float p2 = at(C, d, 2, d, 0), m2 = at(C, d, -2, d, 0);
        deriv = (8.f * (p1 - m1) - (p2 - m2)) * (ih[d] * (1.f / 12.f));
        second = (16.f * (p1 + m1) - 30.f * f0 - (p2 + m2)) * (ih2[d] * (1.f / 12.f));
      }
      float vel;
      if (d == C) {
        vel = f0;
      } else if (SCH == kSchemeAdv2) {
        vel = 0.25f * ((at(d, C, 0, d, -1) + at(d, C, 1, d, -1)) + (at(d, C, 0, d, 0) + at(d, C, 1, d, 0)));
      } else {
        const float w4[4] = {-1.f / 16.f, 9.f / 16.f, 9.f / 16.f, -1.f / 16.f};
        vel = 0.f;
#pragma unroll
        for (int ad = 0; ad < 4; ++ad) {
          float s = 0.f;
#pragma unroll
          for (int ac = 0; ac < 4; ++ac) s += w4[ac] * at(d, C, ac - 1, d, ad - 2);
          vel += w4[ad] * s;
        }
      }
      adv += vel * deriv;
      lap += second;
    }
    return nu * lap - adv;
  }
}

struct Set3 { int a[3]; };

template <typename T, int SCH, int TY>
__global__ void __launch_bounds__(32 * TY) k_stage(Launch L, int zc, float a, Set3 xs, float b,
                                                   Set3 ys, float cdt, Set3 os, float nu) {
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const Fld<T> y[3] = {fld<T>(L, B, ys.a[0]), fld<T>(L, B, ys.a[1]), fld<T>(L, B, ys.a[2])};
    const int k1 = min(k0 + zc, B.n[2]);
    const bool wall[3] = {B.bc[1] == BC_WALL && i == B.n[0] - 1,
                          B.bc[3] == BC_WALL && j == B.n[1] - 1, B.bc[5] == BC_WALL};
    for (int k = k0; k < k1; ++k) {
      float F[3];
      F[0] = rhs_comp<Fld<T>, SCH, 0>(y, i, j, k, ih, ih2, nu);
      F[1] = rhs_comp<Fld<T>, SCH, 1>(y, i, j, k, ih, ih2, nu);
      F[2] = rhs_comp<Fld<T>, SCH, 2>(y, i, j, k, ih, ih2, nu);
      const long long o = (long long)k * B.pz + (long long)j * B.py + i;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool wf = wall[c] && (c != 2 || k == B.n[2] - 1);
        float v = b * y[c](i, j, k) + cdt * F[c];
        if (a != 0.f) v += a * fld<T>(L, B, xs.a[c])(i, j, k);
        wptr<T>(L, B, os.a[c])[o] = cvt<T>(wf ? 0.f : v);
      }
    }
  }
}

// Shared-memory tiled RHS + stage: a CTA loads a (32 + 2H) x (8 + 2H) x
// (TZ + 2H) box of u, v, w (H = 1 for order 2, 2 for order 4) once, then
// evaluates the same rhs_comp arithmetic from shared memory for its
// 32 x 8 x TZ cells.

template <int SX, int SY>
struct SFld {
  const float* t;
  int i0, j0, k0;  // grid index of tile element (0,0,0)
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    return t[((k - k0) * SY + (j - j0)) * SX + (i - i0)];
  }
};

template <typename T, int SCH, int TZ>
__global__ void __launch_bounds__(256) k_stage_tile(Launch L, float a, Set3 xs, float b, Set3 ys,
                                                    float cdt, Set3 os, float nu) {
  constexpr int H = scheme_halo(SCH);
  constexpr int BX = 32, BY = 8, BZ = TZ;
  constexpr int SX = BX + 2 * H, SY = BY + 2 * H, SZ = BZ + 2 * H;
  constexpr int NT = SX * SY * SZ;
  __shared__ float tile[3][NT];
  __shared__ TileTable tt;
  tile_table_build(tt, L, BX, BY, BZ);
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  const int tid = threadIdx.x;
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, BX, BY, BZ, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int g = L.ghost;
    const int py = B.py;
    const long long pz = B.pz;
    // box load; cells beyond the allocated extent (partial tiles) are skipped
    const int xmax = nx + g - 1, ymax = ny + g - 1, zmax = nz + g - 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* src = reinterpret_cast<const T*>(L.base) + B.org[ys.a[c]];
      for (int idx = tid; idx < NT; idx += 256) {
        const int xx = idx % SX, yy = (idx / SX) % SY, zz = idx / (SX * SY);
        const int i = i0 - H + xx, j = j0 - H + yy, k = k0 - H + zz;
        if (i <= xmax && j <= ymax && k <= zmax)
          tile[c][idx] = ldf<T>(src + (long long)k * pz + (long long)j * py + i);
      }
    }
    __syncthreads();
    const SFld<SX, SY> f[3] = {{tile[0], i0 - H, j0 - H, k0 - H}, {tile[1], i0 - H, j0 - H, k0 - H},
                               {tile[2], i0 - H, j0 - H, k0 - H}};
    const int i = i0 + (tid & 31), j = j0 + (tid >> 5);
    if (i < nx && j < ny) {
      const bool wall[3] = {B.bc[1] == BC_WALL && i == nx - 1, B.bc[3] == BC_WALL && j == ny - 1,
                            B.bc[5] == BC_WALL};
      const int k1 = min(k0 + BZ, nz);
      for (int k = k0; k < k1; ++k) {
        float F[3];
        F[0] = rhs_comp<SFld<SX, SY>, SCH, 0>(f, i, j, k, ih, ih2, nu);
        F[1] = rhs_comp<SFld<SX, SY>, SCH, 1>(f, i, j, k, ih, ih2, nu);
        F[2] = rhs_comp<SFld<SX, SY>, SCH, 2>(f, i, j, k, ih, ih2, nu);
        const long long o = (long long)k * pz + (long long)j * py + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool wf = wall[c] && (c != 2 || k == nz - 1);
          float v = b * f[c](i, j, k) + cdt * F[c];
          if (a != 0.f) v += a * ldf<T>(reinterpret_cast<const T*>(L.base) + B.org[xs.a[c]] + o);
          reinterpret_cast<T*>(L.base)[B.org[os.a[c]] + o] = cvt<T>(wf ? 0.f : v);
        }
      }
    }
    __syncthreads();  // the next tile overwrites the box
  }
}

// z-streaming RHS + stage: a CTA owns a 32 x TY column of one block and
// walks it along z with a ring of R shared-memory planes of u, v, w (each
// 32 + 2H by TY + 2H cells, H = 1 for order 2, 2 for order 4): planes
// k - H .. k + H are resident while plane k is computed, and the loads of
// plane k + H + 1 are issued into registers before that and stored into the
// free slot after it, so every field value comes from DRAM about once and
// there is one barrier per plane.  Plane kk lives in slot kk & (R - 1).

template <int SX, int PL, int R>
struct RingFld {
  const float* t;  // ring + component * PL
  int i0, j0;      // grid index of plane element (0, 0)
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    return t[(k & (R - 1)) * (3 * PL) + (j - j0) * SX + (i - i0)];
  }
};

template <typename T, int SCH, int TY>
__global__ void __launch_bounds__(32 * TY) k_stage_ring(Launch L, int zc, float a, Set3 xs,
                                                        float b, Set3 ys, float cdt, Set3 os,
                                                        float nu) {
  constexpr int H = scheme_halo(SCH);
  constexpr int SX = 32 + 2 * H, SY = TY + 2 * H, PL = SX * SY;
  constexpr int R = H == 1 ? 4 : 8;  // >= 2H + 2, a power of two
  constexpr int NT = 32 * TY;
  constexpr int NL = (3 * PL + NT - 1) / NT;  // plane elements loaded per thread
  __shared__ float ring[R * 3 * PL];
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const T* base = reinterpret_cast<const T*>(L.base);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int g = L.ghost;
    const int py = B.py;
    const long long pz = B.pz;
    const int k1 = min(k0 + zc, nz);
    // this thread's share of a plane: ring offset and field offset (plane
    // 0) of each element; elements outside the allocated extent (partial
    // tiles) are not loaded, and only cells outside the block read them
    int soff[NL];
    long long goff[NL];
    bool lok[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int idx = tid + q * NT;
      const int c = idx / PL, rem = idx % PL;
      const int xx = rem % SX, yy = rem / SX;
      const int i = i0 - H + xx, j = j0 - H + yy;
      lok[q] = idx < 3 * PL && i <= nx + g - 1 && j <= ny + g - 1;
      soff[q] = c * PL + rem;
      goff[q] = lok[q] ? B.org[ys.a[c]] + (long long)j * py + i : 0;
    }
    const int kmax = nz + g - 1;
    auto fetch = [&](int kk, float (&v)[NL]) {
#pragma unroll
      for (int q = 0; q < NL; ++q)
        v[q] = (lok[q] && kk <= kmax) ? ldf<T>(base + goff[q] + (long long)kk * pz) : 0.f;
    };
    auto put = [&](int kk, const float (&v)[NL]) {
      float* slot = ring + (kk & (R - 1)) * (3 * PL);
#pragma unroll
      for (int q = 0; q < NL; ++q)
        if (tid + q * NT < 3 * PL) slot[soff[q]] = v[q];
    };
    for (int kk = k0 - H; kk <= k0 + H; ++kk) {
      float v[NL];
      fetch(kk, v);
      put(kk, v);
    }
    __syncthreads();
    const int i = i0 + tx, j = j0 + ty;
    const bool mine = i < nx && j < ny;
    const bool wall[3] = {B.bc[1] == BC_WALL && i == nx - 1, B.bc[3] == BC_WALL && j == ny - 1,
                          B.bc[5] == BC_WALL};
    const long long o0 = (long long)j * py + i;
    const T* X[3] = {base + B.org[xs.a[0]] + o0, base + B.org[xs.a[1]] + o0,
                     base + B.org[xs.a[2]] + o0};
    T* O[3] = {reinterpret_cast<T*>(L.base) + B.org[os.a[0]] + o0,
               reinterpret_cast<T*>(L.base) + B.org[os.a[1]] + o0,
               reinterpret_cast<T*>(L.base) + B.org[os.a[2]] + o0};
    const RingFld<SX, PL, R> f[3] = {{ring, i0 - H, j0 - H}, {ring + PL, i0 - H, j0 - H},
                                     {ring + 2 * PL, i0 - H, j0 - H}};
    for (int k = k0; k < k1; ++k) {
      const int kn = k + H + 1;
      const bool more = kn <= k1 - 1 + H;
      float nxt[NL];
      if (more) fetch(kn, nxt);
      if (mine) {
        float F[3];
        F[0] = rhs_comp<RingFld<SX, PL, R>, SCH, 0>(f, i, j, k, ih, ih2, nu);
        F[1] = rhs_comp<RingFld<SX, PL, R>, SCH, 1>(f, i, j, k, ih, ih2, nu);
        F[2] = rhs_comp<RingFld<SX, PL, R>, SCH, 2>(f, i, j, k, ih, ih2, nu);
        const long long o = (long long)k * pz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool wf = wall[c] && (c != 2 || k == nz - 1);
          float v = b * f[c](i, j, k) + cdt * F[c];
          if (a != 0.f) v += a * ldf<T>(X[c] + o);
          O[c][o] = cvt<T>(wf ? 0.f : v);
        }
      }
      if (more) put(kn, nxt);
      __syncthreads();
    }
  }
}

// --------------------------------------------------------------- divergence
//
// Both walk 32 x TY columns along z with one cell per thread; the block's
// pointers are taken into registers once per tile (the output stores could
// alias the block table as far as the compiler knows) and the z-neighbour
// read by one plane is kept for the next.  The divergence takes the wall
// rule for the normal component below a low wall face itself, so on an
// all-wall grid its input needs no ghost fill.

template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) k_div(Launch L, int zc, Set3 ws, float inv_cdt,
                                                 int r_arr) {
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  const float ihx = L.ih[0], ihy = L.ih[1], ihz = L.ih[2];
  const T* base = reinterpret_cast<const T*>(L.base);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const int py = B.py;
    const long long pz = B.pz;
    const int kn = min(k0 + zc, B.n[2]) - k0;
    const long long o0 = (long long)k0 * pz + (long long)j * py + i;
    const T* u = base + B.org[ws.a[0]] + o0;
    const T* v = base + B.org[ws.a[1]] + o0;
    const T* w = base + B.org[ws.a[2]] + o0;
    T* r = reinterpret_cast<T*>(L.base) + B.org[r_arr] + o0;
    // the normal component one cell below a low face: at a wall it is the
    // wall's normal velocity, 0 (the ghost rule), read without the ghost
    const bool wx = B.bc[0] == BC_WALL && i == 0, wy = B.bc[2] == BC_WALL && j == 0;
    float wm = (B.bc[4] == BC_WALL && k0 == 0) ? 0.f : ldf<T>(w - pz);
#pragma unroll 1
    for (int q = 0; q < kn; ++q) {
      const long long o = (long long)q * pz;
      const float wc = ldf<T>(w + o);
      const float um = wx ? 0.f : ldf<T>(u + o - 1);
      const float vm = wy ? 0.f : ldf<T>(v + o - py);
      const float d = (ldf<T>(u + o) - um) * ihx + (ldf<T>(v + o) - vm) * ihy + (wc - wm) * ihz;
      r[o] = cvt<T>(d * inv_cdt);
      wm = wc;
    }
  }
}

// --------------------------------------------------------------- projection

template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) k_project(Launch L, int zc, Set3 ws, int p_arr,
                                                     float cdt, Set3 os) {
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  const float ihx = L.ih[0], ihy = L.ih[1], ihz = L.ih[2];
  const T* base = reinterpret_cast<const T*>(L.base);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= nx || j >= ny) continue;
    const int py = B.py;
    const long long pz = B.pz;
    const int kn = min(k0 + zc, nz) - k0;
    const long long o0 = (long long)k0 * pz + (long long)j * py + i;
    const T* P = base + B.org[p_arr] + o0;
    const T* W[3] = {base + B.org[ws.a[0]] + o0, base + B.org[ws.a[1]] + o0,
                     base + B.org[ws.a[2]] + o0};
    T* U[3] = {reinterpret_cast<T*>(L.base) + B.org[os.a[0]] + o0,
               reinterpret_cast<T*>(L.base) + B.org[os.a[1]] + o0,
               reinterpret_cast<T*>(L.base) + B.org[os.a[2]] + o0};
    const bool wx = B.bc[1] == BC_WALL && i == nx - 1;
    const bool wy = B.bc[3] == BC_WALL && j == ny - 1;
    const int kwall = B.bc[5] == BC_WALL ? nz - 1 - k0 : -1;
    float pc = ldf<T>(P);
#pragma unroll 1
    for (int q = 0; q < kn; ++q) {
      const long long o = (long long)q * pz;
      const float pzn = ldf<T>(P + o + pz);
      const float g[3] = {(ldf<T>(P + o + 1) - pc) * ihx, (ldf<T>(P + o + py) - pc) * ihy,
                          (pzn - pc) * ihz};
      const bool wf[3] = {wx, wy, q == kwall};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = ldf<T>(W[c] + o) - cdt * g[c];
        U[c][o] = cvt<T>(wf[c] ? 0.f : v);
      }
      pc = pzn;
    }
  }
}

// Whole-array copy (every plane, row and padding element of each block's
// array; an array is one contiguous 128-byte-aligned span of planes x pz
// elements starting g planes, g rows and 128 bytes before the interior
// origin), in 16-byte vectors.
template <typename T>
__global__ void __launch_bounds__(256) k_copy(Launch L, int src, int dst) {
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int xo = kAlignBytes / (int)sizeof(T);
  const int g = L.ghost;
  for (int b = L.b0; b < L.b0 + L.nblocks; ++b) {
    const BlockDev& B = L.blocks[b];
    const long long lead = (long long)g * B.pz + (long long)g * B.py + xo;
    const long long n = (long long)(B.n[2] + 2 * g) * B.pz / V;
    const uint4* s4 =
        reinterpret_cast<const uint4*>(reinterpret_cast<const T*>(L.base) + B.org[src] - lead);
    uint4* d4 = reinterpret_cast<uint4*>(reinterpret_cast<T*>(L.base) + B.org[dst] - lead);
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
      d4[i] = s4[i];
  }
}

// ------------------------------------------------------------------- Jacobi
//
// One weighted Jacobi sweep of the 7-point operator, p' = p + w((N p - r)/diag - p),
// N p = sum_d (p_{+d} + p_{-d}) / h_d^2.  A CTA of 32 x TY threads owns a
// (32 VX) x TY column of one block and streams it along z: the z-neighbours
// stay in registers (planes k-1, k, k+1), the x-neighbours come from the
// neighbouring lane by warp shuffle (one halo load per row end), the
// y-neighbours from a shared-memory copy of plane k (two halo rows).  The
// loads of plane k+1 are issued before plane k is computed.
//
// Ghost-on-write: the 7-point operators read only the first ghost layer of
// p at faces, so a thread that writes a face cell also writes its image into
// that layer (the neighbouring block's ghost for a periodic/neighbour face,
// the mirror ghost for a zero-gradient wall).  Each such ghost cell has one
// owner, so there is no separate halo launch per sweep.

template <typename T, int VX, int TY>
__global__ void __launch_bounds__(32 * TY) k_jacobi(Launch L, int zc, int src, int dst,
                                                    int r_arr, float omega, float inv_diag) {
  constexpr int TX = 32 * VX;
  __shared__ __align__(16) float sm[TY + 2][TX];
  __shared__ RowImage<T> rimg[TY][4];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  __shared__ TileTable tt;
  tile_table_build(tt, L, TX, TY, zc);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int py = B.py;
    const long long pz = B.pz;
    const T* P = reinterpret_cast<const T*>(L.base) + B.org[src];
    const T* R = reinterpret_cast<const T*>(L.base) + B.org[r_arr];
    T* Q = wptr<T>(L, B, dst);
    const int i = i0 + lane * VX;
    const int j = j0 + ty;
    __syncwarp();
    unsigned rm = 0;
    if (lane == 0) rm = row_images<T>(L, B, dst, i0, TX, j, rimg[ty]);
    const unsigned tm = thread_images<VX>(__shfl_sync(0xffffffffu, rm, 0), lane, i, nx);
    const int nv = min(VX, nx - i);
    __syncwarp();
    const int k1 = min(k0 + zc, nz);
    // loads stay inside allocated rows: columns up to nx (first ghost) and
    // rows up to ny (first ghost) are what the interior outputs need
    const bool ld_col = i <= nx;
    const bool ld_row = j <= ny;
    const bool ld = ld_col && ld_row;
    const bool halo_lo = (ty == 0);                 // row j0 - 1 (>= -1, valid)
    const bool halo_hi = (ty == TY - 1) && ld_col && (j0 + TY <= ny);
    const bool xl_ld = (lane == 0) && ld_row;      // column i0 - 1 (>= -1, valid)
    const bool xr_ld = (lane == 31) && ld_row && (i0 + TX <= nx);
    const long long row = (long long)j * py + i;
    const long long row_lo = (long long)(j0 - 1) * py + i;
    const long long row_hi = (long long)(j0 + TY) * py + i;
    const long long xl_off = (long long)j * py + (i0 - 1);
    const long long xr_off = (long long)j * py + (i0 + TX);

    float m[VX], c[VX], q[VX], rr[VX], hl[VX], hh[VX];
    float xl = 0.f, xr = 0.f;
#pragma unroll
    for (int e = 0; e < VX; ++e) m[e] = c[e] = q[e] = rr[e] = hl[e] = hh[e] = 0.f;
    if (ld) {
      ldv<VX>(P + (long long)(k0 - 1) * pz + row, m);
      ldv<VX>(P + (long long)k0 * pz + row, c);
      ldv<VX>(P + (long long)(k0 + 1) * pz + row, q);
      ldv<VX>(R + (long long)k0 * pz + row, rr);
    }
    if (halo_lo && ld_col) ldv<VX>(P + (long long)k0 * pz + row_lo, hl);
    if (halo_hi) ldv<VX>(P + (long long)k0 * pz + row_hi, hh);
    if (xl_ld) xl = ldf<T>(P + (long long)k0 * pz + xl_off);
    if (xr_ld) xr = ldf<T>(P + (long long)k0 * pz + xr_off);

    for (int k = k0; k < k1; ++k) {
      // issue the loads of plane k+1 (used next iteration)
      const bool more = (k + 1 < k1);
      float qn[VX], rn[VX], hln[VX], hhn[VX];
      float xln = 0.f, xrn = 0.f;
#pragma unroll
      for (int e = 0; e < VX; ++e) qn[e] = rn[e] = hln[e] = hhn[e] = 0.f;
      if (more) {
        const long long pk = (long long)(k + 1) * pz;
        if (ld) {
          ldv<VX>(P + pk + pz + row, qn);
          ldv<VX>(R + pk + row, rn);
        }
        if (halo_lo && ld_col) ldv<VX>(P + pk + row_lo, hln);
        if (halo_hi) ldv<VX>(P + pk + row_hi, hhn);
        if (xl_ld) xln = ldf<T>(P + pk + xl_off);
        if (xr_ld) xrn = ldf<T>(P + pk + xr_off);
      }
      // plane k into shared memory (interior rows + two halo rows)
      if constexpr (VX == 4) {
        *reinterpret_cast<float4*>(&sm[ty + 1][lane * 4]) = make_float4(c[0], c[1], c[2], c[3]);
        if (halo_lo) *reinterpret_cast<float4*>(&sm[0][lane * 4]) = make_float4(hl[0], hl[1], hl[2], hl[3]);
        if (ty == TY - 1) *reinterpret_cast<float4*>(&sm[TY + 1][lane * 4]) = make_float4(hh[0], hh[1], hh[2], hh[3]);
      } else if constexpr (VX == 2) {
        *reinterpret_cast<float2*>(&sm[ty + 1][lane * 2]) = make_float2(c[0], c[1]);
        if (halo_lo) *reinterpret_cast<float2*>(&sm[0][lane * 2]) = make_float2(hl[0], hl[1]);
        if (ty == TY - 1) *reinterpret_cast<float2*>(&sm[TY + 1][lane * 2]) = make_float2(hh[0], hh[1]);
      } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) {
          sm[ty + 1][lane * VX + e] = c[e];
          if (halo_lo) sm[0][lane * VX + e] = hl[e];
          if (ty == TY - 1) sm[TY + 1][lane * VX + e] = hh[e];
        }
      }
      float left = __shfl_up_sync(0xffffffffu, c[VX - 1], 1);
      float right = __shfl_down_sync(0xffffffffu, c[0], 1);
      if (lane == 0) left = xl;
      if (lane == 31) right = xr;
      __syncthreads();
      float dn[VX], up[VX];
      if constexpr (VX == 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&sm[ty][lane * 4]);
        const float4 b4 = *reinterpret_cast<const float4*>(&sm[ty + 2][lane * 4]);
        dn[0] = a4.x; dn[1] = a4.y; dn[2] = a4.z; dn[3] = a4.w;
        up[0] = b4.x; up[1] = b4.y; up[2] = b4.z; up[3] = b4.w;
      } else if constexpr (VX == 2) {
        const float2 a2 = *reinterpret_cast<const float2*>(&sm[ty][lane * 2]);
        const float2 b2 = *reinterpret_cast<const float2*>(&sm[ty + 2][lane * 2]);
        dn[0] = a2.x; dn[1] = a2.y;
        up[0] = b2.x; up[1] = b2.y;
      } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) { dn[e] = sm[ty][lane * VX + e]; up[e] = sm[ty + 2][lane * VX + e]; }
      }
      float out[VX];
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        const float xm = e == 0 ? left : c[e - 1];
        const float xp = e == VX - 1 ? right : c[e + 1];
        out[e] = jacobi_update(c[e], xm, xp, dn[e], up[e], m[e], q[e], rr[e], cx, cy, cz,
                                 omega, inv_diag);
      }
      if (j < ny) {
        T* qrow = Q + (long long)k * pz + row;
        if (i + VX <= nx) {
          stv<T, VX>(qrow, out);
        } else {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (i + e < nx) qrow[e] = cvt<T>(out[e]);
        }
        if (tm) put_row_images<T, VX>(rimg[ty], tm, k, lane * VX, nv, out);
        if (k == 0 || k == nz - 1) {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (i + e < nx) p_ghost_z<T>(L, B, dst, i + e, j, k, cvt<T>(out[e]));
        }
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        m[e] = c[e];
        c[e] = q[e];
        q[e] = qn[e];
        rr[e] = rn[e];
        hl[e] = hln[e];
        hh[e] = hhn[e];
      }
      xl = xln;
      xr = xrn;
    }
  }
}

// cp.async-staged sweep: every thread copies its own 16-byte pieces of the
// next planes of p (with the x and y halo) and r into an S-stage shared
// memory ring (cp.async.commit_group / wait_group), so S - 4 planes are in
// flight without holding registers; one barrier per plane.  A plane stage is
// (TY + 2) rows of PW = TX + 2 HX elements of p (HX = 16 bytes of halo pad
// on each side; the x halo cells sit next to the interior) and TY x TX of r.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_n(void* smem, const void* gmem) {
  if constexpr (BYTES == 16) cp_async16(smem, gmem);
  else if constexpr (BYTES == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}

__device__ __forceinline__ void cp_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// 4-byte cp.async to a shared-memory byte address.  No memory clobber: the
// caller orders the copies against its own shared-memory accesses with
// cp.async.wait_group and barriers (which clobber memory), and a clobber
// here would pin the caller's per-thread index arrays to local memory.
__device__ __forceinline__ void cp_async4_s(uint32_t saddr, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gmem));
}

__device__ __forceinline__ void cp_async16_s(uint32_t saddr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gmem));
}

// Copies of plane kk of u, v, w (this thread's share: 16-byte pieces of the
// rows' interior, 4-byte halo cells) into its ring slot, then one commit
// group (empty past the last plane, so that "all but the newest D groups"
// always means the same planes).  width[q]: 16, 4, or 0 (nothing to copy).
template <int NL, int SLOT_BYTES>
__device__ __forceinline__ void stage_issue(uint32_t ring_s, int ring_mask, const int (&soff)[NL],
                                            const long long (&goff)[NL], const int (&width)[NL],
                                            const float* base, int kk, long long pz, bool live) {
  if (live) {
    const uint32_t slot = ring_s + (uint32_t)((kk & ring_mask) * SLOT_BYTES);
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const float* src = base + goff[q] + (long long)kk * pz;
      if (width[q] == 16) cp_async16_s(slot + soff[q], src);
      else if (width[q] == 4) cp_async4_s(slot + soff[q], src);
    }
  }
  cp_commit_group();
}

// FP32 variant of the z-streaming RHS + stage ring: planes of u, v, w are
// copied into the ring with cp.async two planes ahead of the last one the
// stencil needs (no registers hold them, no second pass through registers),
// eight slots so that a slot is rewritten only after every thread has left
// the planes that read it; the stage-2 input is loaded before the plane's
// barrier so its latency overlaps the wait.  Same arithmetic (rhs_comp) and
// results as k_stage_ring.
template <int SCH, int TY>
__global__ void __launch_bounds__(32 * TY) k_stage_async(Launch L, int zc, float a, Set3 xs,
                                                         float b, Set3 ys, float cdt, Set3 os,
                                                         float nu) {
  constexpr int H = scheme_halo(SCH);
  constexpr int D = 2;  // planes in flight beyond k + H
  // a ring row holds x = i0 - XP .. i0 + 31 + XP: the 32 interior cells start
  // 16-byte aligned (column XP), so they arrive as eight 16-byte copies; the
  // H halo cells on each side as 4-byte copies
  constexpr int XP = 4;
  constexpr int SX = 32 + 2 * XP, SY = TY + 2 * H, PL = SX * SY;
  constexpr int R = 8;  // >= 2H + 1 + D and a power of two
  static_assert(2 * H + 1 + D <= R && H <= XP, "ring too small");
  constexpr int NT = 32 * TY;
  constexpr int U = 8 + 2 * H;  // copies per row
  constexpr int NU = 3 * SY * U;
  constexpr int NL = (NU + NT - 1) / NT;
  __shared__ __align__(16) float ring[R * 3 * PL];
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const float* base = reinterpret_cast<const float*>(L.base);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int g = L.ghost;
    const int py = B.py;
    const long long pz = B.pz;
    const int k1 = min(k0 + zc, nz);
    // this thread's copies of a plane: ring byte offset, field offset
    // (plane 0) and width.  A copy starting beyond the allocated extent
    // (partial tiles) is dropped; a 16-byte piece that starts inside may
    // run up to 3 cells past the row's last allocated cell, which stays
    // inside the arena (row pitch, or its 256-byte tail), and only threads
    // outside the block read those cells
    int soff[NL], width[NL];
    long long goff[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int idx = tid + q * NT;
      const int c = idx / (SY * U), rem = idx % (SY * U);
      const int yy = rem / U, cu = rem % U;
      const int x = cu < 8 ? i0 + 4 * cu : (cu - 8 < H ? i0 - H + (cu - 8) : i0 + 32 + (cu - 8 - H));
      const int j = j0 - H + yy;
      const bool ok = idx < NU && x <= nx + g - 1 && j <= ny + g - 1;
      width[q] = ok ? (cu < 8 ? 16 : 4) : 0;
      soff[q] = 4 * (c * PL + yy * SX + XP + (x - i0));
      goff[q] = ok ? B.org[ys.a[c]] + (long long)j * py + x : 0;
    }
    const int kmax = nz + g - 1;
    const int klast = k1 - 1 + H;  // last plane the tile reads
    // one commit group per plane, empty groups past the last plane, so that
    // "all but the newest D groups" always means "up to plane k + H"
    const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));
    for (int kk = k0 - H; kk <= k0 + H + D - 1; ++kk)
      stage_issue<NL, 3 * PL * 4>(ring_s, R - 1, soff, goff, width, base, kk, pz,
                                    kk <= klast && kk <= kmax);
    const int i = i0 + tx, j = j0 + ty;
    const bool mine = i < nx && j < ny;
    const bool wall[3] = {B.bc[1] == BC_WALL && i == nx - 1, B.bc[3] == BC_WALL && j == ny - 1,
                          B.bc[5] == BC_WALL};
    const long long o0 = (long long)j * py + i;
    const float* X[3] = {base + B.org[xs.a[0]] + o0, base + B.org[xs.a[1]] + o0,
                         base + B.org[xs.a[2]] + o0};
    float* O[3] = {reinterpret_cast<float*>(L.base) + B.org[os.a[0]] + o0,
                   reinterpret_cast<float*>(L.base) + B.org[os.a[1]] + o0,
                   reinterpret_cast<float*>(L.base) + B.org[os.a[2]] + o0};
    const RingFld<SX, PL, R> f[3] = {{ring, i0 - XP, j0 - H}, {ring + PL, i0 - XP, j0 - H},
                                     {ring + 2 * PL, i0 - XP, j0 - H}};
    for (int k = k0; k < k1; ++k) {
      {  // plane k + H + D; its slot was last read D + 1 planes ago or more
        const int kk = k + H + D;
        stage_issue<NL, 3 * PL * 4>(ring_s, R - 1, soff, goff, width, base, kk, pz,
                                    kk <= klast && kk <= kmax);
      }
      const long long o = (long long)k * pz;
      float xv[3] = {0.f, 0.f, 0.f};
      if (a != 0.f && mine) {
#pragma unroll
        for (int c = 0; c < 3; ++c) xv[c] = __ldg(X[c] + o);
      }
      cp_wait_group<D>();  // this thread's copies of planes .. k + H have landed
      __syncthreads();
      if (mine) {
        float F[3];
        F[0] = rhs_comp<RingFld<SX, PL, R>, SCH, 0>(f, i, j, k, ih, ih2, nu);
        F[1] = rhs_comp<RingFld<SX, PL, R>, SCH, 1>(f, i, j, k, ih, ih2, nu);
        F[2] = rhs_comp<RingFld<SX, PL, R>, SCH, 2>(f, i, j, k, ih, ih2, nu);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool wf = wall[c] && (c != 2 || k == nz - 1);
          float v = b * f[c](i, j, k) + cdt * F[c];
          if (a != 0.f) v += a * xv[c];
          O[c][o] = wf ? 0.f : v;
        }
      }
    }
    cp_wait_group<0>();  // (only empty groups can be pending) before the next tile's copies
    __syncthreads();
  }
}

// Two x-neighbouring cells per thread (FP32, order-2 schemes): the same
// ring as k_stage_async, 64 cells wide, and the right-hand side of
// rhs_comp evaluated on the pair with packed f32x2 operations (one issue
// for both cells).  A pair of values at x offsets (di, di + 1) from the
// thread's first cell is one aligned 8-byte shared load for even di, or the
// high and low halves of the two aligned pairs around it for odd di.
__device__ __forceinline__ unsigned long long pair_join(unsigned long long a, unsigned long long b) {
  float a0, a1, b0, b1;
  unpk2(a, a0, a1);
  unpk2(b, b0, b1);
  return pk2(a1, b0);
}

template <int SCH, int C, typename LD>
__device__ __forceinline__ unsigned long long rhs_pair(const LD& ld, const float (&ih)[3],
                                                       const float (&ih2)[3], float nu) {
  // offset (0, 0, 0) moved by o1 along axis d1 and o2 along axis d2
  auto at = [&](int comp, int d1, int o1, int d2, int o2) {
    int q[3] = {0, 0, 0};
    q[d1] += o1;
    q[d2] += o2;
    return ld(comp, q[0], q[1], q[2]);
  };
  const unsigned long long f0 = at(C, 0, 0, 0, 0);
  const unsigned long long m2 = pk2(-2.f, -2.f);
  unsigned long long adv = pk2(0.f, 0.f), lap = pk2(0.f, 0.f);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const unsigned long long p1 = at(C, d, 1, d, 0), m1 = at(C, d, -1, d, 0);
    const unsigned long long second = mul2(add2(fma2(m2, f0, p1), m1), pk2(ih2[d], ih2[d]));
    if constexpr (SCH == kSchemeFlux2) {
      const unsigned long long ch = add2(f0, p1), cl = add2(m1, f0);
      unsigned long long dh, dl;
      if (d == C) {
        dh = ch;
        dl = cl;
      } else {
        dh = add2(at(d, C, 0, d, 0), at(d, C, 1, d, 0));
        dl = add2(at(d, C, 0, d, -1), at(d, C, 1, d, -1));
      }
      const float q = 0.25f * ih[d];
      adv = fma2(sub2(mul2(ch, dh), mul2(cl, dl)), pk2(q, q), adv);
    } else {
      const float hh = 0.5f * ih[d];
      const unsigned long long deriv = mul2(sub2(p1, m1), pk2(hh, hh));
      unsigned long long vel;
      if (d == C) {
        vel = f0;
      } else {
        vel = mul2(pk2(0.25f, 0.25f),
                   add2(add2(at(d, C, 0, d, -1), at(d, C, 1, d, -1)),
                        add2(at(d, C, 0, d, 0), at(d, C, 1, d, 0))));
      }
      adv = fma2(vel, deriv, adv);
    }
    lap = add2(lap, second);
  }
  return fma2(pk2(nu, nu), lap, mul2(adv, pk2(-1.f, -1.f)));
}

template <int SCH, int TY>
__global__ void __launch_bounds__(32 * TY) k_stage_pair(Launch L, int zc, float a, Set3 xs,
                                                        float b, Set3 ys, float cdt, Set3 os,
                                                        float nu) {
  static_assert(SCH == kSchemeAdv2 || SCH == kSchemeFlux2, "order-2 schemes only");
  constexpr int H = 1;
  constexpr int D = 2;    // planes in flight beyond k + H
  constexpr int TX = 64;  // cells per CTA row
  constexpr int XP = 4;   // ring column of x = i0 - XP is 0: the interior starts 16-byte aligned
  constexpr int SX = TX + 2 * XP, SY = TY + 2 * H, PL = SX * SY;
  constexpr int R = 8;
  static_assert(2 * H + 1 + D <= R, "ring too small");
  constexpr int NT = 32 * TY;
  constexpr int U = TX / 4 + 2 * H;  // copies per row: 16-byte interior pieces, 4-byte halo cells
  constexpr int NU = 3 * SY * U;
  constexpr int NL = (NU + NT - 1) / NT;
  __shared__ __align__(16) float ring[R * 3 * PL];
  __shared__ TileTable tt;
  tile_table_build(tt, L, TX, TY, zc);
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const float* base = reinterpret_cast<const float*>(L.base);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int g = L.ghost;
    const int py = B.py;
    const long long pz = B.pz;
    const int k1 = min(k0 + zc, nz);
    // this thread's copies of a plane (as in k_stage_async)
    int soff[NL], width[NL];
    long long goff[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int idx = tid + q * NT;
      const int c = idx / (SY * U), rem = idx % (SY * U);
      const int yy = rem / U, cu = rem % U;
      constexpr int NC = TX / 4;
      const int x = cu < NC ? i0 + 4 * cu : (cu - NC < H ? i0 - H + (cu - NC) : i0 + TX + (cu - NC - H));
      const int j = j0 - H + yy;
      const bool ok = idx < NU && x <= nx + g - 1 && j <= ny + g - 1;
      width[q] = ok ? (cu < NC ? 16 : 4) : 0;
      soff[q] = 4 * (c * PL + yy * SX + XP + (x - i0));
      goff[q] = ok ? B.org[ys.a[c]] + (long long)j * py + x : 0;
    }
    const int kmax = nz + g - 1;
    const int klast = k1 - 1 + H;
    const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));
    for (int kk = k0 - H; kk <= k0 + H + D - 1; ++kk)
      stage_issue<NL, 3 * PL * 4>(ring_s, R - 1, soff, goff, width, base, kk, pz,
                                  kk <= klast && kk <= kmax);
    const int i = i0 + 2 * tx, j = j0 + ty;
    const bool mine = i < nx && j < ny;
    const bool two = i + 1 < nx;  // the second cell of the pair is inside the block
    const bool wall_y = B.bc[3] == BC_WALL && j == ny - 1;
    const bool wall_z = B.bc[5] == BC_WALL;
    // wall-normal u on the +x wall face: the last cell in x, either lane
    const bool wx0 = B.bc[1] == BC_WALL && i == nx - 1, wx1 = B.bc[1] == BC_WALL && i + 1 == nx - 1;
    const long long o0 = (long long)j * py + i;
    const int cell = (ty + H) * SX + XP + 2 * tx;
    for (int k = k0; k < k1; ++k) {
      {
        const int kk = k + H + D;
        stage_issue<NL, 3 * PL * 4>(ring_s, R - 1, soff, goff, width, base, kk, pz,
                                    kk <= klast && kk <= kmax);
      }
      const long long o = (long long)k * pz + o0;
      unsigned long long xv[3] = {0ull, 0ull, 0ull};
      if (a != 0.f && mine) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* xp = base + B.org[xs.a[c]] + o;
          xv[c] = two ? __ldg(reinterpret_cast<const unsigned long long*>(xp)) : pk2(__ldg(xp), 0.f);
        }
      }
      cp_wait_group<D>();
      __syncthreads();
      if (mine) {
        auto ld = [&](int comp, int di, int dj, int dk) -> unsigned long long {
          const float* pl = ring + ((k + dk) & (R - 1)) * (3 * PL) + comp * PL + cell + dj * SX;
          if ((di & 1) == 0) return *reinterpret_cast<const unsigned long long*>(pl + di);
          return pair_join(*reinterpret_cast<const unsigned long long*>(pl + di - 1),
                           *reinterpret_cast<const unsigned long long*>(pl + di + 1));
        };
        unsigned long long F[3];
        F[0] = rhs_pair<SCH, 0>(ld, ih, ih2, nu);
        F[1] = rhs_pair<SCH, 1>(ld, ih, ih2, nu);
        F[2] = rhs_pair<SCH, 2>(ld, ih, ih2, nu);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          unsigned long long v = fma2(pk2(cdt, cdt), F[c], mul2(pk2(b, b), ld(c, 0, 0, 0)));
          if (a != 0.f) v = fma2(pk2(a, a), xv[c], v);
          float v0, v1;
          unpk2(v, v0, v1);
          bool w0, w1;
          if (c == 0) { w0 = wx0; w1 = wx1; }
          else if (c == 1) { w0 = w1 = wall_y; }
          else { w0 = w1 = wall_z && k == nz - 1; }
          if (w0) v0 = 0.f;
          if (w1) v1 = 0.f;
          float* op = reinterpret_cast<float*>(L.base) + B.org[os.a[c]] + o;
          if (two) *reinterpret_cast<unsigned long long*>(op) = pk2(v0, v1);
          else *op = v0;
        }
      }
    }
    cp_wait_group<0>();
    __syncthreads();
  }
}

template <typename T, int VX, int TY, int S>
struct AsyncGeom {
  static constexpr int TX = 32 * VX;
  static constexpr int HX = 16 / (int)sizeof(T);
  static constexpr int PW = TX + 2 * HX;
  static constexpr int PELEMS = (TY + 2) * PW;
  static constexpr int RELEMS = TY * TX;
  static constexpr int STAGE_BYTES = ((PELEMS + RELEMS) * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int SMEM = S * STAGE_BYTES;
};

template <typename T, int VX, int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_jacobi_async(Launch L, int zc, int src, int dst,
                                                          int r_arr, float omega,
                                                          float inv_diag) {
  using Gm = AsyncGeom<T, VX, TY, S>;
  constexpr int TX = Gm::TX, HX = Gm::HX, PW = Gm::PW;
  constexpr int VB = VX * (int)sizeof(T);          // bytes per thread vector
  constexpr int XB = sizeof(T) == 4 ? 4 : 4;       // x-halo copy: 1 float or 2 halves
  constexpr int XE = XB / (int)sizeof(T);          // elements in an x-halo copy
  static_assert(S >= 4, "ring needs at least 4 stages");
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  __shared__ TileTable tt;
  tile_table_build(tt, L, TX, TY, zc);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int py = B.py;
    const long long pz = B.pz;
    const int i = i0 + lane * VX;
    const int j = j0 + ty;
    const int k1 = min(k0 + zc, nz);
    const int np = k1 - k0 + 2;  // planes k0 - 1 .. k1
    const T* P0 = reinterpret_cast<const T*>(L.base) + B.org[src];
    const T* R0 = reinterpret_cast<const T*>(L.base) + B.org[r_arr];
    // what this thread copies for every plane
    const bool cp_row = i <= nx && j <= ny;
    const bool cp_r = i <= nx && j < ny;
    const bool cp_lo = ty == 0 && i <= nx;                         // row j0 - 1
    const bool cp_hi = ty == TY - 1 && i <= nx && j0 + TY <= ny;   // row j0 + TY
    const bool cp_xl = lane == 0 && j <= ny;                        // x = i0 - XE .. i0 - 1
    const bool cp_xr = lane == 31 && j <= ny && i0 + TX <= nx;      // x = i0 + TX ..
    const long long g_row = (long long)j * py + i;
    const int s_row = (ty + 1) * PW + HX + lane * VX;
    auto stage_p = [&](int q) { return reinterpret_cast<T*>(smem + (q % S) * Gm::STAGE_BYTES); };
    auto stage_r = [&](int q) { return stage_p(q) + Gm::PELEMS; };
    auto issue = [&](int q) {
      if (q < np) {
        const long long gz = (long long)(k0 - 1 + q) * pz;
        T* sp = stage_p(q);
        if (cp_row) cp_async_n<VB>(sp + s_row, P0 + gz + g_row);
        if (cp_lo) cp_async_n<VB>(sp + HX + lane * VX, P0 + gz + g_row - (long long)(ty + 1) * py);
        if (cp_hi) cp_async_n<VB>(sp + (TY + 1) * PW + HX + lane * VX, P0 + gz + g_row + py);
        if (cp_xl) cp_async_n<XB>(sp + (ty + 1) * PW + HX - XE, P0 + gz + (long long)j * py + i0 - XE);
        if (cp_xr) cp_async_n<XB>(sp + (ty + 1) * PW + HX + TX, P0 + gz + (long long)j * py + i0 + TX);
        if (cp_r && q >= 1 && q <= np - 2)
          cp_async_n<VB>(stage_r(q) + ty * TX + lane * VX, R0 + gz + g_row);
      }
      cp_commit();
    };
    for (int q = 0; q < S - 1; ++q) issue(q);
    T* qo = wptr<T>(L, B, dst) + (long long)k0 * pz + g_row;
    const bool out_row = j < ny && i < nx;
    const bool full_vec = i + VX <= nx;
    const bool face_xj = (i == 0) || (i <= nx - 1 && nx - 1 < i + VX) || j == 0 || j == ny - 1;
    for (int q = 1; q <= np - 2; ++q) {
      cp_wait<S - 4>();  // this thread's copies of plane q + 1 have landed
      __syncthreads();   // everyone's have; plane q - 2 is no longer read
      issue(q + S - 2);
      const T* Pm = stage_p(q - 1);
      const T* Pc = stage_p(q);
      const T* Pp = stage_p(q + 1);
      float c[VX], up[VX], dn[VX], zm[VX], zp[VX], rr[VX];
      ldv<VX>(Pc + s_row, c);
      ldv<VX>(Pc + s_row + PW, up);
      ldv<VX>(Pc + s_row - PW, dn);
      ldv<VX>(Pm + s_row, zm);
      ldv<VX>(Pp + s_row, zp);
      ldv<VX>(stage_r(q) + ty * TX + lane * VX, rr);
      const float left = tof(Pc[s_row - 1]), right = tof(Pc[s_row + VX]);
      float out[VX];
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        const float xm = e == 0 ? left : c[e - 1];
        const float xp = e == VX - 1 ? right : c[e + 1];
        out[e] = jacobi_update(c[e], xm, xp, dn[e], up[e], zm[e], zp[e], rr[e], cx, cy, cz,
                                 omega, inv_diag);
      }
      const int k = k0 + q - 1;
      if (out_row) {
        if (full_vec) {
          stv<T, VX>(qo, out);
        } else {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (i + e < nx) qo[e] = cvt<T>(out[e]);
        }
        if (face_xj || k == 0 || k == nz - 1) {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (i + e < nx) p_ghost_images<T>(L, B, dst, i + e, j, k, cvt<T>(out[e]));
        }
      }
      qo += pz;
    }
    cp_wait<0>();
    __syncthreads();  // the next tile refills the ring
  }
}

// Two fused Jacobi sweeps per pass (temporal blocking): p2 = J(J(p0, r), r).
// A CTA of TY + 4 warps owns a 128 x TY column of a single block and walks
// it along z.  Warp w loads row j0 - 2 + w of p0 (128 cells, 4 per lane, and
// two halo cells on each side) and, one plane ahead, of r; sweep 1 is
// evaluated on the (128 + 2) x (TY + 2) ring-extended tile, sweep 2 on the
// tile itself.  Cells beyond the domain are read through the boundary map
// (periodic wrap, or the mirror image for a zero-gradient wall), which makes
// the ring's sweep-1 values equal to their ghost images, so no ghost layer
// of the intermediate sweep is needed.  Shared memory: 3 planes of p0,
// 3 planes of p1, 2 planes of r; rows are 136 elements with the 128
// interior cells at 4..131 (16-byte aligned) and the halo at 2, 3, 132, 133.

__device__ __forceinline__ int map_coord(int x, int n, bool periodic) {
  if (x >= 0 && x < n) return x;
  if (periodic) return x < 0 ? x + n : x - n;
  return x < 0 ? -1 - x : 2 * n - 1 - x;
}

template <typename T, int TY>
__global__ void __launch_bounds__(32 * (TY + 4)) k_jacobi2(Launch L, int zc, int src, int dst,
                                                          int r_arr, float omega,
                                                          float inv_diag) {
  constexpr int TX = 128, RW = 136, NW = TY + 4;
  __shared__ __align__(16) float P0[3][NW][RW];
  __shared__ __align__(16) float P1[3][TY + 2][RW];
  __shared__ __align__(16) float RR[2][TY + 2][RW];
  __shared__ TileTable tt;
  tile_table_build(tt, L, TX, TY, zc);
  const int lane = threadIdx.x, w = threadIdx.y;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int py = B.py;
    const long long pz = B.pz;
    const bool perx = B.bc[0] == BC_PERIODIC, pery = B.bc[2] == BC_PERIODIC,
               perz = B.bc[4] == BC_PERIODIC;
    const T* P = reinterpret_cast<const T*>(L.base) + B.org[src];
    const T* R = reinterpret_cast<const T*>(L.base) + B.org[r_arr];
    T* Q = reinterpret_cast<T*>(L.base) + B.org[dst];
    const int k1 = min(k0 + zc, nz);
    const int x = i0 + lane * 4;
    // this warp's p0 row and (warps 1..TY+2) r row, mapped into the domain
    const int yrow = map_coord(j0 - 2 + w, ny, pery);
    const bool has_r = w >= 1 && w <= TY + 2;
    // halo columns of lanes 0 and 31, mapped
    const int xl2 = map_coord(i0 - 2, nx, perx), xl1 = map_coord(i0 - 1, nx, perx);
    const int xr1 = map_coord(i0 + TX, nx, perx), xr2 = map_coord(i0 + TX + 1, nx, perx);

    // register staging of one plane of p0 (and r) for this thread
    float sp[4], sr[4];
    float sh0 = 0.f, sh1 = 0.f, shr = 0.f;
    auto load_plane = [&](int z, bool want_r, int zr) {
      const long long ro = (long long)map_coord(z, nz, perz) * pz + (long long)yrow * py;
      ldv<4>(P + ro + x, sp);
      if (lane == 0) { sh0 = ldf<T>(P + ro + xl2); sh1 = ldf<T>(P + ro + xl1); }
      if (lane == 31) { sh0 = ldf<T>(P + ro + xr1); sh1 = ldf<T>(P + ro + xr2); }
      if (want_r && has_r) {
        const long long rro = (long long)map_coord(zr, nz, perz) * pz + (long long)yrow * py;
        ldv<4>(R + rro + x, sr);
        if (lane == 0) shr = ldf<T>(R + rro + xl1);
        if (lane == 31) shr = ldf<T>(R + rro + xr1);
      }
    };
    auto store_plane = [&](int z, bool want_r, int zr) {
      float* prow = &P0[((z % 3) + 3) % 3][w][0];
      *reinterpret_cast<float4*>(prow + 4 + lane * 4) = make_float4(sp[0], sp[1], sp[2], sp[3]);
      if (lane == 0) { prow[2] = sh0; prow[3] = sh1; }
      if (lane == 31) { prow[132] = sh0; prow[133] = sh1; }
      if (want_r && has_r) {
        float* rrow = &RR[((zr % 2) + 2) % 2][w - 1][0];
        *reinterpret_cast<float4*>(rrow + 4 + lane * 4) = make_float4(sr[0], sr[1], sr[2], sr[3]);
        if (lane == 0) rrow[3] = shr;
        if (lane == 31) rrow[132] = shr;
      }
    };
    // sweep 1 at plane z on rows 1..TY+2 (P1 row w - 1), from P0 planes z-1, z, z+1
    auto sweep1 = [&](int z) {
      if (!has_r) return;
      const float* pc = &P0[((z % 3) + 3) % 3][w][0];
      const float* pm = &P0[(((z - 1) % 3) + 3) % 3][w][0];
      const float* pp = &P0[(((z + 1) % 3) + 3) % 3][w][0];
      const float* rr = &RR[((z % 2) + 2) % 2][w - 1][0];
      float* out = &P1[((z % 3) + 3) % 3][w - 1][0];
      const int c0 = 4 + lane * 4;
      const float4 c4 = *reinterpret_cast<const float4*>(pc + c0);
      const float4 u4 = *reinterpret_cast<const float4*>(pc + c0 + RW);
      const float4 d4 = *reinterpret_cast<const float4*>(pc + c0 - RW);
      const float4 m4 = *reinterpret_cast<const float4*>(pm + c0);
      const float4 p4 = *reinterpret_cast<const float4*>(pp + c0);
      const float4 r4 = *reinterpret_cast<const float4*>(rr + c0);
      const float cc[4] = {c4.x, c4.y, c4.z, c4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w},
                  dd[4] = {d4.x, d4.y, d4.z, d4.w}, mm[4] = {m4.x, m4.y, m4.z, m4.w},
                  qq[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
      const float left = pc[c0 - 1], right = pc[c0 + 4];
      float o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float xm = e == 0 ? left : cc[e - 1];
        const float xp = e == 3 ? right : cc[e + 1];
        o[e] = jacobi_update(cc[e], xm, xp, dd[e], uu[e], mm[e], qq[e], rv[e], cx, cy, cz,
                                 omega, inv_diag);
      }
      *reinterpret_cast<float4*>(out + c0) = make_float4(o[0], o[1], o[2], o[3]);
      if (lane == 0 || lane == 31) {  // ring column x = i0 - 1 (index 3) or i0 + TX (132)
        const int c = lane == 0 ? 3 : 132;
        out[c] = jacobi_update(pc[c], pc[c - 1], pc[c + 1], pc[c - RW], pc[c + RW], pm[c], pp[c],
                               rr[c], cx, cy, cz, omega, inv_diag);
      }
    };

    // prologue: sweep 1 at planes k0 - 1 and k0
    load_plane(k0 - 2, false, 0);
    store_plane(k0 - 2, false, 0);
    load_plane(k0 - 1, true, k0 - 1);
    store_plane(k0 - 1, true, k0 - 1);
    load_plane(k0, true, k0);
    store_plane(k0, false, 0);
    const float srk[4] = {sr[0], sr[1], sr[2], sr[3]};
    const float shrk = shr;
    __syncthreads();
    sweep1(k0 - 1);
    __syncthreads();
    // r(k0) into its slot; p0(k0 + 1)
    for (int e = 0; e < 4; ++e) sr[e] = srk[e];
    shr = shrk;
    load_plane(k0 + 1, false, 0);
    store_plane(k0 + 1, false, 0);
    if (has_r) {
      float* rrow = &RR[((k0 % 2) + 2) % 2][w - 1][0];
      *reinterpret_cast<float4*>(rrow + 4 + lane * 4) = make_float4(sr[0], sr[1], sr[2], sr[3]);
      if (lane == 0) rrow[3] = shr;
      if (lane == 31) rrow[132] = shr;
    }
    __syncthreads();
    sweep1(k0);
    // prefetch p0(k0 + 2), r(k0 + 1) for the first iteration
    load_plane(k0 + 2, true, k0 + 1);

    const bool out_warp = w >= 2 && w <= TY + 1;
    const int j = j0 + w - 2;
    const bool face_xj = (x == 0) || (x + 4 == nx) || j == 0 || j == ny - 1;
    for (int m = k0; m < k1; ++m) {
      __syncthreads();  // previous p2 reads and sweep 1 of plane m are done
      store_plane(m + 2, true, m + 1);
      if (m + 1 < k1) load_plane(m + 3, true, m + 2);
      __syncthreads();
      sweep1(m + 1);
      __syncthreads();
      if (out_warp) {
        const float* qc = &P1[((m % 3) + 3) % 3][w - 1][0];
        const float* qm = &P1[(((m - 1) % 3) + 3) % 3][w - 1][0];
        const float* qp = &P1[(((m + 1) % 3) + 3) % 3][w - 1][0];
        const float* rr = &RR[((m % 2) + 2) % 2][w - 1][0];
        const int c0 = 4 + lane * 4;
        const float4 c4 = *reinterpret_cast<const float4*>(qc + c0);
        const float4 u4 = *reinterpret_cast<const float4*>(qc + c0 + RW);
        const float4 d4 = *reinterpret_cast<const float4*>(qc + c0 - RW);
        const float4 m4 = *reinterpret_cast<const float4*>(qm + c0);
        const float4 p4 = *reinterpret_cast<const float4*>(qp + c0);
        const float4 r4 = *reinterpret_cast<const float4*>(rr + c0);
        const float cc[4] = {c4.x, c4.y, c4.z, c4.w}, uu[4] = {u4.x, u4.y, u4.z, u4.w},
                    dd[4] = {d4.x, d4.y, d4.z, d4.w}, mm[4] = {m4.x, m4.y, m4.z, m4.w},
                    qq[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
        const float left = qc[c0 - 1], right = qc[c0 + 4];
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float xm = e == 0 ? left : cc[e - 1];
          const float xp = e == 3 ? right : cc[e + 1];
          o[e] = jacobi_update(cc[e], xm, xp, dd[e], uu[e], mm[e], qq[e], rv[e], cx, cy, cz,
                                   omega, inv_diag);
        }
        T* qo = Q + (long long)m * pz + (long long)j * py + x;
        stv<T, 4>(qo, o);
        if (face_xj || m == 0 || m == nz - 1) {
#pragma unroll
          for (int e = 0; e < 4; ++e) p_ghost_images<T>(L, B, dst, x + e, j, m, cvt<T>(o[e]));
        }
      }
    }
    __syncthreads();  // the next tile reuses the buffers
  }
}

// Direct sweep: one thread per VX consecutive cells of one row, every
// neighbour loaded straight from global memory (x neighbours by shuffle).
// No shared memory and no barrier: each CTA (32 x TY x TZ threads) covers a
// (32 VX) x TY x TZ tile and all its loads are independent, so the memory
// system sees as many requests in flight as an elementwise kernel; the
// y and z neighbours are served by L1/L2 (neighbouring rows and planes are
// read by the same or nearby CTAs).

template <typename T, int VX, int TY, int TZ>
__global__ void __launch_bounds__(32 * TY * TZ) k_jacobi_direct(Launch L, int src, int dst,
                                                               int r_arr, float omega,
                                                               float inv_diag) {
  constexpr int TX = 32 * VX;
  const int lane = threadIdx.x;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  __shared__ TileTable tt;
  tile_table_build(tt, L, TX, TY, TZ);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, TZ, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int j = j0 + threadIdx.y, k = k0 + threadIdx.z;
    if (j >= ny || k >= nz) continue;  // uniform per warp: a warp is one row
    const int py = B.py;
    const long long pz = B.pz;
    const T* P = reinterpret_cast<const T*>(L.base) + B.org[src];
    const T* R = reinterpret_cast<const T*>(L.base) + B.org[r_arr];
    const int i = i0 + lane * VX;
    const long long rowo = (long long)k * pz + (long long)j * py;
    const long long o = rowo + i;
    float c[VX], ym[VX], yp[VX], zm[VX], zp[VX], rr[VX];
#pragma unroll
    for (int e = 0; e < VX; ++e) c[e] = ym[e] = yp[e] = zm[e] = zp[e] = rr[e] = 0.f;
    if (i <= nx) {  // columns up to nx (first ghost) stay inside the row
      ldv<VX>(P + o, c);
      ldv<VX>(P + o - py, ym);
      ldv<VX>(P + o + py, yp);
      ldv<VX>(P + o - pz, zm);
      ldv<VX>(P + o + pz, zp);
      ldv<VX>(R + o, rr);
    }
    float left = __shfl_up_sync(0xffffffffu, c[VX - 1], 1);
    float right = __shfl_down_sync(0xffffffffu, c[0], 1);
    if (lane == 0) left = ldf<T>(P + rowo + i0 - 1);
    if (lane == 31) right = (i0 + TX <= nx) ? ldf<T>(P + rowo + i0 + TX) : 0.f;
    if (i >= nx) continue;
    float out[VX];
#pragma unroll
    for (int e = 0; e < VX; ++e) {
      const float xm = e == 0 ? left : c[e - 1];
      const float xp = e == VX - 1 ? right : c[e + 1];
      out[e] = jacobi_update(c[e], xm, xp, ym[e], yp[e], zm[e], zp[e], rr[e], cx, cy, cz,
                               omega, inv_diag);
    }
    T* qrow = wptr<T>(L, B, dst) + o;
    if (i + VX <= nx) {
      stv<T, VX>(qrow, out);
    } else {
#pragma unroll
      for (int e = 0; e < VX; ++e)
        if (i + e < nx) qrow[e] = cvt<T>(out[e]);
    }
    const bool face = (i == 0) || (nx - 1 < i + VX) || j == 0 || j == ny - 1 || k == 0 ||
                      k == nz - 1;
    if (face) {
#pragma unroll
      for (int e = 0; e < VX; ++e)
        if (i + e < nx) p_ghost_images<T>(L, B, dst, i + e, j, k, cvt<T>(out[e]));
    }
  }
}

// ---------------------------------------------------- compact <-> padded

// One warp per interior row: the compact buffer holds rows of nx elements
// back to back, the array rows start 128-byte aligned at x = 0.  When the
// compact buffer starts 16-byte aligned and nx is a multiple of the vector
// width (so every compact row starts aligned) rows move as 16-byte vectors;
// otherwise element by element.
template <typename T>
__global__ void __launch_bounds__(256) k_pack(Launch L, int arr, T* compact, int to_compact) {
  constexpr int V = 16 / (int)sizeof(T);
  const BlockDev& B = L.blocks[L.b0];
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const int py = B.py;
  const long long pz = B.pz;
  T* a = reinterpret_cast<T*>(L.base) + B.org[arr];
  const long long rows = (long long)ny * nz;
  const int lane = threadIdx.x & 31;
  const bool vec = (nx % V) == 0 && (reinterpret_cast<uintptr_t>(compact) % 16) == 0;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int j = (int)(r % ny), k = (int)(r / ny);
    T* ar = a + (long long)k * pz + (long long)j * py;
    T* cr = compact + r * nx;
    if (vec) {
      uint4* av = reinterpret_cast<uint4*>(ar);
      uint4* cv = reinterpret_cast<uint4*>(cr);
      for (int i = lane; i < nx / V; i += 32) {
        if (to_compact) cv[i] = av[i];
        else av[i] = cv[i];
      }
    } else {
      for (int i = lane; i < nx; i += 32) {
        if (to_compact) cr[i] = ar[i];
        else ar[i] = cr[i];
      }
    }
  }
}

// The pack copy on a few CTAs: thread t of T moves 16-byte vectors
// t + u T of each batch (u < 16), all sixteen loads before the stores, so
// every thread keeps sixteen transfers over the host link in flight;
// consecutive threads take consecutive vectors of a row.
template <typename T>
__global__ void __launch_bounds__(256) k_pack_narrow(Launch L, int arr, T* compact, int to_compact) {
  constexpr int V = 16 / (int)sizeof(T), U = 16;
  const BlockDev& B = L.blocks[L.b0];
  const int nx = B.n[0], ny = B.n[1];
  const long long vpr = nx / V;                                 // vectors per row
  const long long total = vpr * ny * B.n[2];
  const long long py = B.py, pz = B.pz;
  T* a = reinterpret_cast<T*>(L.base) + B.org[arr];
  uint4* cv = reinterpret_cast<uint4*>(compact);
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  auto at = [&](long long k) {  // vector k of the compact order -> the array
    const long long r = k / vpr, v = k - r * vpr;
    const long long j = r % ny, kz = r / ny;
    return reinterpret_cast<uint4*>(a + kz * pz + j * py) + v;
  };
  for (long long base = tid; base < total; base += U * nthr) {
    uint4 x[U];
    if (to_compact) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * nthr < total) x[u] = *at(base + u * nthr);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * nthr < total) cv[base + u * nthr] = x[u];
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * nthr < total) x[u] = cv[base + u * nthr];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * nthr < total) *at(base + u * nthr) = x[u];
    }
  }
}

// --------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reduction of 4 values (sum, max, max, sum) in a fixed tree.
template <int NT>
__device__ __forceinline__ void block_reduce4(double (&v)[4], double (*sh)[4]) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int w = tid >> 5, ln = tid & 31;
  v[0] = warp_sum(v[0]);
  v[1] = warp_max(v[1]);
  v[2] = warp_max(v[2]);
  v[3] = warp_sum(v[3]);
  if (ln == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) sh[w][e] = v[e];
  }
  __syncthreads();
  if (w == 0) {
    constexpr int NW = NT / 32;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    if (ln < NW) {
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = sh[ln][e];
    }
    a[0] = warp_sum(a[0]);
    a[1] = warp_max(a[1]);
    a[2] = warp_max(a[2]);
    a[3] = warp_sum(a[3]);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = a[e];
  }
}

// The column loops are unrolled four deep so that several cells' loads are
// in flight per thread (each thread walks zc cells of one column).
// mode 0: sum |u|^2, max |u_d|, max |D u| and the non-finite count of a
// velocity set; the per-cell work is float-float, each thread's column sum
// (at most zc cells) is added to an FP64 accumulator.  mode 1: sum of
// (L p - r)^2, the residual per cell in float-float, its square in
// float-float, the same column sums.  mode 2: sum of r^2, likewise.
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) k_reduce(Launch L, int zc, int mode, Set3 set,
                                                    int p_arr, int r_arr, double* partials) {
  __shared__ double sh[TY][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, TY, zc);
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const T* base = reinterpret_cast<const T*>(L.base);
  float umax = 0.f;
  FF dmax = {0.f, 0.f};
  int bad = 0;
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const int py = B.py;
    const long long pz = B.pz;
    const int kn = min(k0 + zc, B.n[2]) - k0;
    const long long o0 = (long long)k0 * pz + (long long)j * py + i;
    if (mode == 0) {
      const T* X[3] = {base + B.org[set.a[0]] + o0, base + B.org[set.a[1]] + o0,
                       base + B.org[set.a[2]] + o0};
      const long long back[3] = {1, py, pz};
      FF col = {0.f, 0.f};
#pragma unroll 4
      for (int q = 0; q < kn; ++q) {
        const long long o = (long long)q * pz;
        float x[3], xm[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          x[c] = ldf<T>(X[c] + o);
          xm[c] = ldf<T>(X[c] + o - back[c]);
          umax = fmaxf(umax, fabsf(x[c]));
          bad += !isfinite(x[c]);
        }
        FF div;
        ff_cell(x, xm, ih, col, div);
        div = ff_abs(div);
        if (ff_gt(div, dmax)) dmax = div;
      }
      acc[0] += ff_to_double(col);
    } else if (mode == 1) {
      // e = L p - r per cell in float-float (the sums and differences of
      // the FP32 values exact, the products by 1/h^2 with their rounding
      // error kept), e^2 in float-float summed over the column, each
      // column's sum added to an FP64 accumulator (FP64 issues at a small
      // fraction of the FP32 rate here, so it is kept out of the per-cell
      // work); cells whose square would leave the FP32 range go to FP64
      FF col = {0.f, 0.f};
      double big = 0.0;
      const T* P = base + B.org[p_arr] + o0;
      const T* Rr = base + B.org[r_arr] + o0;
      const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
      const long long step[3] = {1, py, pz};
#pragma unroll 4
      for (int q = 0; q < kn; ++q) {
        const long long o = (long long)q * pz;
        const float pc = ldf<T>(P + o);
        FF lp = {0.f, 0.f};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const FF nbs = ff_two_sum(ldf<T>(P + o + step[d]), ldf<T>(P + o - step[d]));
          const FF sec = ff_add(nbs, FF{-2.f * pc, 0.f});  // 2 pc is exact
          FF t = ff_two_prod(sec.hi, ih2[d]);
          t.lo = __fmaf_rn(sec.lo, ih2[d], t.lo);
          lp = d == 0 ? ff_fast_two_sum(t.hi, t.lo) : ff_add(lp, t);
        }
        const FF e = ff_add(lp, FF{-ldf<T>(Rr + o), 0.f});
        col = ff_add(col, ff_square(e));
        if (fabsf(e.hi) >= kFFSquareMax) big += (double)e.hi * e.hi;
        bad += !isfinite(e.hi);
      }
      acc[0] += ff_to_double(col) + big;
    } else {
      // sum of r^2 (the norm the converged solve measures against), the
      // same float-float column sums
      FF col = {0.f, 0.f};
      double big = 0.0;
      const T* Rr = base + B.org[r_arr] + o0;
#pragma unroll 4
      for (int q = 0; q < kn; ++q) {
        const float rv = ldf<T>(Rr + (long long)q * pz);
        col = ff_add(col, ff_square(FF{rv, 0.f}));
        if (fabsf(rv) >= kFFSquareMax) big += (double)rv * rv;
        bad += !isfinite(rv);
      }
      acc[0] += ff_to_double(col) + big;
    }
  }
  if (mode == 0) {
    acc[1] = umax;
    acc[2] = ff_to_double(dmax);
  }
  acc[3] = bad;
  block_reduce4<32 * TY>(acc, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) partials[4 * blockIdx.x + e] = acc[e];
  }
}

__global__ void __launch_bounds__(256) k_reduce_final(const double* partials, int nparts,
                                                      double* out) {
  __shared__ double sh[8][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = threadIdx.x; p < nparts; p += 256) {
    acc[0] += partials[4 * p];
    acc[1] = fmax(acc[1], partials[4 * p + 1]);
    acc[2] = fmax(acc[2], partials[4 * p + 2]);
    acc[3] += partials[4 * p + 3];
  }
  block_reduce4<256>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = acc[e];
  }
}

// ------------------------------------------------------------------ helpers

template <typename K>
int occupancy(K kernel, int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

unsigned grid_for(const Launch& L, int occ, long long tiles) {
  const long long cap = (long long)L.sms * occ;
  long long gsz = tiles < cap ? tiles : cap;
  return (unsigned)(gsz > 0 ? gsz : 1);
}

Set3 mk3(const int* s) { return Set3{{s[0], s[1], s[2]}}; }

}  // namespace

long long count_tiles(const Launch& L, int tx, int ty, int tz) {
  long long n = 0;
  for (int b = L.b0; b < L.b0 + L.nblocks; ++b) {
    const int* d = L.hn[b];
    n += (long long)((d[0] + tx - 1) / tx) * ((d[1] + ty - 1) / ty) * ((d[2] + tz - 1) / tz);
  }
  return n;
}

#define CFD_DISPATCH_T(dtype, ...)                         \
  switch (dtype) {                                         \
    case 0: { using T = float; __VA_ARGS__; } break;       \
    case 1: { using T = __nv_bfloat16; __VA_ARGS__; } break; \
    default: { using T = __half; __VA_ARGS__; } break;     \
  }

cudaError_t launch_ghost(const Launch& L, const int* arrays, int narr, const GhostItem* items,
                         int nitems) {
  if (nitems == 0 || narr == 0) return cudaSuccess;
  GhostArrays ga{};
  ga.n = narr;
  for (int e = 0; e < narr; ++e) ga.arr[e] = arrays[e];
  const unsigned ctas = (unsigned)((nitems + kGhostWarps - 1) / kGhostWarps);
  if (narr == 1) {
    CFD_DISPATCH_T(L.dtype,
                   k_ghost<T, 1><<<ctas, 32 * kGhostWarps, 0, L.stream>>>(L, items, nitems, ga));
  } else if (narr == 2) {
    CFD_DISPATCH_T(L.dtype,
                   k_ghost<T, 2><<<ctas, 32 * kGhostWarps, 0, L.stream>>>(L, items, nitems, ga));
  } else {
    CFD_DISPATCH_T(L.dtype,
                   k_ghost<T, 4><<<ctas, 32 * kGhostWarps, 0, L.stream>>>(L, items, nitems, ga));
  }
  return cudaGetLastError();
}

template <typename T, int SCH, int TZ>
static void run_stage_tile(const Launch& L, float a, Set3 xs, float b, Set3 ys, float cdt, Set3 os,
                           float nu) {
  const long long tiles = count_tiles(L, 32, 8, TZ);
  auto kern = k_stage_tile<T, SCH, TZ>;
  static const int occ = occupancy(kern, 256);
  kern<<<grid_for(L, occ, tiles), 256, 0, L.stream>>>(L, a, xs, b, ys, cdt, os, nu);
}

template <typename T, int SCH, int TY>
static void run_stage(const Launch& L, int zc, float a, Set3 xs, float b, Set3 ys, float cdt,
                      Set3 os, float nu) {
  const long long tiles = count_tiles(L, 32, TY, zc);
  auto kern = k_stage<T, SCH, TY>;
  static const int occ = occupancy(kern, 32 * TY);
  kern<<<grid_for(L, occ, tiles), dim3(32, TY), 0, L.stream>>>(L, zc, a, xs, b, ys, cdt, os, nu);
}

template <typename T, int SCH, int TY>
static void run_stage_ring(const Launch& L, int zc, float a, Set3 xs, float b, Set3 ys, float cdt,
                           Set3 os, float nu) {
  const long long tiles = count_tiles(L, 32, TY, zc);
  if constexpr (sizeof(T) == 4) {
    auto kern = k_stage_async<SCH, TY>;
    static const int occ = occupancy(kern, 32 * TY);
    kern<<<grid_for(L, occ, tiles), dim3(32, TY), 0, L.stream>>>(L, zc, a, xs, b, ys, cdt, os, nu);
  } else {
    auto kern = k_stage_ring<T, SCH, TY>;
    static const int occ = occupancy(kern, 32 * TY);
    kern<<<grid_for(L, occ, tiles), dim3(32, TY), 0, L.stream>>>(L, zc, a, xs, b, ys, cdt, os, nu);
  }
}

template <int SCH>
static cudaError_t launch_stage_s(const Launch& L, const StencilCfg& c, float a, Set3 xs, float b,
                                  Set3 ys, float cdt, Set3 os, float nu) {
  if constexpr (SCH != kSchemeAdv4) {
    if (c.tile_tz == 3 && L.dtype == 0) {
      const long long tiles = count_tiles(L, 64, 4, c.zc);
      auto kern = k_stage_pair<SCH, 4>;
      static const int occ = occupancy(kern, 128);
      kern<<<grid_for(L, occ, tiles), dim3(32, 4), 0, L.stream>>>(L, c.zc, a, xs, b, ys, cdt, os, nu);
      return cudaGetLastError();
    }
  }
  CFD_DISPATCH_T(L.dtype, {
    if (c.tile_tz == 1 || c.tile_tz == 3) {
      if (c.ty == 4) run_stage_ring<T, SCH, 4>(L, c.zc, a, xs, b, ys, cdt, os, nu);
      else run_stage_ring<T, SCH, 8>(L, c.zc, a, xs, b, ys, cdt, os, nu);
    } else if (c.tile_tz == 2) {
      run_stage_tile<T, SCH, 2>(L, a, xs, b, ys, cdt, os, nu);
    } else if (c.tile_tz == 4) {
      run_stage_tile<T, SCH, 4>(L, a, xs, b, ys, cdt, os, nu);
    } else {
      if (c.ty == 4) run_stage<T, SCH, 4>(L, c.zc, a, xs, b, ys, cdt, os, nu);
      else run_stage<T, SCH, 8>(L, c.zc, a, xs, b, ys, cdt, os, nu);
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_stage(const Launch& L, const StencilCfg& c, int scheme, float a,
                         const int* xset, float b, const int* yset, float cdt, const int* oset,
                         float nu) {
  const Set3 xs = xset ? mk3(xset) : Set3{{0, 0, 0}};
  const Set3 ys = mk3(yset), os = mk3(oset);
  switch (scheme) {
    case kSchemeAdv2: return launch_stage_s<kSchemeAdv2>(L, c, a, xs, b, ys, cdt, os, nu);
    case kSchemeAdv4: return launch_stage_s<kSchemeAdv4>(L, c, a, xs, b, ys, cdt, os, nu);
    case kSchemeFlux2: return launch_stage_s<kSchemeFlux2>(L, c, a, xs, b, ys, cdt, os, nu);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_divergence(const Launch& L, const StencilCfg& c, const int* wset,
                              float inv_cdt, int r_arr) {
  const long long tiles = count_tiles(L, 32, 8, c.zc);
  CFD_DISPATCH_T(L.dtype, {
    auto kern = k_div<T, 8>;
    static const int occ = occupancy(kern, 256);
    kern<<<grid_for(L, occ, tiles), dim3(32, 8), 0, L.stream>>>(L, c.zc, mk3(wset), inv_cdt, r_arr);
  });
  return cudaGetLastError();
}

cudaError_t launch_project(const Launch& L, const StencilCfg& c, const int* wset, int p_arr,
                           float cdt, const int* oset) {
  const long long tiles = count_tiles(L, 32, 8, c.zc);
  CFD_DISPATCH_T(L.dtype, {
    auto kern = k_project<T, 8>;
    static const int occ = occupancy(kern, 256);
    kern<<<grid_for(L, occ, tiles), dim3(32, 8), 0, L.stream>>>(L, c.zc, mk3(wset), p_arr, cdt, mk3(oset));
  });
  return cudaGetLastError();
}

cudaError_t launch_pack(const Launch& L, int arr, void* compact, int to_compact) {
  CFD_DISPATCH_T(L.dtype, {
    auto kern = k_pack<T>;
    static const int occ = occupancy(kern, 256);
    kern<<<(unsigned)(L.sms * occ), 256, 0, L.stream>>>(L, arr, static_cast<T*>(compact),
                                                       to_compact);
  });
  return cudaGetLastError();
}

cudaError_t launch_pack_narrow(const Launch& L, int arr, void* compact, int to_compact) {
  const int es = L.dtype == 0 ? 4 : 2;
  if (L.hn[L.b0][0] % (16 / es) != 0 || reinterpret_cast<uintptr_t>(compact) % 16 != 0)
    return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)std::max(1, L.sms / 8);
  CFD_DISPATCH_T(L.dtype, k_pack_narrow<T><<<grid, 256, 0, L.stream>>>(L, arr, static_cast<T*>(compact),
                                                                        to_compact));
  return cudaGetLastError();
}

cudaError_t launch_copy(const Launch& L, const StencilCfg&, int src, int dst) {
  CFD_DISPATCH_T(L.dtype, {
    auto kern = k_copy<T>;
    static const int occ = occupancy(kern, 256);
    kern<<<(unsigned)(L.sms * occ), 256, 0, L.stream>>>(L, src, dst);
  });
  return cudaGetLastError();
}

template <typename T, int VX, int TY>
static void run_jacobi(const Launch& L, int zc, int src, int dst, int r_arr, float omega,
                       float inv_diag) {
  const long long tiles = count_tiles(L, 32 * VX, TY, zc);
  auto kern = k_jacobi<T, VX, TY>;
  static const int occ = occupancy(kern, 32 * TY);
  kern<<<grid_for(L, occ, tiles), dim3(32, TY), 0, L.stream>>>(L, zc, src, dst, r_arr, omega, inv_diag);
}

cudaError_t launch_jacobi(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                          float omega) {
  const float diag = 2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]);
  const float inv_diag = 1.f / diag;
  CFD_DISPATCH_T(L.dtype, {
    if (c.vx == 4) {
      if (c.ty == 4) run_jacobi<T, 4, 4>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else if (c.ty == 16) run_jacobi<T, 4, 16>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else run_jacobi<T, 4, 8>(L, c.zc, src, dst, r_arr, omega, inv_diag);
    } else if (c.vx == 2) {
      if (c.ty == 4) run_jacobi<T, 2, 4>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else run_jacobi<T, 2, 8>(L, c.zc, src, dst, r_arr, omega, inv_diag);
    } else {
      if (c.ty == 4) run_jacobi<T, 1, 4>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else run_jacobi<T, 1, 8>(L, c.zc, src, dst, r_arr, omega, inv_diag);
    }
  });
  return cudaGetLastError();
}

template <typename T, int TY>
static void run_jacobi2(const Launch& L, int zc, int src, int dst, int r_arr, float omega,
                        float inv_diag) {
  const long long tiles = count_tiles(L, 128, TY, zc);
  auto kern = k_jacobi2<T, TY>;
  static const int occ = occupancy(kern, 32 * (TY + 4));
  kern<<<grid_for(L, occ, tiles), dim3(32, TY + 4), 0, L.stream>>>(L, zc, src, dst, r_arr, omega,
                                                                    inv_diag);
}

cudaError_t launch_jacobi2(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                           float omega) {
  const float inv_diag = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  CFD_DISPATCH_T(L.dtype, {
    if (c.ty == 8) run_jacobi2<T, 8>(L, c.zc, src, dst, r_arr, omega, inv_diag);
    else run_jacobi2<T, 4>(L, c.zc, src, dst, r_arr, omega, inv_diag);
  });
  return cudaGetLastError();
}

template <typename T, int VX, int TY, int S>
static cudaError_t run_jacobi_async(const Launch& L, int zc, int src, int dst, int r_arr,
                                    float omega, float inv_diag) {
  using Gm = AsyncGeom<T, VX, TY, S>;
  auto kern = k_jacobi_async<T, VX, TY, S>;
  static int occ = -1;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
    if (e != cudaSuccess) return e;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * TY, Gm::SMEM) != cudaSuccess ||
        occ < 1)
      occ = 1;
  }
  const long long tiles = count_tiles(L, Gm::TX, TY, zc);
  kern<<<grid_for(L, occ, tiles), dim3(32, TY), Gm::SMEM, L.stream>>>(L, zc, src, dst, r_arr, omega,
                                                                       inv_diag);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_async(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                                float omega) {
  const float inv_diag = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  cudaError_t e = cudaErrorInvalidValue;
  switch (L.dtype) {
    case 0: {
      using T = float;
      if (c.ty == 4 && c.stages == 5) e = run_jacobi_async<T, 4, 4, 5>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else if (c.ty == 4 && c.stages == 6) e = run_jacobi_async<T, 4, 4, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else if (c.ty == 8 && c.stages == 5) e = run_jacobi_async<T, 4, 8, 5>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else if (c.ty == 8) e = run_jacobi_async<T, 4, 8, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      else e = run_jacobi_async<T, 4, 2, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
    } break;
    default: {
      // 16-bit storage: 8 cells per thread keeps the copies at 16 bytes
      auto go = [&](auto tag) {
        using T = decltype(tag);
        if (c.ty == 4 && c.stages == 5) return run_jacobi_async<T, 8, 4, 5>(L, c.zc, src, dst, r_arr, omega, inv_diag);
        if (c.ty == 4 && c.stages == 6) return run_jacobi_async<T, 8, 4, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
        if (c.ty == 8 && c.stages == 5) return run_jacobi_async<T, 8, 8, 5>(L, c.zc, src, dst, r_arr, omega, inv_diag);
        if (c.ty == 8) return run_jacobi_async<T, 8, 8, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
        return run_jacobi_async<T, 8, 2, 6>(L, c.zc, src, dst, r_arr, omega, inv_diag);
      };
      e = L.dtype == 1 ? go(__nv_bfloat16()) : go(__half());
    } break;
  }
  return e;
}

template <typename T, int VX, int TY, int TZ>
static void run_jacobi_direct(const Launch& L, int src, int dst, int r_arr, float omega,
                              float inv_diag) {
  const long long tiles = count_tiles(L, 32 * VX, TY, TZ);
  auto kern = k_jacobi_direct<T, VX, TY, TZ>;
  static const int occ = occupancy(kern, 32 * TY * TZ);
  // enough CTAs for several waves; each walks tiles with a grid stride
  const long long cap = (long long)L.sms * occ * 16;
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  kern<<<grid > 0 ? grid : 1, dim3(32, TY, TZ), 0, L.stream>>>(L, src, dst, r_arr, omega, inv_diag);
}

cudaError_t launch_jacobi_direct(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                                 float omega) {
  const float inv_diag = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  CFD_DISPATCH_T(L.dtype, {
    if (c.vx == 4 && c.ty == 4 && c.zc == 2) run_jacobi_direct<T, 4, 4, 2>(L, src, dst, r_arr, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 8 && c.zc == 1) run_jacobi_direct<T, 4, 8, 1>(L, src, dst, r_arr, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 2 && c.zc == 4) run_jacobi_direct<T, 4, 2, 4>(L, src, dst, r_arr, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 4 && c.zc == 4) run_jacobi_direct<T, 4, 4, 4>(L, src, dst, r_arr, omega, inv_diag);
    else if (c.vx == 2 && c.ty == 4 && c.zc == 2) run_jacobi_direct<T, 2, 4, 2>(L, src, dst, r_arr, omega, inv_diag);
    else if (c.vx == 1 && c.ty == 8 && c.zc == 1) run_jacobi_direct<T, 1, 8, 1>(L, src, dst, r_arr, omega, inv_diag);
    else run_jacobi_direct<T, 4, 4, 1>(L, src, dst, r_arr, omega, inv_diag);
  });
  return cudaGetLastError();
}

cudaError_t launch_reduce(const Launch& L, int mode, const int* set, int p_arr, int r_arr,
                          double* partials, int nparts, double* out) {
  const int zc = 16;
  const long long tiles = count_tiles(L, 32, 8, zc);
  const unsigned grid = (unsigned)(tiles < nparts ? tiles : nparts);
  const Set3 s = set ? mk3(set) : Set3{{0, 0, 0}};
  CFD_DISPATCH_T(L.dtype, {
    k_reduce<T, 8><<<grid, dim3(32, 8), 0, L.stream>>>(L, zc, mode, s, p_arr, r_arr, partials);
  });
  k_reduce_final<<<1, 256, 0, L.stream>>>(partials, (int)grid, out);
  return cudaGetLastError();
}

}  // namespace cfd
