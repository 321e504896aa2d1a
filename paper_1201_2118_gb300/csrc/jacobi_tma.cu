// Weighted Jacobi sweep of the 7-point pressure operator with TMA staging.
//
// Same arithmetic as the register/shuffle sweep: p' = p + w((N p - r)/diag - p).
// A CTA owns a TX x TY column of one block and walks it along z.  One thread
// issues cp.async.bulk.tensor loads of each z-plane of p (with a one-cell
// halo in y and a 16-byte-aligned halo in x) and of r into a ring of S
// shared-memory stages completed through mbarriers; S - 2 planes are in
// flight while a plane is computed, with no registers held for them.  Each
// thread owns VX consecutive x cells of one row: it keeps their z-1 and z
// values in registers, reads z+1, the y neighbours and r from shared memory as
// VX-wide vectors, and takes the x neighbours from the adjacent lanes by warp
// shuffle (the row-end lanes read the halo column).  The output is written with
// plain coalesced stores plus the ghost-on-write images of face cells.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on a timeout the CTA
// sets the grid's device error flag, waits (bounded) for its own loads still
// in flight and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "cfd_internal.h"
#include "dev_common.cuh"
#include "tiles.cuh"
#include "tma_ptx.cuh"

namespace cfd {
namespace {

// A wait that nothing completes: one thread initialises an mbarrier that
// expects one arrival, never arrives, and waits for its first phase through
// the bounded wait of the TMA-staged kernels (form 0: mbar_wait, form 1:
// mbar_wait_split, the form with the polling loop out of line).  When the
// limit runs out it sets bit 2 of the device error flag, as those kernels do
// on a timeout, and returns; it has no copies in flight and holds no other
// resource.
__global__ void __launch_bounds__(32) k_wait_probe(int* err_flag, int form) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  mbar_fence_init();
  const bool ok = form == 0 ? mbar_wait(b, 0u) : mbar_wait_split(b, 0u);
  if (!ok) atomicOr(err_flag, 2);
}

template <typename T, int VX, int TY>
struct TmaGeom {
  static constexpr int TX = 32 * VX;
  static constexpr int HX = 16 / (int)sizeof(T);
  static constexpr int PW = TX + 2 * HX;
  static constexpr int PH = TY + 2;
  static constexpr int PBYTES = PW * PH * (int)sizeof(T);
  static constexpr int RBYTES = TX * TY * (int)sizeof(T);
  static constexpr int PSTRIDE = (PBYTES + 127) / 128 * 128;
  static constexpr int RSTRIDE = (RBYTES + 127) / 128 * 128;
  static constexpr int STAGE = PSTRIDE + RSTRIDE;
};

template <typename T, int VX, int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_jacobi_tma(Launch L, const CUtensorMap* maps, int zc,
                                                        int src_slot, int dst, float omega,
                                                        float inv_diag) {
  using Gm = TmaGeom<T, VX, TY>;
  constexpr int TX = Gm::TX, HX = Gm::HX, PW = Gm::PW;
  extern __shared__ __align__(128) unsigned char smem[];
  // S stages of (p box, r box), then the S mbarriers
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + S * Gm::STAGE);
  __shared__ RowImage<T> rimg[TY][4];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  if (smem_u32(smem) & 127u) {  // TMA destinations need 128-byte alignment
    if (tid == 0) atomicOr(L.err_flag, 4);
    return;
  }
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) mbar_init(smem_u32(&full[s]), 1);
    mbar_fence_init();
  }
  __syncthreads();
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  const Jac2 J2(cx, cy, cz, omega, inv_diag);
  const int g = L.ghost;
  constexpr int xo = kAlignBytes / (int)sizeof(T);
  uint32_t parity = 0;
  int sbase = 0;
  __shared__ TileTable tt;
  __shared__ int flag0;
  flag_at_start(L, flag0);
  tile_table_build(tt, L, TX, TY, zc);
  if (flag0) return;
  int blk = L.b0;
  // tiles claimed at run time from the counter in the grid's flag area:
  // thread 0 claims, the CTA barrier hands the number out (two slots: a
  // slot is rewritten two tiles later, after the planes' barriers between)
  __shared__ unsigned tile_no[2];
  unsigned* const ctr = tile_counter(L);
  const unsigned ctr_wrap = (unsigned)tt.start[L.nblocks] + gridDim.x - 1;
  for (unsigned kq = 0;; ++kq) {
    if (tid == 0) tile_no[kq & 1] = atomicInc(ctr, ctr_wrap);
    __syncthreads();
    const long long t = tile_no[kq & 1];
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int k1 = min(k0 + zc, nz);
    const int np = k1 - k0 + 2;  // planes k0-1 .. k1
    const CUtensorMap* mp = maps + 3 * blk + src_slot;
    const CUtensorMap* mr = maps + 3 * blk + 2;
    const int px = xo + i0 - HX, pyc = g + j0 - 1, rx = xo + i0, ry = g + j0;
    int next_q = 0;
    auto issue = [&](int q) {
      const int s = (sbase + q) % S;
      const int z = g + k0 - 1 + q;
      const bool need_r = (q >= 1 && q <= np - 2);
      const uint32_t bar = smem_u32(&full[s]);
      mbar_expect_tx(bar, Gm::PBYTES + (need_r ? Gm::RBYTES : 0));
      tma_load_3d(smem_u32(smem + s * Gm::STAGE), mp, px, pyc, z, bar);
      if (need_r) tma_load_3d(smem_u32(smem + s * Gm::STAGE + Gm::PSTRIDE), mr, rx, ry, z, bar);
    };
    const int first = np < S ? np : S;
    if (tid == 0)
      for (int q = 0; q < first; ++q) issue(q);
    next_q = first;
    int waited = 0;  // planes 0..waited-1 have completed
    bool bad = false;
    auto wait_plane = [&](int q) {
      const int s = (sbase + q) % S;
      bad |= !mbar_wait(smem_u32(&full[s]), (parity >> s) & 1u);
      parity ^= 1u << s;
      waited = q + 1;
    };
    wait_plane(0);
    wait_plane(1);
    const int j = j0 + ty;
    const int xl = lane * VX;                 // first tile-local x of this thread
    const int row = (ty + 1) * PW + HX + xl;  // its centre in a p box (VX-aligned)
    float m[VX], c[VX];
    {
      const T* P0 = reinterpret_cast<const T*>(smem + ((sbase + 0) % S) * Gm::STAGE);
      const T* P1 = reinterpret_cast<const T*>(smem + ((sbase + 1) % S) * Gm::STAGE);
      ldv<VX>(P0 + row, m);
      ldv<VX>(P1 + row, c);
    }
    // block fields in registers: the output stores may alias the block table
    // as far as the compiler knows, which would force a reload per plane
    const long long pzl = B.pz;
    const int pyl = B.py;
    T* Q = reinterpret_cast<T*>(L.base) + B.org[dst];
    const int x0 = i0 + xl;
    const bool full_vec = x0 + VX <= nx;
    const bool row_ok = j < ny && x0 < nx;
    __syncwarp();
    unsigned rm = 0;
    if (lane == 0) rm = row_images<T>(L, B, dst, i0, TX, j, rimg[ty]);
    const unsigned tm = thread_images<VX>(__shfl_sync(0xffffffffu, rm, 0), lane, x0, nx);
    const int nv = min(VX, nx - x0);
    __syncwarp();
    T* qrow = Q + (long long)(k0 - 1) * pzl + (long long)j * pyl + x0;
    for (int k = k0; k < k1; ++k) {
      const int q = k - k0 + 1;
      wait_plane(q + 1);
      const T* Pq = reinterpret_cast<const T*>(smem + ((sbase + q) % S) * Gm::STAGE);
      const T* Pn = reinterpret_cast<const T*>(smem + ((sbase + q + 1) % S) * Gm::STAGE);
      const T* Rq = reinterpret_cast<const T*>(smem + ((sbase + q) % S) * Gm::STAGE + Gm::PSTRIDE);
      float zp[VX], up[VX], dn[VX], rr[VX];
      ldv<VX>(Pn + row, zp);
      ldv<VX>(Pq + row + PW, up);
      ldv<VX>(Pq + row - PW, dn);
      ldv<VX>(Rq + ty * TX + xl, rr);
      float left = __shfl_up_sync(0xffffffffu, c[VX - 1], 1);
      float right = __shfl_down_sync(0xffffffffu, c[0], 1);
      if (lane == 0) left = tof(Pq[row - 1]);
      if (lane == 31) right = tof(Pq[row + VX]);
      float out[VX];
      if constexpr (VX == 4) {
        jac_row4(J2, c, left, right, dn, up, m, zp, rr, out);
      } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) {
          const float xm = e == 0 ? left : c[e - 1];
          const float xp = e == VX - 1 ? right : c[e + 1];
          out[e] = jacobi_update(c[e], xm, xp, dn[e], up[e], m[e], zp[e], rr[e], cx, cy, cz,
                                 omega, inv_diag);
        }
      }
      qrow += pzl;
      if (row_ok) {
        if (full_vec) {
          stv<T, VX>(qrow, out);
        } else {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (x0 + e < nx) qrow[e] = cvt<T>(out[e]);
        }
        if (tm) put_row_images<T, VX>(rimg[ty], tm, k, xl, nv, out);
        if (k == 0 || k == nz - 1) {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (x0 + e < nx) p_ghost_z<T>(L, B, dst, x0 + e, j, k, cvt<T>(out[e]));
        }
      }
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        m[e] = c[e];
        c[e] = zp[e];
      }
      if (__syncthreads_or(bad)) {
        // a plane never arrived: flag it, drain our own loads, give up
        if (tid == 0) {
          atomicOr(L.err_flag, 2);
          for (int qq = waited; qq < next_q; ++qq) {
            const int s = (sbase + qq) % S;
            mbar_wait(smem_u32(&full[s]), (parity >> s) & 1u);
            parity ^= 1u << s;
          }
        }
        __syncthreads();
        return;
      }
      // planes 0..q are no longer read: refill their stages
      const int limit = q + S;
      if (tid == 0)
        for (int qq = next_q; qq < np && qq <= limit; ++qq) issue(qq);
      next_q = max(next_q, min(np, limit + 1));
    }
    sbase = (sbase + np) % S;
  }
}

// Warp-specialised TMA sweep: warp TY of the CTA is the producer (one lane
// issues the TMA loads of each plane into an S-stage ring, waiting on the
// stage's "empty" mbarrier), warps 0..TY-1 are consumers, one row of 32 VX
// cells each.  A consumer waits only on the "full" mbarrier of the plane it
// needs next and, once it no longer reads a plane, arrives on that stage's
// empty barrier (count TY), so consumer warps never wait for each other and
// there is no CTA-wide barrier per plane.  Consumers read all seven stencil
// points of a cell and r straight from the staged planes (z-1, z, z+1 are
// three stages), so nothing is carried in registers from plane to plane.
// The planes of a CTA are numbered across its tiles; plane f lives in stage
// f % S, its full barrier completes phase f / S, and its empty barrier is
// waited with the opposite parity so the first pass through the ring does
// not wait.

template <typename T, int VX, int TY, int S>
__global__ void __launch_bounds__(32 * (TY + 1)) k_jacobi_ws(Launch L, const CUtensorMap* maps,
                                                             int zc, int src_slot, int dst,
                                                             float omega, float inv_diag) {
  using Gm = TmaGeom<T, VX, TY>;
  constexpr int TX = Gm::TX, HX = Gm::HX, PW = Gm::PW;
  constexpr int STAGE_T = Gm::STAGE / (int)sizeof(T), RS_T = Gm::PSTRIDE / (int)sizeof(T);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + S * Gm::STAGE);
  unsigned long long* empty = full + S;
  const TileQueue tq{empty + S, reinterpret_cast<unsigned*>(empty + S + 4)};
  __shared__ RowImage<T> rimg[TY][4];
  const int lane = threadIdx.x, w = threadIdx.y;
  if (smem_u32(smem) & 127u) {
    if (w == 0 && lane == 0) atomicOr(L.err_flag, 4);
    return;
  }
  if (w == 0 && lane == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), TY);
    }
    tq.init();
    mbar_fence_init();
  }
  __shared__ TileTable tt;
  __shared__ int flag0;
  flag_at_start(L, flag0);
  tile_table_build(tt, L, TX, TY, zc);  // also orders the barrier init before use
  if (flag0) return;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  const int g = L.ghost;
  constexpr int xo = kAlignBytes / (int)sizeof(T);
  const T* ring = reinterpret_cast<const T*>(smem);
  unsigned seq = 0;     // planes of this CTA so far
  unsigned issued = 0;  // planes the producer has issued
  bool bad = false;
  int blk = L.b0;
  // tiles claimed at run time from the counter in the grid's flag area
  unsigned* const ctr = tile_counter(L);
  const unsigned ctr_wrap = (unsigned)tt.start[L.nblocks] + gridDim.x - 1;
  for (unsigned kq = 0;; ++kq) {
    long long t;
    if (w == TY) {
      t = tq.claim(kq, ctr, ctr_wrap, lane);
    } else if (!tq.take(kq, t)) {
      bad = true;
      break;
    }
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int k1 = min(k0 + zc, nz);
    const int np = k1 - k0 + 2;  // planes k0 - 1 .. k1
    if (w == TY) {
      // ---------------- producer
      if (lane == 0) {
        const CUtensorMap* mp = maps + 3 * blk + src_slot;
        const CUtensorMap* mr = maps + 3 * blk + 2;
        const int px = xo + i0 - HX, pyc = g + j0 - 1, rx = xo + i0, ry = g + j0;
        Ring<S> at(seq);
        for (int q = 0; q < np; ++q, at.next()) {
          bad |= !mbar_wait(smem_u32(&empty[at.s]), at.ph ^ 1u);
          if (bad) break;
          ++issued;
          const int z = g + k0 - 1 + q;
          const bool need_r = (q >= 1 && q <= np - 2);
          const uint32_t bar = smem_u32(&full[at.s]);
          unsigned char* st = smem + at.s * Gm::STAGE;
          mbar_expect_tx(bar, Gm::PBYTES + (need_r ? Gm::RBYTES : 0));
          tma_load_3d(smem_u32(st), mp, px, pyc, z, bar);
          if (need_r) tma_load_3d(smem_u32(st + Gm::PSTRIDE), mr, rx, ry, z, bar);
        }
      }
      seq += np;
      if (bad) break;
      continue;
    }
    // ---------------- consumers (warp w = row j0 + w)
    const int j = j0 + w;
    const int xl = lane * VX;
    const int row = (w + 1) * PW + HX + xl;  // this thread's centre in a p box
    const int rrow = RS_T + w * TX + xl;     // and in the r box of the stage
    const long long pzl = B.pz;
    const int pyl = B.py;
    const int x0 = i0 + xl;
    const bool row_ok = j < ny && x0 < nx;
    const bool full_vec = x0 + VX <= nx;
    __syncwarp();
    unsigned rm = 0;
    if (lane == 0) rm = row_images<T>(L, B, dst, i0, TX, j, rimg[w]);
    const unsigned tm = thread_images<VX>(__shfl_sync(0xffffffffu, rm, 0), lane, x0, nx);
    const int nv = min(VX, nx - x0);
    __syncwarp();
    T* qrow = reinterpret_cast<T*>(L.base) + B.org[dst] + (long long)(k0 - 1) * pzl +
              (long long)j * pyl + x0;
    auto release = [&](int s) {
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    };
    // stages of planes q - 1, q and q + 1
    Ring<S> lo(seq), mid(seq), hi(seq);
    mid.next();
    hi.next();
    bad |= !mbar_wait(smem_u32(&full[lo.s]), lo.ph);
    bad |= !mbar_wait(smem_u32(&full[mid.s]), mid.ph);
    hi.next();
    for (int q = 1; q <= np - 2 && !bad; ++q) {
      bad |= !mbar_wait(smem_u32(&full[hi.s]), hi.ph);
      if (bad) break;
      const T* Pm = ring + lo.s * STAGE_T;
      const T* Pc = ring + mid.s * STAGE_T;
      const T* Pp = ring + hi.s * STAGE_T;
      float m[VX], c[VX], zp[VX], up[VX], dn[VX], rr[VX];
      ldv<VX>(Pm + row, m);
      ldv<VX>(Pc + row, c);
      ldv<VX>(Pp + row, zp);
      ldv<VX>(Pc + row + PW, up);
      ldv<VX>(Pc + row - PW, dn);
      ldv<VX>(Pc + rrow, rr);
      const float left = tof(Pc[row - 1]);
      const float right = tof(Pc[row + VX]);
      release(lo.s);
      float out[VX];
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        const float xm = e == 0 ? left : c[e - 1];
        const float xp = e == VX - 1 ? right : c[e + 1];
        out[e] = jacobi_update(c[e], xm, xp, dn[e], up[e], m[e], zp[e], rr[e], cx, cy, cz,
                                 omega, inv_diag);
      }
      const int k = k0 + q - 1;
      qrow += pzl;
      if (row_ok) {
        if (full_vec) {
          stv<T, VX>(qrow, out);
        } else {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (x0 + e < nx) qrow[e] = cvt<T>(out[e]);
        }
        if (tm) put_row_images<T, VX>(rimg[w], tm, k, xl, nv, out);
        if (k == 0 || k == nz - 1) {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (x0 + e < nx) p_ghost_z<T>(L, B, dst, x0 + e, j, k, cvt<T>(out[e]));
        }
      }
      lo = mid;
      mid = hi;
      hi.next();
    }
    if (bad) break;
    release(lo.s);
    release(mid.s);
    seq += np;
  }
  if (bad && lane == 0) atomicOr(L.err_flag, 2);
  if (w == TY && lane == 0)  // never leave with our own copies in flight
    for (unsigned f = issued > (unsigned)S ? issued - S : 0; f < issued; ++f)
      mbar_wait(smem_u32(&full[f % S]), (f / S) & 1u);
}

// Two weighted Jacobi sweeps per launch, warp-specialised (temporal
// blocking for grids whose six faces are walls).  p' = J(p), p'' = J(p')
// with the same r; p' never leaves the SM.
//
// Tile: 32 VX x TY output cells of one block (VX = 4, or 2 for narrow
// blocks), walked along z in chunks of zc planes.  Warps: TY + 2 row warps, one extras warp, one producer warp.
// The producer loads, per plane, the p box (x from i0 - HX, rows j0 - 2 ..
// j0 + TY + 1) and the r box (rows j0 - 1 .. j0 + TY) into an S-stage ring.
// In iteration t, row warps 1 .. TY first take the second sweep on plane
// m - 2 (m = k0 - 1 + t) from slots t - 3 .. t - 1 of a shared-memory ring
// of NS1 first-sweep planes and r from the stage of plane m - 2, and write
// it to global memory with its ghost-on-write images; then row warp w
// (row y = j0 - 1 + w, VX cells per lane) takes the first sweep on plane m
// over x = i0 .. i0 + 32 VX - 1 and the extras warp the cells x = i0 - 1 and
// x = i0 + 32 VX of every row; both store it, rounded to the storage type,
// into slot t (row width 32 VX + 8: x = i0 - 4 at index 0).  An mbarrier per
// slot (one arrival per thread of the TY + 3 row and extras warps) says
// that every row of a first-sweep plane is written; each iteration starts by waiting for the plane of iteration
// t - 2, which is all the second sweep needs from other warps and bounds
// the skew: a warp writing slot t may coexist with one reading slot t - 4,
// so NS1 >= 5; it is 8.  First-sweep values outside the block (walls:
// p'_ghost = p'_face) come from the face cell: the x images are written
// into the ring by the face cell's lane, the y and z images are selected
// in the second sweep of face rows and planes.  PER (every face periodic,
// ghost width >= 2, P's two ghost layers and R's first layer filled before
// the launch): the first sweep is taken on the ghost layer too, from the
// wrapped copies there, which is the first sweep on the cells they copy;
// the second sweep then needs no substitution and writes no ghost images
// (the caller fills the output's ghosts after the launch).

template <typename T, int VX, int TY>
struct Ws2Geom {
  static constexpr int TX = 32 * VX;
  static constexpr int HX = 16 / (int)sizeof(T);
  static constexpr int PW = TX + 2 * HX;  // p and r box width
  static constexpr int PBYTES = PW * (TY + 4) * (int)sizeof(T);
  static constexpr int RBYTES = PW * (TY + 2) * (int)sizeof(T);
  static constexpr int PSTRIDE = (PBYTES + 127) / 128 * 128;
  static constexpr int STAGE = PSTRIDE + (RBYTES + 127) / 128 * 128;
  static constexpr int SW = TX + 8;         // first-sweep row width (floats)
  static constexpr int SPLANE = SW * (TY + 2);
  static constexpr int NS1 = 8;             // first-sweep ring slots (a power of two)
};

__device__ __forceinline__ float jac_point(float c, float xm, float xp, float ym, float yp, float zm,
                                           float zp, float r, float cx, float cy, float cz,
                                           float omega, float inv_diag) {
  return jacobi_update(c, xm, xp, ym, yp, zm, zp, r, cx, cy, cz, omega, inv_diag);
}

// x mod n for 0 <= x < 2n
template <int N>
__device__ __forceinline__ int wrapn(int x) { return x >= N ? x - N : x; }

template <typename T, int VX, int TY, int S, bool PER>
__global__ void __launch_bounds__(32 * (TY + 4), 1) k_jacobi2_ws(Launch L, const CUtensorMap* maps,
                                                              int zc, int src_slot, int dst,
                                                              float omega, float inv_diag) {
  using G = Ws2Geom<T, VX, TY>;
  constexpr int TX = G::TX, HX = G::HX, PW = G::PW, SW = G::SW, NS1 = G::NS1;
  constexpr int NW = TY + 2;              // row warps
  constexpr int PWARP = NW + 1;           // warp NW: extras, warp NW + 1: producer
  constexpr int STAGE_T = G::STAGE / (int)sizeof(T), RS_T = G::PSTRIDE / (int)sizeof(T);
  extern __shared__ __align__(128) unsigned char smem[];
  float* s1 = reinterpret_cast<float*>(smem + S * G::STAGE);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(s1 + NS1 * G::SPLANE);
  unsigned long long* empty = full + S;
  unsigned long long* s1bar = empty + S;
  const TileQueue tq{s1bar + NS1, reinterpret_cast<unsigned*>(s1bar + NS1 + 4)};
  const int lane = threadIdx.x, w = threadIdx.y;
  if (smem_u32(smem) & 127u) {
    if (w == 0 && lane == 0) atomicOr(L.err_flag, 4);
    return;
  }
  if (w == 0 && lane == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 32 * (NW + 1));  // every lane of the row and extras warps
    }
#pragma unroll
    for (int s = 0; s < NS1; ++s) mbar_init(smem_u32(&s1bar[s]), 32 * (NW + 1));
    tq.init();
    mbar_fence_init();
  }
  __shared__ TileTable tt;
  __shared__ int flag0;
  flag_at_start(L, flag0);
  tile_table_build(tt, L, TX, TY, zc);  // also orders the barrier init before use
  if (flag0) return;
  const float cx = L.ih2[0], cy = L.ih2[1], cz = L.ih2[2];
  const Jac2 J2(cx, cy, cz, omega, inv_diag);
  const int g = L.ghost;
  constexpr int xo = kAlignBytes / (int)sizeof(T);
  const T* ring = reinterpret_cast<const T*>(smem);
  unsigned seq = 0;     // p/r planes of this CTA so far
  unsigned it1 = 0;     // first-sweep iterations of this CTA so far
  unsigned issued = 0;  // planes the producer has issued
  bool bad = false;
  int blk = L.b0;
  // tiles claimed at run time from the counter in the grid's flag area
  unsigned* const ctr = tile_counter(L);
  const unsigned ctr_wrap = (unsigned)tt.start[L.nblocks] + gridDim.x - 1;
  for (unsigned k = 0;; ++k) {
    long long t;
    if (w == PWARP) {
      t = tq.claim(k, ctr, ctr_wrap, lane);
    } else if (!tq.take(k, t)) {
      bad = true;
      break;
    }
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, TX, TY, zc, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
    const int k1 = min(k0 + zc, nz);
    const int nzc = k1 - k0;
    const int np = nzc + 4;  // p planes k0 - 2 .. k1 + 1
    if (w == PWARP) {
      // ---------------- producer
      if (lane == 0) {
        const CUtensorMap* mp = maps + 3 * blk + src_slot;
        const CUtensorMap* mr = maps + 3 * blk + 2;
        const int bx = xo + i0 - HX, py0 = g + j0 - 2, ry0 = g + j0 - 1;
        Ring<S> at(seq);
        for (int q = 0; q < np; ++q, at.next()) {
          bad |= !mbar_wait(smem_u32(&empty[at.s]), at.ph ^ 1u);
          if (bad) break;
          ++issued;
          const int z = g + k0 - 2 + q;
          const bool need_r = (q >= 1 && q <= np - 2);
          const uint32_t bar = smem_u32(&full[at.s]);
          unsigned char* st = smem + at.s * G::STAGE;
          mbar_expect_tx(bar, G::PBYTES + (need_r ? G::RBYTES : 0));
          tma_load_3d(smem_u32(st), mp, bx, py0, z, bar);
          if (need_r) tma_load_3d(smem_u32(st + G::PSTRIDE), mr, bx, ry0, z, bar);
        }
      }
      seq += np;
      it1 += nzc + 2;
      if (bad) break;
      continue;
    }
    // ---------------- row warps and the extras warp
    const bool rowwarp = w < NW;
    const int y = j0 - 1 + w;  // row of a row warp
    const bool yreal = rowwarp && y >= 0 && y < ny;
    const bool out_row = w >= 1 && w <= TY && yreal;  // second-sweep rows of this tile
    // first-sweep rows: inside the block, or (PER) also the ghost rows
    const bool y1 = PER ? rowwarp && y >= -1 && y <= ny : yreal;
    const int xl = lane * VX;
    const int x0 = i0 + xl;
    const int nv = min(VX, nx - x0);         // cells of this lane inside the block
    const int prow = (w + 1) * PW + HX + xl; // p box: this lane's first cell
    const int rrow = RS_T + w * PW + HX + xl;
    const int srow = w * SW + 4 + xl;        // first-sweep ring
    const bool xhi_in = nv >= 1 && x0 + nv == nx;  // this lane holds x = nx - 1
    // extras warp: cell c < 2 NW is row c / 2, x = i0 - 1 (even c) or i0 + TX;
    // lane l takes cells l and l + 32
    constexpr int NE = (2 * NW + 31) / 32;
    const long long pzl = B.pz;
    T* qrow = reinterpret_cast<T*>(L.base) + B.org[dst] + (long long)y * B.py + x0 +
              (long long)k0 * pzl;  // plane k0 of the output row
    // this lane has first-sweep cells (PER: also the ghost column x = nx)
    const bool act1 = y1 && (PER ? x0 <= nx : nv > 0);
    const bool act2 = out_row && nv > 0;               // ... and second-sweep outputs
    const bool yface = (y == 0) | (y == ny - 1);
    const bool xface = (lane == 0 && i0 == 0) | xhi_in;  // lanes with an x image
    const int pyl = B.py;
    // Ring cursors, moved on once per iteration t by an add and a wrap: the
    // stages of p planes q - 1 .. q + 2 (q = t), the full barrier of q + 2
    // with its phase, the empty barrier of q - 1, the first-sweep slots of
    // iterations u - 3 .. u (u = it1 + t, numbered across tiles), the slot
    // barrier of u - 2 (waited on, with its phase) and that of u (arrived
    // at), and the output row of plane k0 - 3 + t.  Every lane arrives on
    // the empty and slot barriers itself (their counts are per thread), so
    // no warp sync or single-lane branch is needed.
    const T* const ring_end = ring + S * STAGE_T;
    float* const s1_end = s1 + NS1 * G::SPLANE;
    const uint32_t full0 = smem_u32(&full[0]), empty0 = smem_u32(&empty[0]);
    const uint32_t s1b0 = smem_u32(&s1bar[0]);
    const int st0 = (int)(seq % S);
    const T* stR = ring + (st0 == 0 ? S - 1 : st0 - 1) * STAGE_T;
    const T* stM = ring + st0 * STAGE_T;
    const T* stC = ring + wrapn<S>(st0 + 1) * STAGE_T;
    const T* stP = ring + wrapn<S>(st0 + 2) * STAGE_T;
    uint32_t fbar = full0 + 8u * (uint32_t)wrapn<S>(st0 + 2), fph = ((seq + 2) / S) & 1u;
    uint32_t ebar = empty0 + 8u * (uint32_t)(st0 == 0 ? S - 1 : st0 - 1);
    const unsigned u0 = it1;
    float* sA = s1 + (int)((u0 - 3) & (NS1 - 1)) * G::SPLANE;
    float* sB = s1 + (int)((u0 - 2) & (NS1 - 1)) * G::SPLANE;
    float* sC = s1 + (int)((u0 - 1) & (NS1 - 1)) * G::SPLANE;
    float* sW = s1 + (int)(u0 & (NS1 - 1)) * G::SPLANE;
    uint32_t bwait = s1b0 + 8u * ((u0 - 2) & (NS1 - 1)), bwph = ((u0 - 2) / NS1) & 1u;
    uint32_t barr = s1b0 + 8u * (u0 & (NS1 - 1));
    T* qk = qrow - 3 * pzl;
    auto advance = [&]() {
      stR = stM;
      stM = stC;
      stC = stP;
      stP = stP + STAGE_T == ring_end ? ring : stP + STAGE_T;
      fbar += 8u;
      if (fbar == full0 + 8u * S) {
        fbar = full0;
        fph ^= 1u;
      }
      ebar = ebar + 8u == empty0 + 8u * S ? empty0 : ebar + 8u;
      sA = sB;
      sB = sC;
      sC = sW;
      sW = sW + G::SPLANE == s1_end ? s1 : sW + G::SPLANE;
      bwait += 8u;
      if (bwait == s1b0 + 8u * NS1) {
        bwait = s1b0;
        bwph ^= 1u;
      }
      barr = barr + 8u == s1b0 + 8u * NS1 ? s1b0 : barr + 8u;
      qk += pzl;
    };
    // first sweep on plane m = k0 - 1 + t into slot u = it1 + t
    auto sweep1 = [&](int t) {
      const int m = k0 - 1 + t;
      if (!mbar_wait_split(fbar, fph)) bad = true;
      if (bad) return;
      const T* Pm = stM;
      const T* Pc = stC;
      const T* Pp = stP;
      float* S1 = sW;
      const bool mreal = PER ? (m >= -1) & (m <= nz) : (m >= 0) & (m < nz);
      if (act1 && mreal) {
        float c[VX], zm[VX], zp[VX], yp[VX], ym[VX], rr[VX];
        ldv<VX>(Pc + prow, c);
        ldv<VX>(Pm + prow, zm);
        ldv<VX>(Pp + prow, zp);
        ldv<VX>(Pc + prow + PW, yp);
        ldv<VX>(Pc + prow - PW, ym);
        ldv<VX>(Pc + rrow, rr);
        const float left = tof(Pc[prow - 1]);
        const float right = tof(Pc[prow + VX]);
        float o[VX];
        jac_row<VX>(J2, c, left, right, ym, yp, zm, zp, rr, o);
#pragma unroll
        for (int e = 0; e < VX; ++e) o[e] = tof(cvt<T>(o[e]));
        if constexpr (VX == 4)
          *reinterpret_cast<float4*>(S1 + srow) = make_float4(o[0], o[1], o[2], o[3]);
        else
          *reinterpret_cast<float2*>(S1 + srow) = make_float2(o[0], o[1]);
        if constexpr (!PER) {
          if (lane == 0 && i0 == 0) S1[srow - 1] = o[0];    // x = -1 <- x = 0
          if (xhi_in) S1[srow + nv] = pick<VX>(o, nv - 1);  // x = nx <- x = nx - 1
        }
      }
      if (!rowwarp && mreal) {
#pragma unroll
        for (int q = 0; q < NE; ++q) {
          const int ce = lane + 32 * q;
          const int er = ce >> 1, ex = (ce & 1) ? i0 + TX : i0 - 1, ey = j0 - 1 + er;
          const bool in = PER ? ex >= -1 && ex <= nx && ey >= -1 && ey <= ny
                              : ex >= 0 && ex < nx && ey >= 0 && ey < ny;
          if (ce < 2 * NW && in) {
            const int epi = (er + 1) * PW + HX + (ex - i0);
            const int eri = RS_T + er * PW + HX + (ex - i0);
            S1[er * SW + 4 + (ex - i0)] = tof(cvt<T>(
                jac_point(tof(Pc[epi]), tof(Pc[epi - 1]), tof(Pc[epi + 1]), tof(Pc[epi - PW]),
                          tof(Pc[epi + PW]), tof(Pm[epi]), tof(Pp[epi]), tof(Pc[eri]), cx, cy, cz,
                          omega, inv_diag)));
          }
        }
      }
    };
    // second sweep on plane P = k0 - 3 + t from slots u - 3, u - 2, u - 1
    // (u = it1 + t) and r from the stage of plane P (q = t - 1)
    auto sweep2 = [&](int t) {
      const int P = k0 - 3 + t;
      const float* A = sA + srow;
      const float* Bc = sB + srow;
      const float* C = sC + srow;
      const T* Rp = stR;
      float c[VX], zm[VX], zp[VX], yp[VX], ym[VX], rr[VX];
      ldv<VX>(Bc, c);
      ldv<VX>(A, zm);
      ldv<VX>(C, zp);
      ldv<VX>(Bc + SW, yp);
      ldv<VX>(Bc - SW, ym);
      ldv<VX>(Rp + rrow, rr);
      const float left = Bc[-1];
      const float right = Bc[VX];
      const bool zlo = !PER && P == 0, zhi = !PER && P == nz - 1;
      if (!PER && (yface | zlo | zhi)) {
        // face rows and planes: the first sweep's ghost is the face value
#pragma unroll
        for (int e = 0; e < VX; ++e) {
          if (y == 0) ym[e] = c[e];
          if (y == ny - 1) yp[e] = c[e];
          if (zlo) zm[e] = c[e];
          if (zhi) zp[e] = c[e];
        }
      }
      float out[VX];
      jac_row<VX>(J2, c, left, right, ym, yp, zm, zp, rr, out);
      auto put = [&](T* q) {
        if (nv >= VX) {
          stv<T, VX>(q, out);
        } else {
#pragma unroll
          for (int e = 0; e < VX; ++e)
            if (e < nv) q[e] = cvt<T>(out[e]);
        }
      };
      put(qk);
      // ghost-on-write at the walls (this kernel runs only when all six
      // faces are walls): the first ghost layer takes the face value, in
      // the same block, next to the face cell
      if (!PER && __builtin_expect(xface | yface | zlo | zhi, 0)) {
        if (lane == 0 && i0 == 0) qk[-1] = cvt<T>(out[0]);
        if (xhi_in) qk[nv] = cvt<T>(pick<VX>(out, nv - 1));
        if (y == 0) put(qk - pyl);
        if (y == ny - 1) put(qk + pyl);
        if (zlo) put(qk - pzl);
        if (zhi) put(qk + pzl);
      }
    };
    // end of iteration t: the first-sweep plane of slot u is written and
    // (t >= 1) the stage of plane m - 2 is no longer read
    auto finish = [&](bool first_plane_done, bool stage_done) {
      if (first_plane_done) mbar_arrive(barr);
      if (stage_done) mbar_arrive(ebar);
      advance();
    };
    // planes k0 - 2 and k0 - 1 must be there before the first iteration
    if (!mbar_wait_split(full0 + 8u * (uint32_t)st0, (seq / S) & 1u)) bad = true;
    if (!mbar_wait_split(full0 + 8u * (uint32_t)wrapn<S>(st0 + 1), ((seq + 1) / S) & 1u)) bad = true;
    // Each iteration first waits for the first-sweep plane of two iterations
    // before (also across tiles: this bounds the skew between warps), takes
    // the second sweep (iterations 3 ..), then the first (.. nzc + 1).
    // Iterations 0 .. 2: first sweep only (the first output plane needs the
    // first sweep on k0 - 1 .. k0 + 1).
    for (int t2 = 0; t2 < 3 && !bad; ++t2) {
      if (it1 + t2 >= 2 && !mbar_wait_split(bwait, bwph)) bad = true;
      if (bad) break;
      sweep1(t2);
      if (bad) break;
      finish(true, t2 >= 1);
    }
    // iterations 3 .. nzc + 1: both sweeps
    for (int t2 = 3; t2 <= nzc + 1 && !bad; ++t2) {
      if (!mbar_wait_split(bwait, bwph)) bad = true;
      if (bad) break;
      if (act2) sweep2(t2);
      sweep1(t2);
      if (bad) break;
      finish(true, true);
    }
    // iteration nzc + 2: second sweep on the last plane only
    if (!bad) {
      if (!mbar_wait_split(bwait, bwph)) bad = true;
      if (!bad) {
        if (act2) sweep2(nzc + 2);
        finish(false, true);
      }
    }
    if (bad) break;
    // stages of planes k1, k1 + 1 (q = nzc + 2, nzc + 3): ebar is that of
    // q = nzc + 2 now
    mbar_arrive(ebar);
    mbar_arrive(ebar + 8u == empty0 + 8u * S ? empty0 : ebar + 8u);
    seq += np;
    it1 += nzc + 2;
  }
  if (bad && lane == 0) atomicOr(L.err_flag, 2);
  if (w == PWARP && lane == 0)  // never leave with our own copies in flight
    for (unsigned f = issued > (unsigned)S ? issued - S : 0; f < issued; ++f)
      mbar_wait(smem_u32(&full[f % S]), (f / S) & 1u);
}

template <typename T, int VX, int TY, int S, bool PER>
cudaError_t run_ws2(const Launch& L, const JacobiCfg& c, const void* maps, int src_slot, int dst,
                    float omega, float inv_diag) {
  using G = Ws2Geom<T, VX, TY>;
  auto kern = k_jacobi2_ws<T, VX, TY, S, PER>;
  const int smem = S * G::STAGE + G::NS1 * G::SPLANE * 4 + 8 * (2 * S + G::NS1 + 4) + 16;
  static int occ = -1;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (TY + 4), smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
  }
  const long long tiles = count_tiles(L, G::TX, TY, c.zc);
  long long grid = (long long)L.sms * occ;
  if (tiles < grid) grid = tiles;
  kern<<<(unsigned)(grid > 0 ? grid : 1), dim3(32, TY + 4), smem, L.stream>>>(
      L, static_cast<const CUtensorMap*>(maps), c.zc, src_slot, dst, omega, inv_diag);
  return cudaGetLastError();
}

template <typename T, int VX, int TY, int S>
cudaError_t run_ws(const Launch& L, const JacobiCfg& c, const void* maps, int src_slot, int dst,
                   float omega, float inv_diag) {
  using Gm = TmaGeom<T, VX, TY>;
  auto kern = k_jacobi_ws<T, VX, TY, S>;
  const int smem = S * Gm::STAGE + 16 * S + 8 * 4 + 16;  // stages, full/empty, tile queue
  static int occ = -1;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * (TY + 1), smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
  }
  const long long tiles = count_tiles(L, Gm::TX, TY, c.zc);
  long long grid = (long long)L.sms * occ;
  if (tiles < grid) grid = tiles;
  kern<<<(unsigned)(grid > 0 ? grid : 1), dim3(32, TY + 1), smem, L.stream>>>(
      L, static_cast<const CUtensorMap*>(maps), c.zc, src_slot, dst, omega, inv_diag);
  return cudaGetLastError();
}

template <typename T, int VX, int TY, int S>
cudaError_t run(const Launch& L, const JacobiCfg& c, const void* maps, int src_slot, int dst,
                float omega, float inv_diag) {
  using Gm = TmaGeom<T, VX, TY>;
  auto kern = k_jacobi_tma<T, VX, TY, S>;
  const int smem = S * Gm::STAGE + 8 * S;
  static int occ = -1;
  if (occ < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * TY, smem) != cudaSuccess || occ < 1)
      occ = 1;
  }
  const long long tiles = count_tiles(L, Gm::TX, TY, c.zc);
  long long grid = (long long)L.sms * occ;
  if (tiles < grid) grid = tiles;
  kern<<<(unsigned)(grid > 0 ? grid : 1), dim3(32, TY), smem, L.stream>>>(
      L, static_cast<const CUtensorMap*>(maps), c.zc, src_slot, dst, omega, inv_diag);
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

cudaError_t launch_wait_probe(const Launch& L, int form) {
  k_wait_probe<<<1, 32, 0, L.stream>>>(L.err_flag, form);
  return cudaGetLastError();
}

int tma_box_x(int dtype, int vx, int halo) {
  const int es = dtype == 0 ? 4 : 2;
  return 32 * vx + (halo ? 2 * (16 / es) : 0);
}

bool encode_jacobi_maps(void* out_host, const TmaArray* arrays, int narrays, int dtype,
                        const JacobiCfg& c) {
  auto enc = encoder();
  if (!enc) return false;
  const int es = dtype == 0 ? 4 : 2;
  const CUtensorMapDataType dt = dtype == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : dtype == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUtensorMap* maps = static_cast<CUtensorMap*>(out_host);
  for (int a = 0; a < narrays; ++a) {
    const TmaArray& A = arrays[a];
    const bool is_r = (a % 3) == 2;
    cuuint64_t dims[3] = {(cuuint64_t)A.row_elems, (cuuint64_t)A.rows, (cuuint64_t)A.planes};
    cuuint64_t strides[2] = {(cuuint64_t)A.row_elems * es, (cuuint64_t)A.row_elems * A.rows * es};
    // kind 9 (two sweeps): p box rows j0 - 2 .. j0 + ty + 1, r box with the
    // same x halo and rows j0 - 1 .. j0 + ty
    const bool two = c.kind == 9;
    cuuint32_t box[3] = {(cuuint32_t)tma_box_x(dtype, c.vx, two || !is_r),
                         (cuuint32_t)(c.ty + (two ? (is_r ? 2 : 4) : (is_r ? 0 : 2))), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    memset(&maps[a], 0, sizeof(CUtensorMap));
    CUresult r = enc(&maps[a], dt, 3, A.ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

#define CFD_DISPATCH_T(dtype, ...)                           \
  switch (dtype) {                                           \
    case 0: { using T = float; __VA_ARGS__; } break;         \
    case 1: { using T = __nv_bfloat16; __VA_ARGS__; } break; \
    default: { using T = __half; __VA_ARGS__; } break;       \
  }

template <bool PER>
static cudaError_t dispatch_ws2(const Launch& L, const JacobiCfg& c, const void* maps_dev,
                                int src_slot, int dst, float omega, float inv_diag) {
  cudaError_t e = cudaErrorInvalidValue;
  CFD_DISPATCH_T(L.dtype, {
    if (c.vx == 2 && c.ty == 16) e = run_ws2<T, 2, 16, 6, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 2) e = run_ws2<T, 2, 8, 6, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.ty == 16 && c.stages == 7) e = run_ws2<T, 4, 16, 7, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.ty == 16) e = run_ws2<T, 4, 16, 6, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.stages == 6) e = run_ws2<T, 4, 8, 6, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else e = run_ws2<T, 4, 8, 5, PER>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
  });
  return e;
}

cudaError_t launch_jacobi2_ws(const Launch& L, const JacobiCfg& c, const void* maps_dev,
                              int src_slot, int dst, float omega, bool periodic) {
  const float inv_diag = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  return periodic ? dispatch_ws2<true>(L, c, maps_dev, src_slot, dst, omega, inv_diag)
                  : dispatch_ws2<false>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
}

cudaError_t launch_jacobi_tma(const Launch& L, const JacobiCfg& c, const void* maps_dev,
                              int src_slot, int dst, float omega) {
  const float inv_diag = 1.f / (2.f * (L.ih2[0] + L.ih2[1] + L.ih2[2]));
  cudaError_t e = cudaErrorInvalidValue;
  if (c.kind == 7 && c.vx == 2) {  // 64-wide tiles for narrow blocks
    CFD_DISPATCH_T(L.dtype, {
      if (c.ty == 8) e = run_ws<T, 2, 8, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else e = run_ws<T, 2, 16, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    });
    return e;
  }
  if (c.kind == 7) {
    CFD_DISPATCH_T(L.dtype, {
      if (c.ty == 4 && c.stages == 8) e = run_ws<T, 4, 4, 8>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else if (c.ty == 4) e = run_ws<T, 4, 4, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else if (c.ty == 8 && c.stages == 8) e = run_ws<T, 4, 8, 8>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else if (c.ty == 8) e = run_ws<T, 4, 8, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else if (c.stages == 8) e = run_ws<T, 4, 16, 8>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
      else e = run_ws<T, 4, 16, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    });
    return e;
  }
  CFD_DISPATCH_T(L.dtype, {
    if (c.vx == 4 && c.ty == 4 && c.stages == 4) e = run<T, 4, 4, 4>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 4) e = run<T, 4, 4, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 8 && c.stages == 4) e = run<T, 4, 8, 4>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 8) e = run<T, 4, 8, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 16 && c.stages == 4) e = run<T, 4, 16, 4>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 4 && c.ty == 16) e = run<T, 4, 16, 6>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else if (c.vx == 2 && c.ty == 16) e = run<T, 2, 16, 4>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
    else e = run<T, 2, 8, 4>(L, c, maps_dev, src_slot, dst, omega, inv_diag);
  });
  return e;
}

}  // namespace cfd
