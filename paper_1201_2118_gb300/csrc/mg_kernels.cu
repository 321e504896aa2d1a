// Grid-transfer kernels of the cell-centred multigrid V-cycle for the
// pressure equation L p = r (FP32 storage).
//
// Level l + 1 halves every axis of level l: coarse cell (I, J, K) covers the
// fine cells 2I..2I+1, 2J..2J+1, 2K..2K+1.  Both kernels give one thread one
// coarse cell (32 x 8 threads per CTA over x and y, one CTA row of z per
// grid z index), so a warp reads 64 consecutive fine values of a row.
//
//  * restriction: rc = mean over the 8 children of (r - L p), L the 7-point
//    operator with the fine level's 1/h^2 (fine ghosts must be current);
//  * prolongation: p += the trilinear interpolation of the coarse correction
//    e at the fine centres, which sit a quarter of a coarse cell from the
//    nearest coarse centre along each axis (weights 3/4 and 1/4, reading the
//    coarse ghost layer next to the faces).
#include "cfd_internal.h"
#include "dev_common.cuh"

namespace cfd {
namespace {

__device__ __forceinline__ float2 ld2(const float* q) {
  return __ldg(reinterpret_cast<const float2*>(q));
}

// The two children along x of a coarse cell are one aligned float2 (2I is
// even and every row's x = 0 is 128-byte aligned).
__global__ void __launch_bounds__(256) k_mg_restrict(MgView f, const float* __restrict__ r,
                                                     MgView c, float cx, float cy, float cz) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= c.n[0] || J >= c.n[1]) return;
  const long long fpz = f.pz;
  const int fpy = f.py;
  // start of fine row (2J + jj, 2K + kk) at x = 2I
  auto row = [&](const float* a, int kk, int jj) {
    return a + (long long)(2 * K + kk) * fpz + (long long)(2 * J + jj) * fpy + 2 * I;
  };
  float s = 0.f;
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float* q = row(f.o, cc, b);
      const float2 pc = ld2(q);
      const float xl = __ldg(q - 1), xr = __ldg(q + 2);
      const float2 ym = ld2(row(f.o, cc, b - 1)), yp = ld2(row(f.o, cc, b + 1));
      const float2 zm = ld2(row(f.o, cc - 1, b)), zp = ld2(row(f.o, cc + 1, b));
      const float2 rv = ld2(row(r, cc, b));
      const float lp0 = ((xl + pc.y) - 2.f * pc.x) * cx + ((ym.x + yp.x) - 2.f * pc.x) * cy +
                        ((zm.x + zp.x) - 2.f * pc.x) * cz;
      const float lp1 = ((pc.x + xr) - 2.f * pc.y) * cx + ((ym.y + yp.y) - 2.f * pc.y) * cy +
                        ((zm.y + zp.y) - 2.f * pc.y) * cz;
      s += rv.x - lp0;
      s += rv.y - lp1;
    }
  c.o[(long long)K * c.pz + (long long)J * c.py + I] = 0.125f * s;
}

// The fine cells' face ghost images are written with them (periodic: the
// opposite ghost; wall: the mirror ghost), so the 7-point consumers that
// follow need no ghost launch.
__device__ __forceinline__ void face_images(const MgView& f, const int per[3], int i, int j, int k,
                                            float v) {
  const long long o = (long long)k * f.pz + (long long)j * f.py + i;
  if (i == 0) f.o[o + (per[0] ? f.n[0] : -1)] = v;
  if (i == f.n[0] - 1) f.o[o + (per[0] ? -f.n[0] : 1)] = v;
  if (j == 0) f.o[o + (long long)(per[1] ? f.n[1] : -1) * f.py] = v;
  if (j == f.n[1] - 1) f.o[o + (long long)(per[1] ? -f.n[1] : 1) * f.py] = v;
  if (k == 0) f.o[o + (per[2] ? f.n[2] : -1) * f.pz] = v;
  if (k == f.n[2] - 1) f.o[o + (per[2] ? -f.n[2] : 1) * f.pz] = v;
}

__global__ void __launch_bounds__(256) k_mg_prolong(MgView f, MgView c, int3 per3) {
  const int per[3] = {per3.x, per3.y, per3.z};
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= c.n[0] || J >= c.n[1]) return;
  // the four fine row pairs first: stores through the same pointer would
  // otherwise hold each load back behind the previous row's store
  float2* q[2][2];
  float2 pv[2][2];
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      q[cc][b] = reinterpret_cast<float2*>(f.o + (long long)(2 * K + cc) * f.pz +
                                           (long long)(2 * J + b) * f.py + 2 * I);
      pv[cc][b] = *q[cc][b];
    }
  const float* __restrict__ e = c.o;
  float E[3][3][3];  // coarse correction at offsets -1..1 around (I, J, K)
#pragma unroll
  for (int kk = 0; kk < 3; ++kk)
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
        E[kk][jj][ii] = __ldg(e + (long long)(K + kk - 1) * c.pz + (long long)(J + jj - 1) * c.py +
                              (I + ii - 1));
  const float w[2] = {0.75f, 0.25f};
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      // children (a, b, cc), a = 0, 1: the second coarse neighbour of each
      // lies on its own side
      const int ob = b ? 1 : -1, oc = cc ? 1 : -1;
      float v[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int oa = a ? 1 : -1;
        float t = 0.f;
#pragma unroll
        for (int sc = 0; sc < 2; ++sc)
#pragma unroll
          for (int sb = 0; sb < 2; ++sb)
#pragma unroll
            for (int sa = 0; sa < 2; ++sa)
              t += w[sa] * w[sb] * w[sc] * E[1 + sc * oc][1 + sb * ob][1 + sa * oa];
        v[a] = t;
      }
      pv[cc][b].x += v[0];
      pv[cc][b].y += v[1];
    }
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      *q[cc][b] = pv[cc][b];
      const int i = 2 * I, j = 2 * J + b, k = 2 * K + cc;
      if (i == 0 || i + 1 == f.n[0] - 1 || j == 0 || j == f.n[1] - 1 || k == 0 || k == f.n[2] - 1) {
        face_images(f, per, i, j, k, pv[cc][b].x);
        face_images(f, per, i + 1, j, k, pv[cc][b].y);
      }
    }
}

// ----------------------------------------------------- bottom of the cycle
//
// Each level's P, its ping-pong copy and R hold interior cells only; a
// neighbour index outside the level maps to the cell a ghost fill would
// copy (periodic: wrap; wall: the mirror image, the first interior cell).
// Mapping each axis on its own gives the same edge and corner values as the
// sequential x, y, z ghost passes.  One barrier per sweep.

__device__ __forceinline__ int map_ix(int i, int n, int per) {
  return i < 0 ? (per ? n - 1 : 0) : (i >= n ? (per ? 0 : n - 1) : i);
}

struct BLevel {
  float* p[2];  // iterate and ping-pong copy
  float* r;
  int cur;      // which of p[] holds the iterate
  int n0, n1, n2;
};

__device__ __forceinline__ float bat(const float* a, const BLevel& L, const int per[3], int i,
                                     int j, int k) {
  return a[(map_ix(k, L.n2, per[2]) * L.n1 + map_ix(j, L.n1, per[1])) * L.n0 +
           map_ix(i, L.n0, per[0])];
}

__device__ void bottom_sweeps(BLevel& L, int n, const MgBottom& b, int q) {
  const int cells = L.n0 * L.n1 * L.n2;
  const float cx = b.c[q][0], cy = b.c[q][1], cz = b.c[q][2];
  for (int it = 0; it < n; ++it) {
    const float* src = L.p[L.cur];
    float* dst = L.p[L.cur ^ 1];
    for (int t = threadIdx.x; t < cells; t += blockDim.x) {
      const int i = t % L.n0, j = (t / L.n0) % L.n1, k = t / (L.n0 * L.n1);
      dst[t] = jacobi_update(src[t], bat(src, L, b.per, i - 1, j, k), bat(src, L, b.per, i + 1, j, k),
                             bat(src, L, b.per, i, j - 1, k), bat(src, L, b.per, i, j + 1, k),
                             bat(src, L, b.per, i, j, k - 1), bat(src, L, b.per, i, j, k + 1), L.r[t],
                             cx, cy, cz, b.omega, b.inv_diag[q]);
    }
    L.cur ^= 1;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_mg_bottom(MgBottom b) {
  extern __shared__ __align__(16) float bsm[];
  BLevel lv[kMgBottomLevels];
  {
    float* q = bsm;
    for (int l = 0; l < b.levels; ++l) {
      lv[l].n0 = b.n[l][0];
      lv[l].n1 = b.n[l][1];
      lv[l].n2 = b.n[l][2];
      const int cells = lv[l].n0 * lv[l].n1 * lv[l].n2;
      lv[l].p[0] = q;
      lv[l].p[1] = q + cells;
      lv[l].r = q + 2 * cells;
      lv[l].cur = 0;
      q += 3 * cells;
    }
  }
  {  // level 0: R from global, zero correction
    const BLevel& L = lv[0];
    for (int t = threadIdx.x; t < L.n0 * L.n1 * L.n2; t += blockDim.x) {
      const int i = t % L.n0, j = (t / L.n0) % L.n1, k = t / (L.n0 * L.n1);
      L.r[t] = b.r_in.o[(long long)k * b.r_in.pz + (long long)j * b.r_in.py + i];
      L.p[0][t] = 0.f;
    }
  }
  __syncthreads();
  // down: smooth, restrict the residual, zero the next correction
  for (int l = 0; l + 1 < b.levels; ++l) {
    BLevel& F = lv[l];
    BLevel& C = lv[l + 1];
    bottom_sweeps(F, b.nu1, b, l);
    const float* p = F.p[F.cur];
    const float cx = b.c[l][0], cy = b.c[l][1], cz = b.c[l][2];
    for (int t = threadIdx.x; t < C.n0 * C.n1 * C.n2; t += blockDim.x) {
      const int I = t % C.n0, J = (t / C.n0) % C.n1, K = t / (C.n0 * C.n1);
      float s = 0.f;
      for (int cc = 0; cc < 2; ++cc)
        for (int bb = 0; bb < 2; ++bb)
          for (int a = 0; a < 2; ++a) {
            const int i = 2 * I + a, j = 2 * J + bb, k = 2 * K + cc;
            const float pc = p[(k * F.n1 + j) * F.n0 + i];
            const float lp =
                ((bat(p, F, b.per, i - 1, j, k) + bat(p, F, b.per, i + 1, j, k)) - 2.f * pc) * cx +
                ((bat(p, F, b.per, i, j - 1, k) + bat(p, F, b.per, i, j + 1, k)) - 2.f * pc) * cy +
                ((bat(p, F, b.per, i, j, k - 1) + bat(p, F, b.per, i, j, k + 1)) - 2.f * pc) * cz;
            s += F.r[(k * F.n1 + j) * F.n0 + i] - lp;
          }
      C.r[t] = 0.125f * s;
      C.p[0][t] = 0.f;
    }
    __syncthreads();
  }
  bottom_sweeps(lv[b.levels - 1], b.ncoarse, b, b.levels - 1);
  // up: prolong the correction, smooth
  const float w[2] = {0.75f, 0.25f};
  for (int l = b.levels - 2; l >= 0; --l) {
    BLevel& F = lv[l];
    const BLevel& C = lv[l + 1];
    const float* e = C.p[C.cur];
    float* p = F.p[F.cur];
    for (int t = threadIdx.x; t < F.n0 * F.n1 * F.n2; t += blockDim.x) {
      const int i = t % F.n0, j = (t / F.n0) % F.n1, k = t / (F.n0 * F.n1);
      const int I = i / 2, J = j / 2, K = k / 2;
      const int oi = (i & 1) ? 1 : -1, oj = (j & 1) ? 1 : -1, ok = (k & 1) ? 1 : -1;
      float v = 0.f;
      for (int sc = 0; sc < 2; ++sc)
        for (int sb = 0; sb < 2; ++sb)
          for (int sa = 0; sa < 2; ++sa)
            v += w[sa] * w[sb] * w[sc] * bat(e, C, b.per, I + sa * oi, J + sb * oj, K + sc * ok);
      p[t] += v;
    }
    __syncthreads();
    bottom_sweeps(F, b.nu2, b, l);
  }
  // level 0's correction with its first ghost layer
  const BLevel& L = lv[0];
  const float* p = L.p[L.cur];
  const int e0 = L.n0 + 2, e1 = L.n1 + 2, e2 = L.n2 + 2;
  for (int t = threadIdx.x; t < e0 * e1 * e2; t += blockDim.x) {
    const int i = t % e0 - 1, j = (t / e0) % e1 - 1, k = t / (e0 * e1) - 1;
    b.p_out.o[(long long)k * b.p_out.pz + (long long)j * b.p_out.py + i] = bat(p, L, b.per, i, j, k);
  }
}

dim3 coarse_grid(const MgView& c) {
  return dim3((unsigned)((c.n[0] + 31) / 32), (unsigned)((c.n[1] + 7) / 8), (unsigned)c.n[2]);
}

}  // namespace

cudaError_t launch_mg_restrict(cudaStream_t s, const MgView& fine_p, const float* fine_r,
                               const MgView& coarse_r, const float ih2_fine[3]) {
  k_mg_restrict<<<coarse_grid(coarse_r), dim3(32, 8), 0, s>>>(fine_p, fine_r, coarse_r, ih2_fine[0],
                                                             ih2_fine[1], ih2_fine[2]);
  return cudaGetLastError();
}

size_t mg_bottom_smem(const MgBottom& b) {
  size_t cells = 0;
  for (int l = 0; l < b.levels; ++l) cells += (size_t)b.n[l][0] * b.n[l][1] * b.n[l][2];
  return 3 * cells * sizeof(float);
}

// Largest bottom: kMgBottomCells on its first level, 1/8 of that on each
// further one, three arrays each.
constexpr size_t kMgBottomSmemMax = 3 * sizeof(float) * (kMgBottomCells + kMgBottomCells / 7 + 64);

cudaError_t prepare_mg_bottom() {
  return cudaFuncSetAttribute(k_mg_bottom, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kMgBottomSmemMax);
}

cudaError_t launch_mg_bottom(cudaStream_t s, const MgBottom& b) {
  const size_t smem = mg_bottom_smem(b);
  if (smem > kMgBottomSmemMax) return cudaErrorInvalidValue;
  k_mg_bottom<<<1, 1024, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_mg_prolong(cudaStream_t s, const MgView& fine_p, const MgView& coarse_e,
                              const int periodic[3]) {
  k_mg_prolong<<<coarse_grid(coarse_e), dim3(32, 8), 0, s>>>(
      fine_p, coarse_e, make_int3(periodic[0], periodic[1], periodic[2]));
  return cudaGetLastError();
}

}  // namespace cfd
