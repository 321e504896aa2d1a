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

namespace cfd {
namespace {

__global__ void __launch_bounds__(256) k_mg_restrict(MgView f, const float* __restrict__ r,
                                                     MgView c, float cx, float cy, float cz) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= c.n[0] || J >= c.n[1]) return;
  const float* __restrict__ p = f.o;
  const long long fpz = f.pz;
  const int fpy = f.py;
  // p at local offsets (kk, jj, ii) in -1..2 around fine cell (2I, 2J, 2K)
  auto P = [&](int kk, int jj, int ii) -> float {
    return __ldg(p + (long long)(2 * K + kk) * fpz + (long long)(2 * J + jj) * fpy + (2 * I + ii));
  };
  float s = 0.f;
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float pc = P(cc, b, a);
        const float lp = ((P(cc, b, a - 1) + P(cc, b, a + 1)) - 2.f * pc) * cx +
                         ((P(cc, b - 1, a) + P(cc, b + 1, a)) - 2.f * pc) * cy +
                         ((P(cc - 1, b, a) + P(cc + 1, b, a)) - 2.f * pc) * cz;
        const float rv =
            __ldg(r + (long long)(2 * K + cc) * fpz + (long long)(2 * J + b) * fpy + (2 * I + a));
        s += rv - lp;
      }
  c.o[(long long)K * c.pz + (long long)J * c.py + I] = 0.125f * s;
}

__global__ void __launch_bounds__(256) k_mg_prolong(MgView f, MgView c) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= c.n[0] || J >= c.n[1]) return;
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
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        // child (a, b, cc): its second coarse neighbour lies on its own side
        const int oa = a ? 1 : -1, ob = b ? 1 : -1, oc = cc ? 1 : -1;
        float v = 0.f;
#pragma unroll
        for (int sc = 0; sc < 2; ++sc)
#pragma unroll
          for (int sb = 0; sb < 2; ++sb)
#pragma unroll
            for (int sa = 0; sa < 2; ++sa)
              v += w[sa] * w[sb] * w[sc] * E[1 + sc * oc][1 + sb * ob][1 + sa * oa];
        float* q = f.o + (long long)(2 * K + cc) * f.pz + (long long)(2 * J + b) * f.py + (2 * I + a);
        *q += v;
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

cudaError_t launch_mg_prolong(cudaStream_t s, const MgView& fine_p, const MgView& coarse_e) {
  k_mg_prolong<<<coarse_grid(coarse_e), dim3(32, 8), 0, s>>>(fine_p, coarse_e);
  return cudaGetLastError();
}

}  // namespace cfd
