// Discrete adjoint of the RK2 projection step (periodic block, order 2).
//
// The transposes used (MAC grid, periodic): L^T = L, D^T = -G, G^T = -D, and
// one weighted Jacobi sweep p' = M p - (w/diag) r has a symmetric M.  For K
// sweeps started from warm start p0, the transpose maps a cotangent lam of
// the result to
//   lam_r  = -(w/diag) b_K,   lam_p0 = b_{K+1} - b_K,
// where b_{m+1} = M b_m + lam, b_1 = lam: that recursion is the forward
// sweep itself with r = -(diag/w) lam, so the adjoint solve runs the forward
// Jacobi kernel.  The RHS F(u) = -(u.grad)u + nu lap u is transposed in
// gather form at the stored forward state (reads within two cells, so the
// differentiable grid has ghost width 2); dL/dnu is accumulated in FP64 with
// a fixed-order reduction (no atomics: the result is deterministic).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cfd_internal.h"
#include "tiles.cuh"

namespace cfd {
namespace {

__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }


struct F3 {
  const float* p;
  int py;
  long long pz;
  __device__ __forceinline__ float operator()(int i, int j, int k) const {
    return ldg(p + (long long)k * pz + (long long)j * py + i);
  }
};

constexpr int kTY = 8, kZC = 16;

// lam_p2 = lam_p + c_dt D(lam_u); writes b_1 = lam_p2 into P and the
// Jacobi right-hand side R = -(diag/w) lam_p2.
__global__ void __launch_bounds__(32 * kTY) k_adj_proj(Launch L, AdjSet lam, int lp, float c_dt,
                                                       float r_scale, int p_out, int r_out) {
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, kTY, kZC);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, kTY, kZC, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const float* base_f = reinterpret_cast<const float*>(L.base);
    const F3 u{base_f + B.org[lam.a[0]], B.py, B.pz}, v{base_f + B.org[lam.a[1]], B.py, B.pz},
        w{base_f + B.org[lam.a[2]], B.py, B.pz}, p{base_f + B.org[lp], B.py, B.pz};
    float* P = reinterpret_cast<float*>(L.base) + B.org[p_out];
    float* R = reinterpret_cast<float*>(L.base) + B.org[r_out];
    const int k1 = min(k0 + kZC, B.n[2]);
    for (int k = k0; k < k1; ++k) {
      const float d = (u(i, j, k) - u(i - 1, j, k)) * L.ih[0] + (v(i, j, k) - v(i, j - 1, k)) * L.ih[1] +
                      (w(i, j, k) - w(i, j, k - 1)) * L.ih[2];
      const float l = p(i, j, k) + c_dt * d;
      const long long o = (long long)k * B.pz + (long long)j * B.py + i;
      P[o] = l;
      R[o] = r_scale * l;
    }
  }
}

// lam_W = lam_u + coef G b_K (coef = (w/diag)/c_dt);  lam_p = b_{K+1} - b_K.
__global__ void __launch_bounds__(32 * kTY) k_adj_wp(Launch L, AdjSet lam, int bk, int bk1,
                                                     float coef, AdjSet wout, int lp) {
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, kTY, kZC);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, kTY, kZC, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const float* bf = reinterpret_cast<const float*>(L.base);
    const F3 b{bf + B.org[bk], B.py, B.pz}, b1{bf + B.org[bk1], B.py, B.pz};
    const int k1 = min(k0 + kZC, B.n[2]);
    for (int k = k0; k < k1; ++k) {
      const long long o = (long long)k * B.pz + (long long)j * B.py + i;
      const float bc = b(i, j, k);
      const float g[3] = {(b(i + 1, j, k) - bc) * L.ih[0], (b(i, j + 1, k) - bc) * L.ih[1],
                          (b(i, j, k + 1) - bc) * L.ih[2]};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float l = ldg(bf + B.org[lam.a[c]] + o);
        reinterpret_cast<float*>(L.base)[B.org[wout.a[c]] + o] = l + coef * g[c];
      }
      reinterpret_cast<float*>(L.base)[B.org[lp] + o] = b1(i, j, k) - bc;
    }
  }
}

// Transposed RHS at state y for target component T at interior point (i,j,k):
//   adj_T = nu lap(lam_T)
//         + sum_d [lam_T(+d) vel_d(+d) - lam_T(-d) vel_d(-d)] / (2 h_d)
//         - lam_T (y_T(+T) - y_T(-T)) / (2 h_T)
//         - sum_{c != T} sum_{a in {0,-1}, b in {0,+1}} 1/4 lam_c(x) (y_c(x+T) - y_c(x-T)) / (2 h_T),
//           x = (i,j,k) + a e_c + b e_T,
// where vel_d(x) at a T-point is y_T(x) for d == T and otherwise the
// 4-point average of y_d over x + {0,1} e_T + {-1,0} e_d.
template <int TT>
__device__ __forceinline__ float adj_rhs_comp(const F3 (&lam)[3], const F3 (&y)[3], int i, int j,
                                              int k, const float (&ih)[3], const float (&ih2)[3],
                                              float nu, double& lap_dot) {
  auto at = [&](const F3& f, int d1, int o1, int d2, int o2, int d3, int o3) -> float {
    int q[3] = {i, j, k};
    q[d1] += o1;
    q[d2] += o2;
    q[d3] += o3;
    return f(q[0], q[1], q[2]);
  };
  const float l0 = lam[TT](i, j, k);
  float adj = 0.f, lapy = 0.f;
  const float y0 = y[TT](i, j, k);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float lp = at(lam[TT], d, 1, d, 0, d, 0), lm = at(lam[TT], d, -1, d, 0, d, 0);
    adj += nu * (lp - 2.f * l0 + lm) * ih2[d];
    lapy += (at(y[TT], d, 1, d, 0, d, 0) - 2.f * y0 + at(y[TT], d, -1, d, 0, d, 0)) * ih2[d];
    float vp, vm;
    if (d == TT) {
      vp = at(y[TT], d, 1, d, 0, d, 0);
      vm = at(y[TT], d, -1, d, 0, d, 0);
    } else {
      // vel_d at the T-point x = (i,j,k) +/- e_d
      vp = 0.25f * ((at(y[d], d, 0, TT, 0, d, 0) + at(y[d], d, 0, TT, 1, d, 0)) +
                    (at(y[d], d, 1, TT, 0, d, 0) + at(y[d], d, 1, TT, 1, d, 0)));
      vm = 0.25f * ((at(y[d], d, -2, TT, 0, d, 0) + at(y[d], d, -2, TT, 1, d, 0)) +
                    (at(y[d], d, -1, TT, 0, d, 0) + at(y[d], d, -1, TT, 1, d, 0)));
    }
    adj += (lp * vp - lm * vm) * (0.5f * ih[d]);
  }
  adj -= l0 * (at(y[TT], TT, 1, TT, 0, TT, 0) - at(y[TT], TT, -1, TT, 0, TT, 0)) * (0.5f * ih[TT]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c == TT) continue;
    float s = 0.f;
#pragma unroll
    for (int a = -1; a <= 0; ++a)
#pragma unroll
      for (int b = 0; b <= 1; ++b) {
        const float lc = at(lam[c], c, a, TT, b, TT, 0);
        const float dy = at(y[c], c, a, TT, b + 1, TT, 0) - at(y[c], c, a, TT, b - 1, TT, 0);
        s += lc * dy;
      }
    adj -= 0.25f * s * (0.5f * ih[TT]);
  }
  lap_dot += (double)l0 * (double)lapy;
  return adj;
}

// The same for the conservative (flux) form.  On the periodic grid,
// summation by parts turns sum_p lam_c(p) F_c(p) (advective part) into
// sum_{c,d,q} E_cd(q) g_cd(q) with E_cd(q) = A B / 4,
// A = y_c(q) + y_c(q + e_c') (c' = d), B = y_d(q) + y_d(q + e_c) and
// g_cd(q) = (lam_c(q + e_d) - lam_c(q)) / h_d; its derivative by y_T(x) is
//   1/4 sum_d [B_Td(x) g_Td(x) + B_Td(x - e_d) g_Td(x - e_d)]   (through A)
// + 1/4 sum_c [A_cT(x) g_cT(x) + A_cT(x - e_c) g_cT(x - e_c)]   (through B),
// B_Td(q) = y_d(q) + y_d(q + e_T), A_cT(q) = y_c(q) + y_c(q + e_T).
template <int TT>
__device__ __forceinline__ float adj_rhs_comp_flux(const F3 (&lam)[3], const F3 (&y)[3], int i,
                                                   int j, int k, const float (&ih)[3],
                                                   const float (&ih2)[3], float nu,
                                                   double& lap_dot) {
  auto at = [&](const F3& f, int d1, int o1, int d2, int o2) -> float {
    int q[3] = {i, j, k};
    q[d1] += o1;
    q[d2] += o2;
    return f(q[0], q[1], q[2]);
  };
  const float l0 = lam[TT](i, j, k);
  const float y0 = y[TT](i, j, k);
  float adj = 0.f, lapy = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float lp = at(lam[TT], d, 1, d, 0), lm = at(lam[TT], d, -1, d, 0);
    adj += nu * (lp - 2.f * l0 + lm) * ih2[d];
    lapy += (at(y[TT], d, 1, d, 0) - 2.f * y0 + at(y[TT], d, -1, d, 0)) * ih2[d];
    // through A (c = T): q = x and q = x - e_d
    const float bx = at(y[d], d, 0, TT, 0) + at(y[d], TT, 1, d, 0);
    const float bm = at(y[d], d, -1, TT, 0) + at(y[d], d, -1, TT, 1);
    adj += 0.25f * (bx * (lp - l0) + bm * (l0 - lm)) * ih[d];
    // through B (d = T, here c = d): q = x and q = x - e_c
    const float ax = at(y[d], d, 0, TT, 0) + at(y[d], TT, 1, d, 0);
    const float am = at(y[d], d, -1, TT, 0) + at(y[d], d, -1, TT, 1);
    const float gx = at(lam[d], TT, 1, d, 0) - at(lam[d], TT, 0, d, 0);
    const float gm = at(lam[d], d, -1, TT, 1) - at(lam[d], d, -1, TT, 0);
    adj += 0.25f * (ax * gx + am * gm) * ih[TT];
  }
  lap_dot += (double)l0 * (double)lapy;
  return adj;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// out_T = [acc ? out_T : 0] + b lam_T + c adj_T;  x_T = a lam_T (if x set);
// per-CTA FP64 partial of <lam, lap y> into partials[blockIdx.x].
template <bool FLUX>
__global__ void __launch_bounds__(32 * kTY) k_adj_stage(Launch L, AdjSet lam_set, Ptr3 ys,
                                                        AdjSet out_set, int acc, float b, float c,
                                                        int has_x, AdjSet x_set, float a,
                                                        float nu, double* partials) {
  __shared__ double sh[kTY];
  const float ih[3] = {L.ih[0], L.ih[1], L.ih[2]};
  const float ih2[3] = {L.ih2[0], L.ih2[1], L.ih2[2]};
  double dot = 0.0;
  __shared__ TileTable tt;
  tile_table_build(tt, L, 32, kTY, kZC);
  int blk = L.b0;
  for (long long t = blockIdx.x;; t += gridDim.x) {
    int i0, j0, k0;
    if (!tile_locate(tt, L, t, 32, kTY, kZC, blk, i0, j0, k0)) break;
    const BlockDev& B = L.blocks[blk];
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i >= B.n[0] || j >= B.n[1]) continue;
    const float* bf = reinterpret_cast<const float*>(L.base);
    const F3 lam[3] = {{bf + B.org[lam_set.a[0]], B.py, B.pz}, {bf + B.org[lam_set.a[1]], B.py, B.pz},
                       {bf + B.org[lam_set.a[2]], B.py, B.pz}};
    const F3 y[3] = {{ys.p[0], B.py, B.pz}, {ys.p[1], B.py, B.pz}, {ys.p[2], B.py, B.pz}};
    const int k1 = min(k0 + kZC, B.n[2]);
    for (int k = k0; k < k1; ++k) {
      const long long o = (long long)k * B.pz + (long long)j * B.py + i;
      float adj[3];
      if constexpr (FLUX) {
        adj[0] = adj_rhs_comp_flux<0>(lam, y, i, j, k, ih, ih2, nu, dot);
        adj[1] = adj_rhs_comp_flux<1>(lam, y, i, j, k, ih, ih2, nu, dot);
        adj[2] = adj_rhs_comp_flux<2>(lam, y, i, j, k, ih, ih2, nu, dot);
      } else {
        adj[0] = adj_rhs_comp<0>(lam, y, i, j, k, ih, ih2, nu, dot);
        adj[1] = adj_rhs_comp<1>(lam, y, i, j, k, ih, ih2, nu, dot);
        adj[2] = adj_rhs_comp<2>(lam, y, i, j, k, ih, ih2, nu, dot);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float* op = reinterpret_cast<float*>(L.base) + B.org[out_set.a[m]] + o;
        const float l = lam[m](i, j, k);
        float v = b * l + c * adj[m];
        if (acc) v += *op;
        *op = v;
        if (has_x) reinterpret_cast<float*>(L.base)[B.org[x_set.a[m]] + o] = a * l;
      }
    }
  }
  dot = warp_sum(dot);
  const int w = threadIdx.y, ln = threadIdx.x;
  if (ln == 0) sh[w] = dot;
  __syncthreads();
  if (w == 0) {
    double s = ln < kTY ? sh[ln] : 0.0;
    s = warp_sum(s);
    if (ln == 0) partials[blockIdx.x] = s;
  }
}

// acc += coef * sum(partials[0..n)) in a fixed order (one warp).
__global__ void __launch_bounds__(32) k_nu_final(const double* partials, int n, double coef,
                                                 double* acc) {
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += 32) s += partials[q];
  s = warp_sum(s);
  if (threadIdx.x == 0) *acc += coef * s;
}

template <typename K>
unsigned grid_size(const Launch& L, K kern, int threads, long long tiles, int cap_parts) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0) != cudaSuccess || occ < 1) occ = 1;
  long long cap = (long long)L.sms * occ;
  if (cap_parts > 0 && cap > cap_parts) cap = cap_parts;
  return (unsigned)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

}  // namespace

cudaError_t launch_adj_proj(const Launch& L, const AdjSet& lam, int lp, float c_dt, float r_scale,
                            int p_out, int r_out) {
  const long long tiles = count_tiles(L, 32, kTY, kZC);
  k_adj_proj<<<grid_size(L, k_adj_proj, 32 * kTY, tiles, 0), dim3(32, kTY), 0, L.stream>>>(
      L, lam, lp, c_dt, r_scale, p_out, r_out);
  return cudaGetLastError();
}

cudaError_t launch_adj_wp(const Launch& L, const AdjSet& lam, int bk, int bk1, float coef,
                          const AdjSet& wout, int lp) {
  const long long tiles = count_tiles(L, 32, kTY, kZC);
  k_adj_wp<<<grid_size(L, k_adj_wp, 32 * kTY, tiles, 0), dim3(32, kTY), 0, L.stream>>>(
      L, lam, bk, bk1, coef, wout, lp);
  return cudaGetLastError();
}

cudaError_t launch_adj_stage(const Launch& L, const AdjSet& lam, const Ptr3& y, const AdjSet& out,
                             int acc, float b, float c, int has_x, const AdjSet& x, float a,
                             float nu, double* partials, int nparts, double* nu_acc,
                             double nu_coef, bool flux) {
  const long long tiles = count_tiles(L, 32, kTY, kZC);
  auto kern = flux ? k_adj_stage<true> : k_adj_stage<false>;
  const unsigned grid = grid_size(L, kern, 32 * kTY, tiles, nparts);
  kern<<<grid, dim3(32, kTY), 0, L.stream>>>(L, lam, y, out, acc, b, c, has_x, x, a, nu, partials);
  k_nu_final<<<1, 32, 0, L.stream>>>(partials, (int)grid, nu_coef, nu_acc);
  return cudaGetLastError();
}

}  // namespace cfd
