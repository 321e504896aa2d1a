// Internal types shared by the runtime and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cfd {

constexpr int kNumArrays = 16;   // matches CFD_NUM_ARRAYS
constexpr int kMaxBlocks = 512;
constexpr int kAlignBytes = 128; // interior x = 0 of every row, and row pitch
constexpr int kMaxGhost = 2;

// Array ids (same numbering as cfd_array).
enum Arr {
  A_U = 0, A_V = 1, A_W = 2, A_P = 3,
  A_WU = 4, A_WV = 5, A_WW = 6,
  A_U1 = 7, A_V1 = 8, A_W1 = 9,
  A_P2 = 10, A_R = 11,
  A_LU = 12, A_LV = 13, A_LW = 14, A_LP = 15   // adjoint state (dL/du, dL/dp)
};

// Field kind of each array: 0 u, 1 v, 2 w (velocity components), 3 scalar.
__host__ __device__ inline int array_kind(int a) {
  if (a == A_P || a == A_P2 || a == A_R || a == A_LP) return 3;
  if (a < 3) return a;
  if (a >= A_LU) return a - A_LU;
  return (a - 4) % 3;
}

enum Bc { BC_PERIODIC = 0, BC_WALL = 1 };

// One grid component (block) as the kernels see it.
struct BlockDev {
  int n[3];                    // interior cells
  int py;                      // row pitch (elements)
  long long pz;                // plane pitch (elements)
  long long org[kNumArrays];   // element offset of interior (0,0,0) per array
  int nbr[6];                  // neighbour block per face (self if periodic single block)
  int bc[6];                   // Bc per face
  float wall[6][3];            // wall velocity per face
};

static_assert(sizeof(BlockDev) % 8 == 0, "the block table is copied as words");

// What every launch needs.
struct Launch {
  const BlockDev* blocks;      // device table (all blocks)
  int b0;                      // first block this launch covers
  int nblocks;                 // blocks b0 .. b0 + nblocks - 1
  void* base;                  // arena base (arrays addressed by element offsets)
  int dtype;                   // 0 f32, 1 bf16, 2 f16
  int ghost;
  float ih[3];                 // 1/h
  float ih2[3];                // 1/h^2
  int* err_flag;               // device error word
  cudaStream_t stream;
  int sms;                     // multiprocessor count
  // host copy of block dims for grid sizing
  const int (*hn)[3];
};

// Kernel variants (autotuned).
//   kind 0: register/shuffle sweep (any block size, plain loads)
//   kind 1: TMA-staged sweep (tensor maps per block, S-stage mbarrier ring)
//   kind 2: direct sweep (no shared memory; zc = z-planes per CTA, TZ)
//   kind 3: cp.async-staged sweep (per-thread async copies, S-stage ring)
//   kind 7: warp-specialised TMA sweep (producer warp, empty/full mbarriers,
//           no CTA barrier per plane)
//   kind 5: two fused sweeps per launch (temporal blocking, single block,
//           nx % 128 == 0, ny % ty == 0); odd counts end with one kind-0 sweep
//   kind 9: two sweeps per launch, warp-specialised TMA, tiles claimed from a
//           counter (single block with walls on all six faces, or the
//           periodic form with two ghost layers, block sets included); odd
//           counts end with one kind-0 sweep
struct JacobiCfg { int kind, vx, ty, zc, stages; };
// Point kernels: rows per CTA (32 x ty threads) and z chunk; the RHS + stage
// kernel either reads neighbours through L1 (tile_tz = 0) or from a
// shared-memory box of 32 x 8 x tile_tz cells plus halo (tile_tz = 2 or 4).
struct StencilCfg { int ty, zc, tile_tz; };

// One array as a 3D tensor for TMA: start of the allocation, row length
// (the row pitch, elements), rows per plane and planes.
struct TmaArray { void* ptr; long long row_elems, rows, planes; };
constexpr int kTmaMapBytes = 128;

// Encodes the Jacobi tensor maps (per block: P, P2, R) for config c into
// out_host (narrays x 128 bytes).  False if the driver entry point or an
// encoding fails.
bool encode_jacobi_maps(void* out_host, const TmaArray* arrays, int narrays, int dtype,
                        const JacobiCfg& c);
cudaError_t launch_jacobi_tma(const Launch& L, const JacobiCfg& c, const void* maps_dev,
                              int src_slot, int dst, float omega);
// Interior of one array of the launch's (single) block <-> a compact
// (nz, ny, nx) buffer in device memory: to_compact 0 scatters the buffer
// into the array, 1 gathers the array into the buffer.
cudaError_t launch_pack(const Launch& L, int arr, void* compact, int to_compact);
// The same copy on a few CTAs (one per eight SMs) with sixteen 16-byte
// transfers in flight per thread: for page-locked host buffers, so that a
// transfer keeps the host link busy without taking the SMs from other work.
// Needs nx a multiple of the 16-byte vector and a 16-byte aligned buffer
// (returns cudaErrorInvalidValue otherwise; the caller falls back).
cudaError_t launch_pack_narrow(const Launch& L, int arr, void* compact, int to_compact);
// One CTA waits (bounded) on an mbarrier that nothing completes; sets the
// device error flag when the wait runs out (failure-detection self-test).
cudaError_t launch_wait_probe(const Launch& L, int form);

// Two sweeps per launch (kind 9), src -> dst; single block, walls on all
// faces, or (periodic) all faces periodic with ghost width >= 2, src's two
// ghost layers and R's first filled before the launch, dst's ghosts not
// written.
cudaError_t launch_jacobi2_ws(const Launch& L, const JacobiCfg& c, const void* maps_dev,
                              int src_slot, int dst, float omega, bool periodic);

long long count_tiles(const Launch& L, int tx, int ty, int tz);

// Adjoint kernels (FP32 storage, single periodic block, order 2, either
// advection form).
struct AdjSet { int a[3]; };
struct Ptr3 { const float* p[3]; };  // interior origins of stored forward states
cudaError_t launch_adj_proj(const Launch& L, const AdjSet& lam, int lp, float c_dt, float r_scale,
                            int p_out, int r_out);
cudaError_t launch_adj_wp(const Launch& L, const AdjSet& lam, int bk, int bk1, float coef,
                          const AdjSet& wout, int lp);
cudaError_t launch_adj_stage(const Launch& L, const AdjSet& lam, const Ptr3& y, const AdjSet& out,
                             int acc, float b, float c, int has_x, const AdjSet& x, float a,
                             float nu, double* partials, int nparts, double* nu_acc,
                             double nu_coef, bool flux);

// One piece of a block's ghost shell, built on the host, from the box of
// one direction (dx, dy, dz) around block dst (g layers deep along the axes
// where d is non-zero, the block's extent elsewhere), copied from block src.
// ax = {inner axis, row axis j, plane axis k}; per those axes: destination
// origin d0 (ghost index in dst), source origin s0 and step st in src (+1:
// the shifted copy across a periodic or block-to-block face, -1: the mirror
// image at a wall).  wface[a] is the wall face met along axis a (x, y, z),
// -1 if none; the wall rules compose in that axis order.  The piece is the
// inner-axis range i0 .. i0 + ni - 1 (ni <= kGhostItemCells) of rows
// rj0 .. rj0 + nrows - 1 of plane rk; a warp lays its lanes out as 2^sh
// columns by 32 >> sh rows and covers it in at most eight steps (passes
// over the row range: P = ni / 2^sh rounded up).
constexpr int kGhostItemCells = 256;
struct GhostItem {
  int dst, src;
  int ax[3];
  int d0[3], s0[3], st[3];
  int wface[3];
  int i0, ni, rj0, nrows, rk;
  int sh, passes;
};

cudaError_t launch_ghost(const Launch& L, const int* arrays, int narr, const GhostItem* items,
                         int nitems);
// Momentum-advection scheme of the RHS + stage kernels: the advective form
// of order 2 or 4 (the value is the order) or the order-2 conservative
// (flux) form.  The stencil reach is scheme_halo() cells per axis.
enum : int { kSchemeAdv2 = 2, kSchemeFlux2 = 3, kSchemeAdv4 = 4 };
__host__ __device__ constexpr int scheme_halo(int scheme) { return scheme == kSchemeAdv4 ? 2 : 1; }

cudaError_t launch_stage(const Launch& L, const StencilCfg& c, int scheme, float a,
                         const int* xset, float b, const int* yset, float cdt, const int* oset,
                         float nu);
cudaError_t launch_divergence(const Launch& L, const StencilCfg& c, const int* wset,
                              float inv_cdt, int r_arr);
cudaError_t launch_jacobi(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                          float omega);
cudaError_t launch_jacobi2(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                           float omega);
cudaError_t launch_jacobi_async(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                                float omega);
cudaError_t launch_jacobi_direct(const Launch& L, const JacobiCfg& c, int src, int dst, int r_arr,
                                 float omega);
cudaError_t launch_project(const Launch& L, const StencilCfg& c, const int* wset, int p_arr,
                           float cdt, const int* oset);
cudaError_t launch_copy(const Launch& L, const StencilCfg& c, int src, int dst);

// Multigrid grid transfers (FP32 storage).  A view is the interior origin of
// one array of one level with its pitches and interior dims.
struct MgView { float* o; int n[3]; int py; long long pz; };
// coarse_r = mean over each coarse cell's 8 children of (fine_r - L fine_p).
cudaError_t launch_mg_restrict(cudaStream_t s, const MgView& fine_p, const float* fine_r,
                               const MgView& coarse_r, const float ih2_fine[3]);
// fine_p += trilinear interpolation of coarse_e (ghosts current) at the fine
// centres; the face ghost images of fine_p (periodic or mirror per axis) are
// written too (edges and corners are not).
cudaError_t launch_mg_prolong(cudaStream_t s, const MgView& fine_p, const MgView& coarse_e,
                              const int periodic[3]);

// The bottom of a V-cycle in one CTA: levels 0 .. levels - 1 of it (level 0
// = the first level with at most kMgBottomCells cells) live in shared
// memory.  r_in is level 0's R (from the restriction above it); p_out
// receives level 0's correction with its first ghost layer (edges and
// corners included).
constexpr int kMgBottomLevels = 12;
constexpr int kMgBottomCells = 8192;
struct MgBottom {
  int levels;
  int n[kMgBottomLevels][3];
  float c[kMgBottomLevels][3];     // 1/h^2 per axis
  float inv_diag[kMgBottomLevels];
  int per[3];                      // axis periodic (else walls, zero-gradient ghosts)
  int nu1, nu2, ncoarse;
  float omega;
  MgView r_in, p_out;
};
size_t mg_bottom_smem(const MgBottom& b);
// Raises the bottom kernel's shared-memory limit (once per process, before
// any stream capture that may launch it).
cudaError_t prepare_mg_bottom();
cudaError_t launch_mg_bottom(cudaStream_t s, const MgBottom& b);

// FP64 reductions: per-CTA partials into 'partials' (nparts x 4 doubles),
// then a one-CTA fixed-order pass into 'out' (4 doubles).
// mode 0: velocity set (sum |u|^2, max |u_d|, max |D u|, non-finite count)
// mode 1: pressure residual (sum (L p - r)^2, -, -, non-finite count)
cudaError_t launch_reduce(const Launch& L, int mode, const int* set, int p_arr, int r_arr,
                          double* partials, int nparts, double* out);

}  // namespace cfd
