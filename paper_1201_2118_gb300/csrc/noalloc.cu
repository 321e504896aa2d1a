// Allocation-free FP64 velocity reduction.
//
// Some callers cannot allocate device memory at the moment they want these
// diagnostics: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not a capturable operation), host frameworks whose
// device memory is owned by their own pool allocator, and monitoring hooks
// in a time loop that must not trigger the device-wide synchronisation a
// cudaMalloc/cudaFree can cause.  This variant of the reduction kernel
// therefore keeps its per-plane partial sums in a fixed static device array
// of this library instead of in caller- or library-allocated scratch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gb300cfd.h"
#include "ffloat.cuh"

namespace {

// One slot of 4 doubles per z-plane: at most kMaxPlanes planes (128 KiB).
// Every GPU that loads the library holds this array until process exit.
constexpr int kMaxPlanes = 4096;
__device__ __align__(256) double g_plane_partials[kMaxPlanes * 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_partials_addr[kMaxDevices] = {};

thread_local std::string t_noalloc_err;

__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Sum |u|^2, max |u_d|, max |D u| and the non-finite count of one z-plane per
// CTA (the grid reduction's float-float per-cell arithmetic, each cell's
// |u|^2 added to an FP64 sum), written to
// partials[4 z .. 4 z + 3].  Every slot 0..nz-1 is written by every call, so
// the static array needs no clearing between calls.
template <typename T>
__global__ void __launch_bounds__(256) k_plane_partials(const T* u, const T* v, const T* w,
                                                        int nx, int ny, long long py,
                                                        long long pz, float ihx, float ihy,
                                                        float ihz, double* partials) {
  __shared__ double sh[8][4];
  const int k = blockIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  const float ih[3] = {ihx, ihy, ihz};
  float umax = 0.f;
  cfd::FF dmax = {0.f, 0.f};
  int bad = 0;
  // 64-bit cell index: nx * ny may come within 256 of 2^31 - 1
  const long long cells = (long long)nx * ny;
  for (long long c = threadIdx.x; c < cells; c += 256) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    const long long o = (long long)k * pz + (long long)j * py + i;
    const float x[3] = {ld(u + o), ld(v + o), ld(w + o)};
    const float xm[3] = {ld(u + o - 1), ld(v + o - py), ld(w + o - pz)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      umax = fmaxf(umax, fabsf(x[d]));
      bad += !isfinite(x[d]);
    }
    cfd::FF sq = {0.f, 0.f}, div;
    cfd::ff_cell(x, xm, ih, sq, div);
    a[0] += cfd::ff_to_double(sq);
    div = cfd::ff_abs(div);
    if (cfd::ff_gt(div, dmax)) dmax = div;
  }
  a[1] = umax;
  a[2] = cfd::ff_to_double(dmax);
  a[3] = bad;
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
  a[0] = wsum(a[0]);
  a[1] = wmax(a[1]);
  a[2] = wmax(a[2]);
  a[3] = wsum(a[3]);
  if (ln == 0)
    for (int e = 0; e < 4; ++e) sh[wid][e] = a[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < 8; ++q) {
      s[0] += sh[q][0];
      s[1] = fmax(s[1], sh[q][1]);
      s[2] = fmax(s[2], sh[q][2]);
      s[3] += sh[q][3];
    }
    for (int e = 0; e < 4; ++e) partials[4 * k + e] = s[e];
  }
}

// Fixed-order pass over the nz plane slots: out = {sum, max, max, count}.
__global__ void __launch_bounds__(32) k_planes_final(const double* partials, int nz,
                                                     double h3half, double* out) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int z = threadIdx.x; z < nz; z += 32) {
    a[0] += partials[4 * z];
    a[1] = fmax(a[1], partials[4 * z + 1]);
    a[2] = fmax(a[2], partials[4 * z + 2]);
    a[3] += partials[4 * z + 3];
  }
  a[0] = wsum(a[0]);
  a[1] = wmax(a[1]);
  a[2] = wmax(a[2]);
  a[3] = wsum(a[3]);
  if (threadIdx.x == 0) {
    out[0] = a[0] * h3half;
    out[1] = a[1];
    out[2] = a[2];
    out[3] = a[3];
  }
}

cfd_status nfail(cfd_status s, const std::string& m) {
  t_noalloc_err = m;
  return s;
}

// Device address of the static array on the current device (looked up once
// per device, with that device current).
cfd_status partials_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(CFD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(CFD_EUNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_plane_partials);
    if (e != cudaSuccess)
      return nfail(CFD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return CFD_OK;
}

}  // namespace

extern "C" const char* cfd_noalloc_last_error(void) { return t_noalloc_err.c_str(); }

extern "C" cfd_status cfd_reduce_velocity_noalloc(const void* u, const void* v, const void* w,
                                                  int dtype, const int dims[3],
                                                  long long pitch_y, long long pitch_z,
                                                  const double h[3], double* out_dev,
                                                  void* stream) {
  if (!u || !v || !w || !dims || !h || !out_dev) return nfail(CFD_EINVAL, "null argument");
  if (dtype < CFD_F32 || dtype > CFD_F16) return nfail(CFD_EINVAL, "unknown dtype");
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return nfail(CFD_EINVAL, "dims must be >= 1");
  if (dims[2] > kMaxPlanes)
    return nfail(CFD_EINVAL, "nz = " + std::to_string(dims[2]) + " exceeds the static scratch of " +
                                 std::to_string(kMaxPlanes) + " planes");
  if ((long long)dims[0] * dims[1] > (1LL << 31) - 1) return nfail(CFD_EINVAL, "plane too large");
  if (pitch_y < dims[0] || pitch_z < pitch_y * dims[1]) return nfail(CFD_EINVAL, "pitches too small");
  for (int d = 0; d < 3; ++d)
    if (!(h[d] > 0.0)) return nfail(CFD_EINVAL, "h must be > 0");
  double* partials = nullptr;
  cfd_status s = partials_on_current_device(&partials);
  if (s != CFD_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float ih[3] = {(float)(1.0 / h[0]), (float)(1.0 / h[1]), (float)(1.0 / h[2])};
  const int nz = dims[2];
  switch (dtype) {
    case CFD_F32:
      k_plane_partials<float><<<nz, 256, 0, st>>>(
          static_cast<const float*>(u), static_cast<const float*>(v), static_cast<const float*>(w),
          dims[0], dims[1], pitch_y, pitch_z, ih[0], ih[1], ih[2], partials);
      break;
    case CFD_BF16:
      k_plane_partials<__nv_bfloat16><<<nz, 256, 0, st>>>(
          static_cast<const __nv_bfloat16*>(u), static_cast<const __nv_bfloat16*>(v),
          static_cast<const __nv_bfloat16*>(w), dims[0], dims[1], pitch_y, pitch_z, ih[0], ih[1],
          ih[2], partials);
      break;
    default:
      k_plane_partials<__half><<<nz, 256, 0, st>>>(
          static_cast<const __half*>(u), static_cast<const __half*>(v),
          static_cast<const __half*>(w), dims[0], dims[1], pitch_y, pitch_z, ih[0], ih[1], ih[2],
          partials);
      break;
  }
  k_planes_final<<<1, 32, 0, st>>>(partials, nz, 0.5 * h[0] * h[1] * h[2], out_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(CFD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return CFD_OK;
}
