// Inline-PTX building blocks of the TMA-staged kernels: mbarrier set-up,
// arrival and bounded waits, and 3-D tiled bulk tensor loads into shared
// memory.  Every wait is bounded by kWaitLimitNs of %globaltimer; a wait
// that gives up returns false and the caller sets the device error flag.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "cfd_internal.h"

namespace cfd {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// try_wait with a suspend-time hint: the waiting thread sleeps until the
// phase completes or about 100 us have passed, instead of polling
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(100000)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait_sleep(bar, parity))
    if (gtimer() - t0 > kWaitLimitNs) return false;
  return true;
}
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait_sleep(bar, parity))
    if (gtimer() - t0 > kWaitLimitNs) return false;
  return true;
}
// The same bounded wait with the polling loop out of line (less code in
// kernels that wait several times per plane; the call raises the register
// count of kernels that run two CTAs per SM, which use mbar_wait).
__device__ __forceinline__ bool mbar_wait_split(uint32_t bar, uint32_t parity) {
  return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Position in the ring: stage index and phase parity of plane f.
template <int S>
struct Ring {
  int s;
  uint32_t ph;
  __device__ __forceinline__ explicit Ring(unsigned f) : s((int)(f % S)), ph((f / S) & 1u) {}
  __device__ __forceinline__ void next() {
    if (++s == S) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// The device error flag as a launch finds it: thread (0, 0) copies it to
// shared memory before the CTA's first barrier; after that barrier every
// thread tests the copy.  A launch that finds it set (a bounded wait of an
// earlier launch gave up, and results are undefined until memory is bound
// again) does no work, so a failed solve costs one wait limit, not one per
// launch.
__device__ __forceinline__ void flag_at_start(const Launch& L, int& shared_copy) {
  if (threadIdx.x == 0 && threadIdx.y == 0) shared_copy = *reinterpret_cast<volatile int*>(L.err_flag);
}

// The tile counter of a launch: a word of the grid's flag area (zeroed when
// memory is bound), 128 bytes after the device error flag.
__device__ __forceinline__ unsigned* tile_counter(const Launch& L) {
  return reinterpret_cast<unsigned*>(L.err_flag) + 32;
}

// Tiles claimed at run time by warp-specialised kernels: lane 0 of the
// producer warp takes the next tile number from a counter in device memory
// and hands it to the CTA's other warps through a four-slot queue guarded by
// mbarriers (count 1).  Every CTA ends on one claim past the last tile, so
// atomicInc with wrap = tiles + CTAs - 1 leaves the counter at 0 for the
// next launch.  An SM that shares its issue slots with other work takes
// fewer tiles instead of holding up the launch.
struct TileQueue {
  unsigned long long* bar;  // 4 mbarriers
  unsigned* slot;           // 4 tile numbers
  __device__ __forceinline__ void init() const {
#pragma unroll
    for (int s = 0; s < 4; ++s) mbar_init(smem_u32(&bar[s]), 1);
  }
  // producer warp, every lane: the k-th tile of this CTA
  __device__ __forceinline__ unsigned claim(unsigned k, unsigned* ctr, unsigned wrap,
                                            int lane) const {
    unsigned v = 0;
    if (lane == 0) {
      v = atomicInc(ctr, wrap);
      slot[k & 3] = v;
      mbar_arrive(smem_u32(&bar[k & 3]));
    }
    return __shfl_sync(0xffffffffu, v, 0);
  }
  // the other warps: false if the bounded wait gave up
  __device__ __forceinline__ bool take(unsigned k, long long& t) const {
    if (!mbar_wait_split(smem_u32(&bar[k & 3]), (k >> 2) & 1u)) return false;
    t = slot[k & 3];
    return true;
  }
};

}  // namespace
}  // namespace cfd
