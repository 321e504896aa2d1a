// Flattened tile list over the blocks of one launch.
//
// Tiles are numbered block by block (x fastest, then y, then z chunks).  A
// CTA first builds, in shared memory, the prefix sums of the tile counts of
// the blocks this launch covers (one thread per block), then maps a tile
// number to (block, tile origin) by binary search, so a CTA never walks the
// block table with a chain of dependent global loads.
#pragma once

#include "cfd_internal.h"

namespace cfd {

struct TileTable {
  int start[kMaxBlocks + 1];  // start[b] = first tile of block b0 + b
};

__device__ __forceinline__ int tiles_cdiv(int a, int b) { return (a + b - 1) / b; }

// All threads of the CTA must call this (it synchronises).
__device__ __forceinline__ void tile_table_build(TileTable& tt, const Launch& L, int tx, int ty,
                                                 int tz) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  for (int b = tid; b < L.nblocks; b += nthr) {
    const BlockDev& B = L.blocks[L.b0 + b];
    tt.start[b + 1] = tiles_cdiv(B.n[0], tx) * tiles_cdiv(B.n[1], ty) * tiles_cdiv(B.n[2], tz);
  }
  __syncthreads();
  if (tid == 0) {
    tt.start[0] = 0;
    for (int b = 0; b < L.nblocks; ++b) tt.start[b + 1] += tt.start[b];
  }
  __syncthreads();
}

// Tile t -> block index (absolute) and tile origin; false past the end.
__device__ __forceinline__ bool tile_locate(const TileTable& tt, const Launch& L, long long t,
                                            int tx, int ty, int tz, int& b, int& i0, int& j0,
                                            int& k0) {
  if (t >= tt.start[L.nblocks]) return false;
  int lo = 0, hi = L.nblocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tt.start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  b = L.b0 + lo;
  const BlockDev& B = L.blocks[b];
  const int nxT = tiles_cdiv(B.n[0], tx), nyT = tiles_cdiv(B.n[1], ty);
  int l = (int)(t - tt.start[lo]);
  i0 = (l % nxT) * tx;
  l /= nxT;
  j0 = (l % nyT) * ty;
  k0 = (l / nyT) * tz;
  return true;
}

}  // namespace cfd
