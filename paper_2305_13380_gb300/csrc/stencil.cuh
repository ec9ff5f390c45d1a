// stencil.cuh -- the 27-cell neighbourhood of a target cell on the uniform
// periodic grid (Sec. 2.1: every neighbour of a particle lies in its own cell
// or one of the 26 adjacent cells, because cells are at least H wide), and the
// warp-cooperative staging of those cells' particles into shared memory.
#pragma once
#include "sph_internal.cuh"

namespace sphk {

// Lane k < 27 of a warp describes neighbour k = (dx+1) + 3 (dy+1) + 9 (dz+1):
// its sorted range and the offset of its particles' cell-relative positions
// when seen from the target cell (a periodic image is just another offset).
struct NbLane {
  int32_t start, len;
  float ox, oy, oz;
};

__device__ __forceinline__ NbLane neighbour_lane(int lane, int32_t cell_base, int32_t cx, int32_t cy,
                                                 int32_t cz, int32_t nc, float cell,
                                                 const int32_t* __restrict__ cell_start) {
  NbLane r;
  r.start = 0;
  r.len = 0;
  r.ox = r.oy = r.oz = 0.0f;
  if (lane < 27) {
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    int32_t nx = cx + dx, ny = cy + dy, nz = cz + dz;
    nx += nx < 0 ? nc : 0;
    nx -= nx >= nc ? nc : 0;
    ny += ny < 0 ? nc : 0;
    ny -= ny >= nc ? nc : 0;
    nz += nz < 0 ? nc : 0;
    nz -= nz >= nc ? nc : 0;
    const int32_t nbc = cell_base + nx + nc * (ny + nc * nz);
    r.start = cell_start[nbc];
    r.len = cell_start[nbc + 1] - r.start;
    r.ox = (float)dx * cell;
    r.oy = (float)dy * cell;
    r.oz = (float)dz * cell;
  }
  return r;
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Copies the virtual source range [v0, v0 + cap) of the concatenation of the
// 27 neighbour cells into shared memory through `put(slot, j, ox, oy, oz)`.
// Returns the number of sources staged.  Warp-collective.
template <class Put>
__device__ __forceinline__ int stage_sources(int v0, int cap, const NbLane& nb, int lane, Put put) {
  int cum = 0;
#pragma unroll 1
  for (int k = 0; k < 27; ++k) {
    const int32_t st = __shfl_sync(0xffffffffu, nb.start, k);
    const int32_t len = __shfl_sync(0xffffffffu, nb.len, k);
    const float ox = __shfl_sync(0xffffffffu, nb.ox, k);
    const float oy = __shfl_sync(0xffffffffu, nb.oy, k);
    const float oz = __shfl_sync(0xffffffffu, nb.oz, k);
    const int lo = max(v0, cum), hi = min(v0 + cap, cum + len);
    for (int v = lo + lane; v < hi; v += 32) put(v - v0, st + (v - cum), ox, oy, oz);
    cum += len;
  }
  __syncwarp();
  return min(cum, v0 + cap) - v0;
}

}  // namespace sphk
