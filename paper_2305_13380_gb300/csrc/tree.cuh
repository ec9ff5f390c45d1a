// tree.cuh -- records of the nested-grid (octree) path shared by the tree
// build and the tree loop kernels.
#pragma once
#include <stdint.h>

#include "sph_internal.cuh"

namespace sphk {

// Depth of the Morton order below a top cell: 2^10 = 1024 sub-cells per side.
constexpr int kTreeDepth = 10;
constexpr int kTreeFine = 1 << kTreeDepth;

// A target group: the particles of one cell at one level, targets
// [start, next group's start) in target order; the cell has side
// cell / 2^depth and integer position (lx, ly, lz) (in units of its side)
// inside top cell `cell` (global cell id).
struct TreeLeaf {
  int32_t start;
  int32_t depth;
  int32_t cell;
  int32_t lx, ly, lz;
  int32_t pad;
};

// One of the 27 neighbour cells of a group: source-order range [lo, hi) and the
// periodic shift of each axis (2 bits each, value + 1 in {0, 1, 2}).
struct TreeRange {
  int32_t lo, hi;
  int32_t shift;
  int32_t pad;
};

// Tree loops: lanes per target, list entries kept per (target, lane), and the
// list radius as a multiple of the starting support (a target whose support
// outgrows it is solved by the per-target kernel).  A reach just above the
// starting support keeps the lists (and the force pairs read from them) short;
// measured on the 2M clustered box with the per-target kernel: 1.01-1.03
// within 1 % of each other, 1.05 10 % and 1.1 15 % slower per step, 1.0 (every
// growing support queued) four times slower.
#ifndef SPH_TREE_LIST
#define SPH_TREE_LIST 32
#endif
#ifndef SPH_TREE_LIST_REACH
#define SPH_TREE_LIST_REACH 1.02f
#endif
#ifndef SPH_TREE_TPP
#define SPH_TREE_TPP 8
#endif
constexpr int kTreeTpp = SPH_TREE_TPP;  // a power of two dividing 8
constexpr int kTreeList = SPH_TREE_LIST;
constexpr int kTreeListRegion = SPH_TREE_LIST;
constexpr float kTreeListReach = SPH_TREE_LIST_REACH;

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  // 10 bits -> every third bit of 30
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}

// First index in [lo, hi) whose key >= v.
__device__ __forceinline__ int64_t lower_bound64(const uint64_t* __restrict__ a, int64_t lo, int64_t hi,
                                                 uint64_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The cell of particle key `key` at depth d, as a group record (start unused).
__device__ __forceinline__ TreeLeaf cell_at_depth(uint64_t key, int d) {
  TreeLeaf L;
  const uint32_t m = (uint32_t)(key & 0x3fffffffull);
  const int sh = kTreeDepth - d;
  L.start = 0;
  L.depth = d;
  L.cell = (int32_t)(key >> 30);
  L.lx = (int32_t)(compact3(m) >> sh);
  L.ly = (int32_t)(compact3(m >> 1) >> sh);
  L.lz = (int32_t)(compact3(m >> 2) >> sh);
  L.pad = 0;
  return L;
}

// Neighbour r (0..26, offsets (r % 3, r / 3 % 3, r / 9) - 1) of cell L at its
// depth: the source-order range of the cell of the same side there, with the
// periodic shift of each axis.
__device__ __forceinline__ TreeRange neighbour_range(const GridDev& G, const TreeLeaf& L, int r,
                                                     const uint64_t* __restrict__ skey,
                                                     const int32_t* __restrict__ cell_start) {
  const int32_t local = L.cell - G.cell_base, nc = G.n_c;
  const int32_t kx = local % nc, ky = (local / nc) % nc, kz = local / (nc * nc);
  const int d = L.depth;
  const int64_t span = (int64_t)nc << d;  // cells of this side per box side
  const int dxs = r % 3 - 1, dys = (r / 3) % 3 - 1, dzs = r / 9 - 1;
  int64_t gx = ((int64_t)kx << d) + L.lx + dxs;
  int64_t gy = ((int64_t)ky << d) + L.ly + dys;
  int64_t gz = ((int64_t)kz << d) + L.lz + dzs;
  int sx = 0, sy = 0, sz = 0;
  if (gx < 0) { gx += span; sx = -1; } else if (gx >= span) { gx -= span; sx = 1; }
  if (gy < 0) { gy += span; sy = -1; } else if (gy >= span) { gy -= span; sy = 1; }
  if (gz < 0) { gz += span; sz = -1; } else if (gz >= span) { gz -= span; sz = 1; }
  const int32_t cx = (int32_t)(gx >> d), cy = (int32_t)(gy >> d), cz = (int32_t)(gz >> d);
  const uint32_t mx = (uint32_t)(gx & ((1 << d) - 1)) << (kTreeDepth - d);
  const uint32_t my = (uint32_t)(gy & ((1 << d) - 1)) << (kTreeDepth - d);
  const uint32_t mz = (uint32_t)(gz & ((1 << d) - 1)) << (kTreeDepth - d);
  const int32_t cid = G.cell_base + cx + nc * (cy + nc * cz);
  const uint64_t base = ((uint64_t)(uint32_t)cid << 30) | (spread3(mx) | (spread3(my) << 1) | (spread3(mz) << 2));
  const uint64_t width = (uint64_t)1 << (3 * (kTreeDepth - d));
  const int64_t c0 = cell_start[cid], c1 = cell_start[cid + 1];
  TreeRange R;
  R.lo = (int32_t)lower_bound64(skey, c0, c1, base);
  R.hi = (int32_t)lower_bound64(skey, R.lo, c1, base + width);
  R.shift = (sx + 1) | ((sy + 1) << 2) | ((sz + 1) << 4);
  R.pad = 0;
  return R;
}

}  // namespace sphk
