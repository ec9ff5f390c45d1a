// tree.cuh -- records of the nested-grid (octree) path shared by the tree
// build and the tree loop kernels.
#pragma once
#include <stdint.h>

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
// list radius as a multiple of the starting support (a Newton step that
// outgrows it sends the warp to the list-free path).
constexpr int kTreeTpp = 4;
constexpr int kTreeList = 32;
constexpr int kTreeListRegion = 32;
constexpr float kTreeListReach = 1.1f;

}  // namespace sphk
