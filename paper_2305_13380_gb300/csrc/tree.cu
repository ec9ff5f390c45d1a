// tree.cu -- nested grids for inputs whose smoothing lengths span orders of
// magnitude (Sec. 2.1 and Sec. 9.1: a top-level grid whose cells are
// recursively split into 8 children, particles stored depth-first so that
// every cell at every level is a contiguous range, and interactions taken
// between cells of the size that matches the local h).
//
// The top level is the uniform grid of cells.cu (cells >= the largest
// support).  Below each top cell the particles are ordered by the Morton code
// of their position at depth kTreeDepth (1024 sub-cells per side), giving a
// 64-bit source key (top cell id << 30 | Morton code) that the stable radix
// sort orders: "source order".  A cell at depth d is the set of keys sharing
// their top 30 - 3 (kTreeDepth - d) Morton bits, i.e. one contiguous range.
//
// Levels.  A cell holding at most n_leaf particles is not split.  Each
// particle works at its own level: the deepest depth d whose cell side is at
// least (1 + margin) H_i, stopping at a cell with at most n_leaf particles or
// at kTreeDepth.  (A rule on the largest H of a whole cell would keep a dense
// core at the coarse level of the one wide particle beside it; per particle,
// each target's 27 neighbour cells stay ~H wide.)  Targets are grouped by
// (cell at their level, level) through a second sort: "target order", with
// groups contiguous.  A group's sources are the particles of the 27 cells of
// its level around it, one source-order range each (binary search), which
// hold every particle within one cell side of the group: enough for the
// density of its targets, whose supports are at most that side.
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "tree.cuh"

namespace sphk {

// Fine coordinate on one axis: g = floor(1024 fl(fl(x n_c) / L)), clamped to
// the top cell k (the same product and quotient that define k).
__device__ __forceinline__ int32_t fine_coord(double x, double L, int32_t n_c, int32_t k) {
  const double s = __ddiv_rn(__dmul_rn(x, (double)n_c), L);
  int64_t g = (int64_t)floor(s * (double)kTreeFine);
  const int64_t lo = (int64_t)k * kTreeFine, hi = lo + kTreeFine - 1;
  g = g < lo ? lo : (g > hi ? hi : g);
  return (int32_t)g;
}

__global__ void k_tree_key(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ z, const int64_t* __restrict__ sim_offset,
                           int n_sims, const GridDev* __restrict__ grid,
                           const int32_t* __restrict__ cell_key, uint64_t* __restrict__ key64,
                           uint64_t* __restrict__ key64_copy) {
  const WarpRange wr = warp_range(n);
  SimCursor sc;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(sim_offset, n_sims, p);
    const GridDev G = grid[s];
    const int32_t c = cell_key[p];
    const int32_t local = c - G.cell_base;
    const int32_t kx = local % G.n_c, ky = (local / G.n_c) % G.n_c, kz = local / (G.n_c * G.n_c);
    const uint32_t lx = (uint32_t)(fine_coord(x[p], G.L, G.n_c, kx) - kx * kTreeFine);
    const uint32_t ly = (uint32_t)(fine_coord(y[p], G.L, G.n_c, ky) - ky * kTreeFine);
    const uint32_t lz = (uint32_t)(fine_coord(z[p], G.L, G.n_c, kz) - kz * kTreeFine);
    const uint64_t k = ((uint64_t)(uint32_t)c << 30) | (spread3(lx) | (spread3(ly) << 1) | (spread3(lz) << 2));
    key64[p] = k;
    key64_copy[p] = k;
  }
}

// Source keys in source order.
__global__ void k_tree_sorted(int64_t n, const int32_t* __restrict__ perm, const uint64_t* __restrict__ key64,
                              uint64_t* __restrict__ skey) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    skey[s] = key64[perm[s]];
}

// Level of each particle (source order) by descending from its top cell, its
// level and cell side, and its target key (top cell, Morton prefix of its cell at that
// level, level) with a copy for the sort.
__global__ void k_tree_level(int64_t n, const uint64_t* __restrict__ skey, const int32_t* __restrict__ perm,
                             const float* __restrict__ h, int n_sims,
                             const GridDev* __restrict__ grid, int n_leaf, double margin, float gamma_k,
                             int8_t* __restrict__ level, float* __restrict__ leaf_side,
                             uint64_t* __restrict__ tkey, uint64_t* __restrict__ tkey_copy) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = skey[s];
    const int32_t c = (int32_t)(key >> 30);
    const GridDev G = grid[sim_of_cell(grid, n_sims, c)];
    const double reach = (1.0 + margin) * (double)(gamma_k * h[perm[s]]);
    // A cell holding s has at most n_leaf particles only if it lies within
    // (s - n_leaf, s + n_leaf) in source order: if the key n_leaf places away
    // on either side shares its prefix, the cell holds more; else its bounds
    // are searched in that window (a few loads near s, instead of bisecting
    // each level's cell from its parent's range)
    const int64_t wl = s - n_leaf, wr = s + n_leaf;
    const uint64_t kl = wl >= 0 ? skey[wl] : 0ull, kr = wr < n ? skey[wr] : 0ull;
    int d = 0;
    // the side of level d + 1, G.cell / 2^(d + 1), by exact halvings (no
    // FP64 division: this GPU's FP64 pipe is slow)
    double side_next = 0.5 * G.cell;
    for (;; ++d, side_next *= 0.5) {
      const int sh = 3 * (kTreeDepth - d);
      const uint64_t pre = key >> sh;
      bool small = false;  // the cell holds at most n_leaf particles
      if (!((wl >= 0 && (kl >> sh) == pre) || (wr < n && (kr >> sh) == pre))) {
        const int64_t lo = lower_bound64(skey, wl + 1 > 0 ? wl + 1 : 0, s + 1, pre << sh);
        const int64_t hi = lower_bound64(skey, s + 1, wr < n ? wr : n, (pre + 1) << sh);
        small = hi - lo <= n_leaf;
      }
      if (d == kTreeDepth || small) break;
      if (side_next < reach) break;
    }
    level[s] = (int8_t)d;
    leaf_side[s] = G.cell_f * __int_as_float((127 - d) << 23);  // G.cell_f / 2^d, exact
    const int sh = 3 * (kTreeDepth - d);
    const uint64_t m = ((key & 0x3fffffffull) >> sh) << sh;
    const uint64_t t = ((uint64_t)(uint32_t)c << 34) | (m << 4) | (uint64_t)d;
    tkey[s] = t;
    tkey_copy[s] = t;
  }
}

// Target keys in target order (tgt: target order -> source index).
__global__ void k_tree_tsorted(int64_t n, const int32_t* __restrict__ tgt, const uint64_t* __restrict__ tkey,
                               uint64_t* __restrict__ tsorted) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    tsorted[k] = tkey[tgt[k]];
}

__global__ void k_tree_leaf_flag(int64_t n, const uint64_t* __restrict__ tsorted, int32_t* __restrict__ flag) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    flag[k] = (k == 0) || (tsorted[k] != tsorted[k - 1]);
}

// After the exclusive scan of flag (-> leaf_of), the group records.
__global__ void k_tree_leaf_fill(int64_t n, const uint64_t* __restrict__ tsorted, const int32_t* __restrict__ flag,
                                 const int32_t* __restrict__ leaf_of, TreeLeaf* __restrict__ leaves) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[k]) continue;
    const uint64_t t = tsorted[k];
    const int d = (int)(t & 15u);
    const uint32_t m = (uint32_t)((t >> 4) & 0x3fffffffull);
    const int sh = kTreeDepth - d;
    TreeLeaf L;
    L.start = (int32_t)k;
    L.depth = d;
    L.cell = (int32_t)(t >> 34);
    L.lx = (int32_t)(compact3(m) >> sh);
    L.ly = (int32_t)(compact3(m >> 1) >> sh);
    L.lz = (int32_t)(compact3(m >> 2) >> sh);
    L.pad = 0;
    leaves[leaf_of[k]] = L;
  }
}

__global__ void k_tree_leaf_count(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ leaf_of,
                                  int32_t* __restrict__ n_leaves, TreeLeaf* __restrict__ leaves) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int32_t nl = n > 0 ? leaf_of[n - 1] + flag[n - 1] : 0;
    *n_leaves = nl;
    leaves[nl].start = (int32_t)n;  // sentinel: end of the last group
  }
}

// 27 neighbour ranges of each leaf: the cells of the leaf's side around it,
// with the periodic shift (-1, 0, +1 boxes) of each axis packed in `shift`.
__global__ void k_tree_neigh(const TreeLeaf* __restrict__ leaves, const int32_t* __restrict__ n_leaves_p,
                             const uint64_t* __restrict__ skey, int64_t n, const int32_t* __restrict__ cell_start,
                             int n_sims, const GridDev* __restrict__ grid, TreeRange* __restrict__ ranges) {
  const int32_t nl = *n_leaves_p;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nl * 27;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t li = (int32_t)(t / 27);
    const TreeLeaf L = leaves[li];
    const GridDev G = grid[sim_of_cell(grid, n_sims, L.cell)];
    ranges[t] = neighbour_range(G, L, (int)(t % 27), skey, cell_start);
  }
}

// Per particle in tree order: the fine integer position (kTreeFine sub-cells
// per top cell, over the whole box) with the reverse-pair threshold, the FP32 offset from that sub-cell's
// corner (differences of positions stay exact at the leaf scale) with the
// mass, the velocity with u, the starting h, and the list radius
// min(leaf side, kListReach * gamma_K * h).
__global__ void k_tree_gather(int64_t n, const int32_t* __restrict__ perm, const uint64_t* __restrict__ skey,
                              int n_sims, const GridDev* __restrict__ grid, const double* __restrict__ x,
                              const double* __restrict__ y, const double* __restrict__ z,
                              const float* __restrict__ m, const float* __restrict__ vx,
                              const float* __restrict__ vy, const float* __restrict__ vz,
                              const float* __restrict__ u, const float* __restrict__ h,
                              const float* __restrict__ leaf_side, float list_reach, float gamma_k,
                              int4* __restrict__ fine,
                              float4* __restrict__ rel, float4* __restrict__ vel4, float* __restrict__ hs,
                              float* __restrict__ lrad) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[s];
    const uint64_t key = skey[s];
    const int32_t c = (int32_t)(key >> 30);
    const GridDev G = grid[sim_of_cell(grid, n_sims, c)];
    const int32_t local = c - G.cell_base, nc = G.n_c;
    const int32_t kx = local % nc, ky = (local / nc) % nc, kz = local / (nc * nc);
    const uint32_t mc = (uint32_t)(key & 0x3fffffffu);
    const int32_t gx = kx * kTreeFine + (int32_t)compact3(mc);
    const int32_t gy = ky * kTreeFine + (int32_t)compact3(mc >> 1);
    const int32_t gz = kz * kTreeFine + (int32_t)compact3(mc >> 2);
    const double sf = G.cell / (double)kTreeFine;
    const float hp = h[p];
    const float R = fminf(leaf_side[s], list_reach * gamma_k * hp);
    // w: the list radius lowered by a margin of the leaf side (the reverse
    // pairs' threshold, read with the fine position)
    fine[s] = make_int4(gx, gy, gz, __float_as_int(R - 0x1p-18f * leaf_side[s]));
    rel[s] = make_float4((float)(x[p] - (double)gx * sf), (float)(y[p] - (double)gy * sf),
                         (float)(z[p] - (double)gz * sf), m[p]);
    vel4[s] = make_float4(vx[p], vy[p], vz[p], u[p]);
    hs[s] = hp;
    lrad[s] = R;
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int blocks_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_tree_build(const TreeBuildArgs& a, cudaStream_t st) {
  const int64_t n = a.n_total;
  if (n <= 0) {
    k_tree_leaf_count<<<1, 32, 0, st>>>(0, a.flag, a.leaf_of, a.n_leaves, a.leaves);
    return cudaGetLastError();
  }
  int cbits = 1;
  while (cbits < 30 && ((int64_t)1 << cbits) <= a.cap_cells) ++cbits;
  // source order: (top cell, Morton code), ties by pool index
  k_tree_key<<<blocks_n(n), 256, 0, st>>>(n, a.x, a.y, a.z, a.sim_offset, a.n_sims, a.grid, a.cell_key,
                                          a.key64, a.key64_b);
  cudaError_t e = radix_sort_index64(n, 30 + cbits, a.key64_b, a.key64_c, a.perm, a.rv, a.hist, st);
  if (e != cudaSuccess) return e;
  k_tree_sorted<<<blocks_n(n), 256, 0, st>>>(n, a.perm, a.key64, a.skey);
  // levels and target order: (top cell, cell at the level, level), ties by source index
  k_tree_level<<<blocks_n(n), 256, 0, st>>>(n, a.skey, a.perm, a.h, a.n_sims, a.grid, a.n_leaf,
                                            a.margin, a.gamma_k, a.level, a.leaf_side, a.key64, a.key64_b);
  e = radix_sort_index64(n, 34 + cbits, a.key64_b, a.key64_c, a.tgt, a.rv, a.hist, st);
  if (e != cudaSuccess) return e;
  k_tree_tsorted<<<blocks_n(n), 256, 0, st>>>(n, a.tgt, a.key64, a.key64_c);
  k_tree_leaf_flag<<<blocks_n(n), 256, 0, st>>>(n, a.key64_c, a.flag);
  cudaMemcpyAsync(a.leaf_of, a.flag, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
  e = scan_exclusive_host_n(a.leaf_of, n, a.scan_tmp, st);
  if (e != cudaSuccess) return e;
  k_tree_leaf_fill<<<blocks_n(n), 256, 0, st>>>(n, a.key64_c, a.flag, a.leaf_of, a.leaves);
  k_tree_leaf_count<<<1, 32, 0, st>>>(n, a.flag, a.leaf_of, a.n_leaves, a.leaves);
  k_tree_neigh<<<blocks_n(n * 4), 256, 0, st>>>(a.leaves, a.n_leaves, a.skey, n, a.cell_start, a.n_sims, a.grid,
                                                a.ranges);
  return cudaGetLastError();
}

cudaError_t launch_tree_gather(const TreeGatherArgs& a, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  k_tree_gather<<<blocks_n(a.n_total), 256, 0, st>>>(a.n_total, a.perm, a.skey, a.n_sims, a.grid, a.x, a.y, a.z,
                                                     a.m, a.vx, a.vy, a.vz, a.u, a.h, a.leaf_side, a.list_reach,
                                                     a.gamma_k, a.fine, a.rel, a.vel4, a.hs, a.lrad);
  return cudaGetLastError();
}

}  // namespace sphh
