// blocks.cuh -- 2x2x2 blocks of cells for the loop kernels.
//
// A thread block of 8 warps owns a block of (up to) 2x2x2 target cells, one
// warp per cell.  The union of their 27-cell neighbourhoods is the
// (w+2)^3 <= 4x4x4 box of cells around the block; it is staged once in shared
// memory for all 8 warps (64 cells instead of 8 x 27).  Staged positions are
// relative to the centre of the block's first 2x2x2 cells, i.e. within two
// cells of the origin, so FP32 offsets keep the precision of the cell scale.
// Each warp then walks its own 3x3x3 sub-box as 9 contiguous runs of three
// cells (staged rows are contiguous along x).
#pragma once
#include "sph_internal.cuh"

namespace sphk {

constexpr int kBlkWarps = 8;
// Staged sources per block: a 4x4x4-cell box of a jittered lattice with cells
// of ~2.4 spacings holds up to ~1100 particles.  The density and force loops
// use the same capacity, so they stage (and overflow) identically.
constexpr int kBlkStageCap = 1216;
// Kernels with a wider support (in units of h) have larger cells and more
// particles per cell, in proportion to gamma_K^3: the Wendland C2 kernel
// (x1.14) stages up to 1400 sources, the quartic spline (x1.35) up to 1520,
// the most that keeps two force blocks per SM.
template <int K>
__host__ __device__ constexpr int stage_cap() {
  return K == kKernQuartic ? 1520 : (K == kKernWendlandC2 ? 1400 : kBlkStageCap);
}
// Neighbour-list entries per lane (sources within one cell size; with two
// lanes per target a lattice lane holds ~28 +- 4).
constexpr int kLaneListCap = 44;
// Global neighbour-list region per (target, lane): 48 u16 entries = 96 bytes,
// written and read as 16-byte vectors.  The plain lists of a target's lanes
// lie one after another in the target's 4 regions (list_offset); the
// symmetric force's lists keep one region per lane.
constexpr int kListRegion = 48;

// Offset (u16 entries) of lane sub's plain list in its target's regions: the
// lower lanes' published counts (0xffff: not published) rounded up to
// 16-byte words.
__device__ __forceinline__ int list_offset(const uint16_t* __restrict__ list_cnt, int32_t ti, int sub) {
  const uint2 c = *reinterpret_cast<const uint2*>(list_cnt + (int64_t)ti * 4);
  const uint32_t n0 = c.x & 0xffffu, n1 = c.x >> 16, n2 = c.y & 0xffffu;
  int off = 0;
  if (sub > 0 && n0 != 0xffffu) off += (int)((n0 + 7u) & ~7u);
  if (sub > 1 && n1 != 0xffffu) off += (int)((n1 + 7u) & ~7u);
  if (sub > 2 && n2 != 0xffffu) off += (int)((n2 + 7u) & ~7u);
  return off;
}
constexpr int kBlkThreads = 32 * kBlkWarps;
constexpr int kMaxStaged = 64;  // staged cells per block (4 x 4 x 4)

struct BlockGeom {
  GridDev G;
  int32_t c0x, c0y, c0z;  // first cell of the block on each axis
  int32_t wx, wy, wz;     // cells of the block on each axis (1 or 2)
  int32_t ex, ey, ez;     // staged cells on each axis (w + 2)
};

__device__ __forceinline__ int sim_of_block(const GridDev* __restrict__ grid, int n_sims, int32_t b) {
  int lo = 0, hi = n_sims - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (grid[mid].blk_base <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ BlockGeom block_geom(const GridDev* __restrict__ grid, int n_sims, int32_t b) {
  BlockGeom g;
  g.G = grid[sim_of_block(grid, n_sims, b)];
  const int32_t nb = (g.G.n_c + 1) >> 1;
  const int32_t local = b - g.G.blk_base;
  const int32_t bx = local % nb, by = (local / nb) % nb, bz = local / (nb * nb);
  g.c0x = 2 * bx;
  g.c0y = 2 * by;
  g.c0z = 2 * bz;
  g.wx = min(2, g.G.n_c - g.c0x);
  g.wy = min(2, g.G.n_c - g.c0y);
  g.wz = min(2, g.G.n_c - g.c0z);
  g.ex = g.wx + 2;
  g.ey = g.wy + 2;
  g.ez = g.wz + 2;
  return g;
}

// Global cell id of staged cell (sx, sy, sz), with periodic wrap.
__device__ __forceinline__ int32_t staged_cell_id(const BlockGeom& g, int sx, int sy, int sz) {
  const int32_t nc = g.G.n_c;
  int32_t x = g.c0x - 1 + sx, y = g.c0y - 1 + sy, z = g.c0z - 1 + sz;
  x += x < 0 ? nc : 0;
  x -= x >= nc ? nc : 0;
  y += y < 0 ? nc : 0;
  y -= y >= nc ? nc : 0;
  z += z < 0 ? nc : 0;
  z -= z >= nc ? nc : 0;
  return g.G.cell_base + x + nc * (y + nc * z);
}

// Shared tables of the staged cells: global start, count, staged start.
struct StageTable {
  int32_t gstart[kMaxStaged];
  int32_t len[kMaxStaged];
  int32_t start[kMaxStaged + 1];
};

// Fills the table (block-collective; ends with __syncthreads()).  Returns the
// number of staged sources.
__device__ __forceinline__ int32_t build_stage_table(const BlockGeom& g,
                                                     const int32_t* __restrict__ cell_start,
                                                     StageTable& T) {
  const int n_stage = g.ex * g.ey * g.ez;
  const int t = threadIdx.x;
  if (t < kMaxStaged) {
    int32_t a = 0, l = 0;
    if (t < n_stage) {
      const int sx = t % g.ex, sy = (t / g.ex) % g.ey, sz = t / (g.ex * g.ey);
      const int32_t cid = staged_cell_id(g, sx, sy, sz);
      a = cell_start[cid];
      l = cell_start[cid + 1] - a;
    }
    T.gstart[t] = a;
    T.len[t] = l;
    // inclusive scan over the 64 entries held by warps 0 and 1
    int32_t v = l;
    const int lane = t & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    T.start[t + 1] = v;  // warp-local inclusive sums, fixed below
  }
  __syncthreads();
  if (t >= 32 && t < kMaxStaged) T.start[t + 1] += T.start[32];
  if (t == 0) T.start[0] = 0;
  __syncthreads();
  return T.start[kMaxStaged];
}

// Staged cell of staged source v (binary search over T.start).
__device__ __forceinline__ int staged_cell_of(const StageTable& T, int32_t v) {
  int lo = 0, hi = kMaxStaged - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.start[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Offset (in cells) of staged cell k relative to the block centre.
__device__ __forceinline__ void staged_offset(const BlockGeom& g, int k, float& ox, float& oy, float& oz) {
  const int sx = k % g.ex, sy = (k / g.ex) % g.ey, sz = k / (g.ex * g.ey);
  ox = (float)(sx - 2) * g.G.cell_f;
  oy = (float)(sy - 2) * g.G.cell_f;
  oz = (float)(sz - 2) * g.G.cell_f;
}

// The targets of a block: the particles of its (up to 8) cells in staged
// order, split into rounds of `per` targets (tpp lanes each): about n/8
// targets per round, at most 16 (two lanes per target) or 8 (four lanes per
// target).  Warp w starts with round w and then takes the next unclaimed
// round from a shared counter, so that when a block has more rounds than
// warps, warps finishing early pick up the rest.  (Measured on the 2M
// lattice, fixed rounds of 8 targets with four lanes each were 11 % slower
// in the density loop: more lane combines, no better balance.)
struct BlockTargets {
  int32_t cell_k[8];      // staged cell index of block cell i
  int32_t cell_first[9];  // prefix of the block cells' particle counts
  int32_t n;              // targets in the block
  int32_t per, tpp, lg, rounds;
  int32_t next;           // next unclaimed round
  int32_t wcount[kBlkWarps];  // active targets per warp slice (masked builds)
};

// The round after `rd` for this warp (warp-collective).
__device__ __forceinline__ int next_round(BlockTargets& B, int lane) {
  int r = 0;
  if (lane == 0) r = atomicAdd(&B.next, 1);
  return __shfl_sync(0xffffffffu, r, 0);
}

// Block-collective; ends with __syncthreads().  Targets are dealt to warps
// in rounds of `per` targets with tpp lanes each: 4 lanes up to 8 targets a
// round, else 2 lanes for up to 16.  Kernels wider than the cubic spline (K)
// always take 4 lanes: their lists are 1.2-1.4 times longer, and at 2 lanes
// a few percent of lanes would overflow their list, which sends every warp
// holding one down the direct path.  The density and the force call this
// with the same K (and mask), so their rounds (and list columns) agree.
//
// act (sorted order, may be null): only targets with act != 0 are dealt, in
// the same order; the block's particles are compacted with one ballot per
// warp and 256 targets at a time.
//
// lanes (a tuning knob, the same for the density and the force): 0 = the
// rule above, 2 or 4 = that many lanes for every target (up to 16 or 8
// targets a round).
template <int K = kKernCubic>
__device__ __forceinline__ void build_targets(const BlockGeom& g, const StageTable& T, BlockTargets& B,
                                              uint16_t* tgt_slot, uint8_t* tgt_cell,
                                              const uint8_t* __restrict__ act = nullptr, int lanes = 0) {
  if (threadIdx.x == 0) {
    int i = 0, run = 0;
    for (int z = 1; z <= g.wz; ++z)
      for (int y = 1; y <= g.wy; ++y)
        for (int x = 1; x <= g.wx; ++x) {
          const int k = x + g.ex * (y + g.ey * z);
          B.cell_k[i] = k;
          B.cell_first[i] = run;
          run += T.len[k];
          ++i;
        }
    for (; i < 8; ++i) {
      B.cell_k[i] = 0;
      B.cell_first[i] = run;
    }
    B.cell_first[8] = run;
    B.n = run;
  }
  __syncthreads();
  const int run = B.cell_first[8];
  int n = run;
  if (act == nullptr) {
    for (int e = threadIdx.x; e < run; e += blockDim.x) {
      int i = 0;
      while (i < 7 && B.cell_first[i + 1] <= e) ++i;
      tgt_slot[e] = (uint16_t)(T.start[B.cell_k[i]] + (e - B.cell_first[i]));
      tgt_cell[e] = (uint8_t)i;
    }
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    n = 0;
    for (int e0 = 0; e0 < run; e0 += blockDim.x) {
      const int e = e0 + threadIdx.x;
      bool on = false;
      int i = 0;
      if (e < run) {
        while (i < 7 && B.cell_first[i + 1] <= e) ++i;
        on = act[T.gstart[B.cell_k[i]] + (e - B.cell_first[i])] != 0;
      }
      const unsigned m = __ballot_sync(0xffffffffu, on);
      if (lane == 0) B.wcount[warp] = __popc(m);
      __syncthreads();
      int off = n, tot = 0;
      for (int w = 0; w < kBlkWarps; ++w) {
        off += w < warp ? B.wcount[w] : 0;
        tot += B.wcount[w];
      }
      if (on) {
        const int pos = off + __popc(m & ((1u << lane) - 1u));
        tgt_slot[pos] = (uint16_t)(T.start[B.cell_k[i]] + (e - B.cell_first[i]));
        tgt_cell[pos] = (uint8_t)i;
      }
      n += tot;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    B.n = n;
    int per = (n + kBlkWarps - 1) / kBlkWarps;
    per = per < 1 ? 1 : per;
    if ((K != kKernCubic || lanes == 4) && per > 8) per = 8;
    const int tpp = lanes == 2 ? 2 : (per <= 8 ? 4 : 2);
    if (per > 16) per = 16;
    B.per = per;
    B.tpp = tpp;
    B.lg = tpp == 4 ? 2 : 1;
    B.rounds = (n + per - 1) / per;
    B.next = kBlkWarps;
  }
  __syncthreads();
}

// Warp w's target cell inside the block, and whether it exists.
__device__ __forceinline__ bool warp_cell(const BlockGeom& g, int w, int& tx, int& ty, int& tz) {
  tx = w & 1;
  ty = (w >> 1) & 1;
  tz = w >> 2;
  return tx < g.wx && ty < g.wy && tz < g.wz;
}

// Run r (0..8) of a warp's 3x3x3 neighbourhood: staged cells (tx..tx+2, ty+dy, tz+dz)
// are contiguous; returns [a, b) in staged source indices.
__device__ __forceinline__ void warp_run(const BlockGeom& g, const StageTable& T, int tx, int ty, int tz,
                                         int r, int32_t& a, int32_t& b) {
  const int dy = r % 3, dz = r / 3;
  const int k0 = tx + g.ex * ((ty + dy) + g.ey * (tz + dz));
  a = T.start[k0];
  b = T.start[k0 + 3];
}

}  // namespace sphk
