// tree_loops.cu -- density and force loops on the leaves of the nested grids
// (tree.cu).  Same mathematics as density.cu / force.cu (Sec. 3.1 and 3.2);
// the unit of work is a leaf and the 27 cells of its size around it.
//
// Positions.  Every particle carries its fine integer position (1024
// sub-cells per top cell) and its FP32 offset from that sub-cell's corner.
// Relative to a leaf corner a position is
//     (fine - corner + shift * N_fine) * s_fine + offset,
// the integer part exact, so FP32 keeps the sub-cell scale's precision
// however wide the top cells are.
//
// Density, one warp per leaf, kTreeTpp lanes per target:
//   1. the 27 ranges are staged in chunks relative to the leaf corner;
//   2. each target keeps, in per-lane lists, the sources closer than its list
//      radius R_i = min(leaf side, kTreeListReach * starting support);
//   3. Newton-Raphson passes read r^2 from the lists; a target whose support
//      outgrows R_i (or whose list overflows) leaves its group for the
//      per-target kernel (k_tree_density_fb at its own level: a warp per
//      target over its 27 cells), so that its round-mates do not wait;
//   4. the final pass at the converged h gathers the sources from memory and
//      publishes the lists for the force loop.
// A force pair needs r < max(H_i, H_j).  The list of i holds every j with
// r < R_i >= H_i; a j with H_j > r >= R_i is only in j's own reach, so the
// density of j emits it as a reverse pair (receiver i, source j).  Reverse
// pairs are grouped by receiver and sorted by source (deterministic order).
//
// Force, one warp per leaf: each target walks its list and its reverse pairs.
// The same kernels run the SPHENIX force and gradient pass (Sec. 3.3) with a
// fifth record per source (kTSphenix, kTGradient).
// Whether a pair is the list's or a reverse pair is decided in the target's
// own leaf frame with the same arithmetic as the density filter, so no pair is
// counted twice or dropped at the boundary; emission uses a margin so that the
// reverse pairs are a superset.
#include <type_traits>

#include "sph_internal.cuh"
#include "sph_launch.h"
#include "tree.cuh"

namespace sphk {

constexpr int kTWarps = 4;       // warps per CTA
#ifndef SPH_TREE_TCAP
#define SPH_TREE_TCAP 384
#endif
constexpr int kTCap = SPH_TREE_TCAP;  // staged sources per warp and chunk
constexpr int kTRows = kTreeList + 1;  // + one scratch row for the branch-free append
constexpr int kTPer = 32 / kTreeTpp;   // targets per round
constexpr int kTChildren = 27 * 8;      // children of the 27 neighbour cells

// Pruning tables of a warp's group (groups that do not fit one staging chunk).
struct TPrune {
  int32_t cv[kTChildren + 4];    // virtual start of each child (Morton order), + end
  int32_t hoff[kTChildren + 4];  // offsets of the round's hit children, + total
  uint8_t hch[kTChildren];       // the round's hit children, in order
  int32_t rlo[28], rcum[28], rsc[28];  // per neighbour range: first source, virtual start, shift
  uint32_t cact[(kTChildren + 31) / 32];  // masked loops: children holding a masked source
};
constexpr size_t kTPruneBytes = (sizeof(TPrune) + 15) / 16 * 16;
constexpr size_t kTWarpSmem = (size_t)kTCap * (sizeof(float4) + sizeof(uint32_t)) +
                              (size_t)kTRows * 32 * (sizeof(float) + sizeof(uint32_t)) + kTPruneBytes;
constexpr size_t kTDensSmem = kTWarps * kTWarpSmem;
constexpr int kNoShift = 1 | (1 << 2) | (1 << 4);
// list_cnt marker: the target is solved by the per-target kernels
constexpr uint16_t kListFallback = 0xfffe;
// fallback queue entries: a target index, with this bit for a target queued
// from its group (solved at its own level), and this one for a target outside
// the mask of masked loops (its current support sends reverse pairs only);
// indices stay below 2^29
constexpr int32_t kFbOwnLevel = 1 << 30;
constexpr int32_t kFbPassive = 1 << 29;
constexpr int32_t kFbIndex = kFbPassive - 1;
static_assert(kTWarpSmem % 16 == 0, "per-warp regions keep float4 alignment");
static_assert(kTreeList <= kTreeListRegion, "published lists fit their regions");
// a target's published list: its lanes' lists packed one after another in a
// region of kTreeTpp * kTreeListRegion entries, the count in list_cnt[target]
constexpr int kTreeListTarget = kTreeTpp * kTreeListRegion;

struct TGeo {
  float s_fine;        // side of a fine sub-cell
  float side;          // side of the leaf
  double side_d;
  int32_t nfine;       // fine sub-cells per box side
  int32_t ox, oy, oz;  // fine integer position of the leaf corner
  double L;
};

__device__ __forceinline__ TGeo leaf_geo(const TreeLeaf& Lf, const GridDev& G) {
  TGeo g;
  const int32_t local = Lf.cell - G.cell_base, nc = G.n_c;
  const int32_t kx = local % nc, ky = (local / nc) % nc, kz = local / (nc * nc);
  const int sh = kTreeDepth - Lf.depth;
  g.ox = kx * kTreeFine + (Lf.lx << sh);
  g.oy = ky * kTreeFine + (Lf.ly << sh);
  g.oz = kz * kTreeFine + (Lf.lz << sh);
  g.s_fine = (float)(G.cell / (double)kTreeFine);
  g.side_d = G.cell * __longlong_as_double((long long)(1023 - Lf.depth) << 52);  // G.cell / 2^depth, exact
  g.side = (float)g.side_d;
  g.nfine = nc * kTreeFine;
  g.L = G.L;
  return g;
}

// Position relative to the leaf corner of a particle seen with periodic shift
// code sc (2 bits per axis, shift + 1).
__device__ __forceinline__ float3 rel_to(const TGeo& g, const float4& rel, const int4& fine, int sc) {
  const int sx = (sc & 3) - 1, sy = ((sc >> 2) & 3) - 1, sz = ((sc >> 4) & 3) - 1;
  const int32_t dx = fine.x - g.ox + sx * g.nfine;
  const int32_t dy = fine.y - g.oy + sy * g.nfine;
  const int32_t dz = fine.z - g.oz + sz * g.nfine;
  return make_float3(fmaf((float)dx, g.s_fine, rel.x), fmaf((float)dy, g.s_fine, rel.y),
                     fmaf((float)dz, g.s_fine, rel.z));
}

__device__ __forceinline__ float r2_of(const float3& a, const float4& b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Pair vector x_i - x_j with the exact integer part (sc = shift code of j).
__device__ __forceinline__ float3 pair_vec(const TGeo& g, const float4& rel_i, const int4& fine_i,
                                           const float4& rel_j, const int4& fine_j, int sc) {
  const int sx = (sc & 3) - 1, sy = ((sc >> 2) & 3) - 1, sz = ((sc >> 4) & 3) - 1;
  const int32_t dx = fine_i.x - fine_j.x - sx * g.nfine;
  const int32_t dy = fine_i.y - fine_j.y - sy * g.nfine;
  const int32_t dz = fine_i.z - fine_j.z - sz * g.nfine;
  return make_float3(fmaf((float)dx, g.s_fine, rel_i.x - rel_j.x), fmaf((float)dy, g.s_fine, rel_i.y - rel_j.y),
                     fmaf((float)dz, g.s_fine, rel_i.z - rel_j.z));
}

// List entries pack the tree-order index (26 bits) with the shift code.
__device__ __forceinline__ uint32_t pack_js(int32_t j, int sc) { return (uint32_t)j | ((uint32_t)sc << 26); }
__device__ __forceinline__ int32_t unpack_j(uint32_t e) { return (int32_t)(e & 0x3ffffffu); }
__device__ __forceinline__ int unpack_s(uint32_t e) { return (int)(e >> 26); }
// Shift code of i seen from j, given that of j seen from i.
__device__ __forceinline__ int mirror_s(int sc) {
  return (2 - (sc & 3)) | ((2 - ((sc >> 2) & 3)) << 2) | ((2 - ((sc >> 4) & 3)) << 4);
}

// Groups are handed out one per warp from a counter: their costs differ by
// orders of magnitude (a coarse group beside a dense core stages thousands of
// sources), so a static assignment leaves a few warps running long after the
// others are done.
__device__ __forceinline__ int32_t next_group(int32_t* work, int lane) {
  int32_t g = 0;
  if (lane == 0) g = atomicAdd(work, 1);
  return __shfl_sync(0xffffffffu, g, 0);
}

struct TDSums {
  float w, dw, mw, mdw, div, cx, cy, cz;
  int npair;
};

__device__ __forceinline__ void tds_zero(TDSums& s) {
  s.w = s.dw = s.mw = s.mdw = s.div = s.cx = s.cy = s.cz = 0.f;
  s.npair = 0;
}

// One density pair with x_ij = (dx, dy, dz) (same terms as density.cu).
template <int K>
__device__ __forceinline__ void tdens_pair(float dx, float dy, float dz, const float4& vi, const float4& vj,
                                           float mj, float H, float Hinv, TDSums& s) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float q = r2 * rinv * Hinv;
  float w, g;
  kernel_w_g<K>(q, H * rinv, w, g);
  const float dw = fmaf(q * q, g, 3.0f * w);
  s.w += w;
  s.dw += dw;
  s.mw = fmaf(mj, w, s.mw);
  s.mdw = fmaf(mj, dw, s.mdw);
  const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;
  const float mg = mj * g;
  s.div = fmaf(mg, fmaf(ux, dx, fmaf(uy, dy, uz * dz)), s.div);
  s.cx = fmaf(mg, fmaf(uz, dy, -uy * dz), s.cx);
  s.cy = fmaf(mg, fmaf(ux, dz, -uz * dx), s.cy);
  s.cz = fmaf(mg, fmaf(uy, dx, -ux * dy), s.cz);
  s.npair += q < 1.0f;
}

// n-hat and its h-derivative terms of one pair (Newton passes).
template <int K>
__device__ __forceinline__ void tnewton_pair(float r2, float H, float Hinv, float& Sw, float& Sdw) {
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float q = r2 * rinv * Hinv;
  float w, dw;
  kernel_w_dw<K>(q, w, dw);
  Sw += w;
  Sdw += dw;
}

// Sum over the kTreeTpp lanes of a target (called by all 32 lanes).
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
  for (int o = 1; o < kTreeTpp; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int gsumi(int v) {
#pragma unroll
  for (int o = 1; o < kTreeTpp; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float gmax(float v) {
#pragma unroll
  for (int o = 1; o < kTreeTpp; o <<= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// True for every lane of a target if any of its lanes has b (called by all
// 32 lanes).
__device__ __forceinline__ bool group_any(bool b, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, b);
  return ((m >> (lane & ~(kTreeTpp - 1))) & ((1u << kTreeTpp) - 1u)) != 0u;
}

__device__ __forceinline__ void tcombine(TDSums& s) {
  s.w = gsum(s.w);
  s.dw = gsum(s.dw);
  s.mw = gsum(s.mw);
  s.mdw = gsum(s.mdw);
  s.div = gsum(s.div);
  s.cx = gsum(s.cx);
  s.cy = gsum(s.cy);
  s.cz = gsum(s.cz);
  s.npair = gsumi(s.npair);
}

// The leaf's 27 ranges, lane r < 27 holding range r; lanes 27..31 hold empty
// ranges, so lane 27's cumulative start is the total.
struct TRanges {
  int32_t lo, cum, sc;
  int nsrc;
};

__device__ __forceinline__ TRanges load_ranges(const TreeRange* __restrict__ ranges, int32_t li, int lane) {
  TRanges R;
  int32_t len = 0;
  R.lo = 0;
  R.sc = kNoShift;
  if (lane < 27) {
    const TreeRange t = ranges[(int64_t)li * 27 + lane];
    R.lo = t.lo;
    len = t.hi - t.lo;
    R.sc = t.shift;
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  R.cum = incl - len;
  R.nsrc = __shfl_sync(0xffffffffu, incl, 31);
  return R;
}

// Pruning tables of a group: per neighbour range its first source, virtual
// start and shift, and the virtual start of each of its 8 children (which
// are contiguous in Morton order; a cell of the deepest level has one).
// Lanes 0..26 search their range's keys.  Called by the whole warp.
__device__ __forceinline__ void prune_tables(const uint64_t* __restrict__ skey, const TRanges& R, int depth,
                                             int lane, TPrune* pr, const int32_t* __restrict__ act_pre = nullptr) {
  const int32_t cum_next = __shfl_down_sync(0xffffffffu, R.cum, 1);
  if (act_pre != nullptr) {
    if (lane < (kTChildren + 31) / 32) pr->cact[lane] = 0u;
    __syncwarp();
  }
  if (lane < 27) {
    const int32_t len = cum_next - R.cum;
    pr->rlo[lane] = R.lo;
    pr->rcum[lane] = R.cum;
    pr->rsc[lane] = R.sc;
    int32_t* cvr = pr->cv + lane * 8;
    cvr[0] = R.cum;
    if (depth < kTreeDepth && len > 0) {
      const int sh = 3 * (kTreeDepth - depth - 1);
      const uint64_t base = (skey[R.lo] >> (sh + 3)) << (sh + 3);
      // the seven child boundaries bisected together: each round takes one
      // step of every search, so its loads are in flight at once (a chain of
      // log2(len) loads instead of seven such chains)
      int32_t lo[7], hi[7];
#pragma unroll
      for (int c = 0; c < 7; ++c) {
        lo[c] = R.lo;
        hi[c] = R.lo + len;
      }
      for (bool more = true; more;) {
        more = false;
#pragma unroll
        for (int c = 0; c < 7; ++c) {
          if (lo[c] < hi[c]) {
            const int32_t mid = (int32_t)(((uint32_t)lo[c] + (uint32_t)hi[c]) >> 1);
            if (skey[mid] < base + ((uint64_t)(c + 1) << sh)) lo[c] = mid + 1; else hi[c] = mid;
            more = more || lo[c] < hi[c];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 7; ++c) cvr[c + 1] = R.cum + (lo[c] - R.lo);
    } else {
      for (int c = 1; c < 8; ++c) cvr[c] = R.cum + len;
    }
    if (act_pre != nullptr) {
      // which children hold a masked source (prefix sums over the range)
      unsigned bits = 0u;
      int32_t a0 = act_pre[R.lo];
      for (int c = 0; c < 8; ++c) {
        const int32_t v1 = c < 7 ? cvr[c + 1] : R.cum + len;
        const int32_t a1 = act_pre[R.lo + (v1 - R.cum)];
        bits |= (a1 > a0 ? 1u : 0u) << c;
        a0 = a1;
      }
      // 8 children of range `lane` are bits 8 lane .. 8 lane + 7
      if (bits) atomicOr(&pr->cact[lane >> 2], bits << (8 * (lane & 3)));
    }
  }
  if (lane == 0) pr->cv[kTChildren] = R.nsrc;
  __syncwarp();
}

// Squared distance from p (relative to the group corner) to child ch's box:
// neighbour r = ch / 8 at offset (r % 3, r / 3 % 3, r / 9) - 1 cells, child
// bits (x, y, z) = bits 0, 1, 2 of ch % 8, child side cside.
__device__ __forceinline__ float child_dist2(int ch, float side, float cside, const float3& p) {
  const int r = ch >> 3, c = ch & 7;
  const float bx = (float)(r % 3 - 1) * side + (float)(c & 1) * cside;
  const float by = (float)((r / 3) % 3 - 1) * side + (float)((c >> 1) & 1) * cside;
  const float bz = (float)(r / 9 - 1) * side + (float)((c >> 2) & 1) * cside;
  const float ex = fmaxf(fmaxf(bx - p.x, p.x - (bx + cside)), 0.0f);
  const float ey = fmaxf(fmaxf(by - p.y, p.y - (by + cside)), 0.0f);
  const float ez = fmaxf(fmaxf(bz - p.z, p.z - (bz + cside)), 0.0f);
  return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// The children any target of the round can reach: each target's lanes test
// 27 children each (ch = sub + 8 m) against its list radius, the union over
// the round's targets is compacted in child order with the offsets of their
// sources.  Returns the union's source count.  Called by the whole warp.
// lane sub owns children sub + kTreeTpp k (k < kCh) of every neighbour cell:
// bit m kCh + k of a lane's child mask
constexpr int kCh = 8 / kTreeTpp;
using ChMask = std::conditional_t<(27 * kCh > 32), unsigned long long, uint32_t>;

__device__ __forceinline__ int union_round(ChMask mine, int lane, TPrune* pr, int& nh);

__device__ __forceinline__ int prune_round(bool valid, int sub, int lane, const float3& pi, float Rb2,
                                           float side, float cside, TPrune* pr, int& nh, bool need_act = false) {
  using Mask = ChMask;
  Mask mine = 0;
  if (valid) {
    for (int m = 0; m < 27; ++m) {
#pragma unroll
      for (int k = 0; k < kCh; ++k) {
        const int ch = 8 * m + sub + kTreeTpp * k;
        // a target outside the mask reaches only the children with a masked
        // source (its list serves only reverse pairs to those)
        if (pr->cv[ch] < pr->cv[ch + 1] && (!need_act || ((pr->cact[ch >> 5] >> (ch & 31)) & 1u)) &&
            child_dist2(ch, side, cside, pi) < Rb2)
          mine |= (Mask)1 << (m * kCh + k);
      }
    }
  }
  return union_round(mine, lane, pr, nh);
}

// The lane's candidate children of a group (bits as above): those holding a
// source, and (mask_only) a masked one.  Called once per group, after
// prune_tables.
__device__ __forceinline__ ChMask group_candidates(int sub, const TPrune* pr, bool mask_only) {
  ChMask c = 0;
  for (int m = 0; m < 27; ++m) {
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
      const int ch = 8 * m + sub + kTreeTpp * k;
      if (pr->cv[ch] < pr->cv[ch + 1] && (!mask_only || ((pr->cact[ch >> 5] >> (ch & 31)) & 1u)))
        c |= (ChMask)1 << (m * kCh + k);
    }
  }
  return c;
}

// prune_round with the candidates precomputed per group and the box
// distances taken per axis: along each axis a lane's child boxes take three
// positions (the neighbour offset, its child bit fixed), so nine squared
// distances give all 27 (the sum's rounding lies far inside the margin of
// Rb2).
__device__ __forceinline__ int prune_round_fast(bool valid, int sub, int lane, const float3& pi, float Rb2,
                                                float side, float cside, TPrune* pr, int& nh, ChMask cand) {
  ChMask mine = 0;
  if (valid) {
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
      const int c = sub + kTreeTpp * k;
      const float cx = (float)(c & 1) * cside, cy = (float)((c >> 1) & 1) * cside, cz = (float)(c >> 2) * cside;
      float ex[3], ey[3], ez[3];
#pragma unroll
      for (int o = 0; o < 3; ++o) {
        const float b0 = (float)(o - 1) * side;
        const float dx = fmaxf(fmaxf(b0 + cx - pi.x, pi.x - (b0 + cx + cside)), 0.0f);
        const float dy = fmaxf(fmaxf(b0 + cy - pi.y, pi.y - (b0 + cy + cside)), 0.0f);
        const float dz = fmaxf(fmaxf(b0 + cz - pi.z, pi.z - (b0 + cz + cside)), 0.0f);
        ex[o] = dx * dx;
        ey[o] = dy * dy;
        ez[o] = dz * dz;
      }
#pragma unroll
      for (int m = 0; m < 27; ++m) {
        const ChMask bit = (ChMask)1 << (m * kCh + k);
        if ((cand & bit) && ex[m % 3] + ey[(m / 3) % 3] + ez[m / 9] < Rb2) mine |= bit;
      }
    }
  }
  return union_round(mine, lane, pr, nh);
}

// The union over the round's targets of their children, compacted in child
// order with the offsets of their sources; returns the union's source count.
// Called by the whole warp.
__device__ __forceinline__ int union_round(ChMask mine, int lane, TPrune* pr, int& nh) {
#pragma unroll
  for (int o = kTreeTpp; o < 32; o <<= 1) mine |= __shfl_xor_sync(0xffffffffu, mine, o);
  // lanes 0..kTreeTpp-1 hold the union; compacted in child order
  nh = 0;
  for (int m = 0; m < 27; ++m) {
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
      const bool hb = lane < kTreeTpp && ((mine >> (m * kCh + k)) & 1u);
      const unsigned b = __ballot_sync(0xffffffffu, hb);
      if (hb) {
        const int ch = 8 * m + kTreeTpp * k + lane;
        const int idx = nh + __popc(b & ((1u << lane) - 1u));
        pr->hch[idx] = (uint8_t)ch;
        pr->hoff[idx] = pr->cv[ch + 1] - pr->cv[ch];
      }
      nh += __popc(b);
    }
  }
  __syncwarp();
  int run = 0;
  for (int k0 = 0; k0 < nh; k0 += 32) {
    const int k = k0 + lane;
    const int v = k < nh ? pr->hoff[k] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int w = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += w;
    }
    if (k < nh) pr->hoff[k] = run + incl - v;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) pr->hoff[nh] = run;
  __syncwarp();
  return run;
}

// Stages cnt sources into spos / sidx [0, cnt) relative to the group corner
// (w: the mass, or the mask bit of masked loops); item u is source map(u) (its
// index and shift code).  A lane takes its items four at a time and issues
// their loads together, so that four L2 latencies overlap instead of running
// one after another.  Called by the whole warp.
template <class Map>
__device__ __forceinline__ void tstage_items(int cnt, int lane, const TGeo& g, const float4* __restrict__ rel,
                                             const int4* __restrict__ fine, float4* spos, uint32_t* sidx,
                                             const uint8_t* __restrict__ act, Map map) {
  for (int u0 = lane; u0 < cnt; u0 += 4 * 32) {
    int32_t j[4];
    int sc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      j[i] = 0;
      sc[i] = kNoShift;
      if (u0 + 32 * i < cnt) map(u0 + 32 * i, j[i], sc[i]);
    }
    float4 rj[4];
    int4 fj[4];
    float aw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      rj[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      fj[i] = make_int4(0, 0, 0, 0);
      aw[i] = 0.0f;
      if (u0 + 32 * i < cnt) {
        rj[i] = rel[j[i]];
        fj[i] = fine[j[i]];
        if (act != nullptr) aw[i] = (float)act[j[i]];
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int u = u0 + 32 * i;
      if (u < cnt) {
        const float3 p = rel_to(g, rj[i], fj[i], sc[i]);
        spos[u] = make_float4(p.x, p.y, p.z, act != nullptr ? aw[i] : rj[i].w);
        sidx[u] = pack_js(j[i], sc[i]);
      }
    }
  }
  __syncwarp();
}

// Stages sources [u0, u0 + kTCap) of the round's hit children (flattened)
// relative to the group corner.  Called by the whole warp.
__device__ __forceinline__ int tstage_union(int u0, int total, int nh, const TPrune* pr, int lane,
                                            const TGeo& g, const float4* __restrict__ rel,
                                            const int4* __restrict__ fine, float4* spos, uint32_t* sidx,
                                            const uint8_t* __restrict__ act = nullptr) {
  const int cnt = min(kTCap, total - u0);
  tstage_items(cnt, lane, g, rel, fine, spos, sidx, act, [&](int u, int32_t& j, int& sc) {
    const int uu = u0 + u;
    int lo = 0, hi = nh - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pr->hoff[mid] <= uu) lo = mid; else hi = mid - 1;
    }
    const int ch = pr->hch[lo];
    const int vv = pr->cv[ch] + (uu - pr->hoff[lo]);
    const int r = ch >> 3;
    j = pr->rlo[r] + (vv - pr->rcum[r]);
    sc = pr->rsc[r];
  });
  return cnt;
}

// Stages sources [v0, v0 + kTCap) of the concatenated ranges relative to the
// leaf corner (the ranges' first sources, starts and shifts go to pr first).
// Called by the whole warp.
__device__ __forceinline__ int tstage(int v0, const TRanges& R, int lane, const TGeo& g,
                                      const float4* __restrict__ rel, const int4* __restrict__ fine, float4* spos,
                                      uint32_t* sidx, TPrune* pr, const uint8_t* __restrict__ act = nullptr) {
  const int cnt = min(kTCap, R.nsrc - v0);
  if (lane < 28) {
    pr->rlo[lane] = R.lo;
    pr->rcum[lane] = R.cum;  // lane 27 (an empty range): the total
    pr->rsc[lane] = R.sc;
  }
  __syncwarp();
  tstage_items(cnt, lane, g, rel, fine, spos, sidx, act, [&](int u, int32_t& j, int& sc) {
    const int v = v0 + u;
    // the last range starting at or before v (an empty range shares its
    // start with the next one)
    int lo = 0, hi = 26;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pr->rcum[mid] <= v) lo = mid; else hi = mid - 1;
    }
    j = pr->rlo[lo] + (v - pr->rcum[lo]);
    sc = pr->rsc[lo];
  });
  return cnt;
}

// Reverse pair of target ti (support H, leaf side s_i) and source j (shift
// code sc of j seen from ti) at r^2 = r2 in ti's frame: wanted when r < H and
// r reaches past j's list radius, lowered by a margin above the rounding of r
// in either frame (the force decides again, exactly, in j's frame).  thr_j
// is j's list radius less 2^-18 of its leaf side (fine[j].w).
__device__ __forceinline__ bool want_reverse_t(float thr_j, int32_t ti, int32_t j, float r2, float H2, float H,
                                               float s_i) {
  if (!(r2 < H2) || j == ti) return false;
  const float thr = thr_j - 0x1p-18f * (s_i + H);
  return !(thr > 0.0f && r2 < thr * thr);
}
__device__ __forceinline__ bool want_reverse(const sphh::TreeDensityArgs& a, int32_t ti, int32_t j, float r2,
                                             float H2, float H, float s_i) {
  return want_reverse_t(__int_as_float(a.fine[j].w), ti, j, r2, H2, H, s_i);
}

// Appends the wanted records of the warp (one counter atomic per warp).
// Called by all 32 lanes.
__device__ __forceinline__ void emit_warp(const sphh::TreeDensityArgs& a, bool want, uint64_t rec, int lane) {
  const unsigned em = __ballot_sync(0xffffffffu, want);
  if (!em) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(a.rev_count, (unsigned long long)__popc(em));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (want) {
    const unsigned long long k = base + (unsigned long long)__popc(em & ((1u << lane) - 1u));
    if (k < (unsigned long long)a.rev_cap) {
      a.rev_raw[k] = rec;
      atomicAdd(&a.rev_start[(int32_t)(rec >> 32)], 1);
    } else {
      atomicOr(a.status, SPH_ST_CAPACITY);
    }
  }
}

__device__ __forceinline__ uint64_t reverse_rec(int32_t j, int32_t ti, int sc) {
  return ((uint64_t)(uint32_t)j << 32) | pack_js(ti, mirror_s(sc));
}

// Appends the list entries marked in each lane's mask wm (bit e: entry e of
// the lane's column in lje): one counter atomic for the warp, then every
// lane writes its records at its offset.  Called by all 32 lanes.
// one mask bit per list entry
using TMark = std::conditional_t<(kTreeList > 32), unsigned long long, uint32_t>;
__device__ __forceinline__ int tmark_popc(uint32_t m) { return __popc(m); }
__device__ __forceinline__ int tmark_popc(unsigned long long m) { return __popcll(m); }
__device__ __forceinline__ int tmark_ffs(uint32_t m) { return __ffs((int)m); }
__device__ __forceinline__ int tmark_ffs(unsigned long long m) { return __ffsll((long long)m); }

__device__ __forceinline__ void emit_marked(const sphh::TreeDensityArgs& a, TMark wm, const uint32_t* lje,
                                            int32_t ti, int lane) {
  static_assert(kTreeList <= 64, "one mask bit per list entry");
  const int my = tmark_popc(wm);
  int incl = my;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(a.rev_count, (unsigned long long)total);
  unsigned long long k = __shfl_sync(0xffffffffu, base, 0) + (unsigned long long)(incl - my);
  while (wm) {
    const int e = tmark_ffs(wm) - 1;
    wm &= wm - 1u;
    const uint32_t je = lje[e * 32 + lane];
    const int32_t j = unpack_j(je);
    if (k < (unsigned long long)a.rev_cap) {
      a.rev_raw[k] = reverse_rec(j, ti, unpack_s(je));
      atomicAdd(&a.rev_start[j], 1);
    } else {
      atomicOr(a.status, SPH_ST_CAPACITY);
    }
    ++k;
  }
}

// Outputs of target ti (source index) from its sums at h (Sec. 3.1 and the
// equation of state of Sec. 3.2).
template <int K>
__device__ __forceinline__ void tdens_write(const sphh::TreeDensityArgs& a, const PhysDev& ph, int32_t ti,
                                            float h, const TDSums& s, float u_i, int passes, bool noconv) {
  const int32_t p = a.perm[ti];
  const float H = KernT<K>::gamma * h;
  const float Hinv = 1.0f / H;
  const float H2inv = Hinv * Hinv;
  const float rho = s.mw * H2inv * Hinv;
  const float fval = 1.0f / (1.0f - s.mdw / (3.0f * s.mw));
  const float div = s.div * H2inv / s.mw;
  const float curl = sqrtf(fmaf(s.cx, s.cx, fmaf(s.cy, s.cy, s.cz * s.cz))) * H2inv / s.mw;
  const float P = (ph.gamma - 1.0f) * u_i * rho;
  const float cs = sqrtf(ph.gamma * P / rho);
  const float hf = h;
  a.h[p] = hf;
  a.rho[p] = rho;
  a.f[p] = fval;
  a.div_v[p] = div;
  a.curl_v[p] = curl;
  a.P[p] = P;
  a.c[p] = cs;
  a.B[p] = fabsf(div) / (fabsf(div) + curl + ph.eps_balsara * cs / hf);
  if (a.n_iter) a.n_iter[p] = passes;
  if (noconv) atomicOr(a.status, SPH_ST_H_NOCONV);
}

// kMask: the masked loops (a.act, a.act_pre set); the plain instance carries
// none of their tests.
template <int K, bool kMask>
__global__ void __launch_bounds__(kTWarps * 32) k_tree_density(sphh::TreeDensityArgs a, PhysDev ph) {
  extern __shared__ __align__(16) unsigned char tsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const NewtonConst nwt = newton_const<K>(ph);
  unsigned char* base = tsm + (size_t)warp * kTWarpSmem;
  float4* spos = reinterpret_cast<float4*>(base);
  uint32_t* sidx = reinterpret_cast<uint32_t*>(spos + kTCap);
  float* lr2 = reinterpret_cast<float*>(sidx + kTCap);
  uint32_t* lje = reinterpret_cast<uint32_t*>(lr2 + kTRows * 32);
  TPrune* pr = reinterpret_cast<TPrune*>(lje + kTRows * 32);
  const int t = lane / kTreeTpp, sub = lane % kTreeTpp;
  const int32_t nl = *a.n_leaves;
  unsigned long long pair_acc = 0, free_acc = 0;
  for (int32_t li = next_group(a.work, lane); li < nl; li = next_group(a.work, lane)) {
    const TreeLeaf Lf = a.leaves[li];
    const int32_t t_lo = Lf.start, n_t = a.leaves[li + 1].start - Lf.start;
    const GridDev G = a.grid[sim_of_cell(a.grid, a.n_sims, Lf.cell)];
    const TGeo g = leaf_geo(Lf, G);
    const TRanges R = load_ranges(a.ranges, li, lane);
    if (kMask) {
      // masked loops: a group without a masked particle in its 27 cells has
      // no masked target and no masked receiver of a reverse pair
      const int32_t cum_next = __shfl_down_sync(0xffffffffu, R.cum, 1);
      const int32_t na = lane < 27 ? a.act_pre[R.lo + (cum_next - R.cum)] - a.act_pre[R.lo] : 0;
      if (!__any_sync(0xffffffffu, na > 0)) continue;
    }
    const int nsrc = R.nsrc;
    const float hcap = h_cap<K>(g.side_d, g.L);
    const bool one_chunk = nsrc <= kTCap;
    // children are half the cell (a cell at the deepest level has one child)
    const float cside = Lf.depth < kTreeDepth ? 0.5f * g.side : g.side;
    // (masked loops: the staged w is 1 for a masked source, else 0)
    ChMask cand_all = 0, cand_act = 0;
    if (one_chunk) {
      tstage(0, R, lane, g, a.rel, a.fine, spos, sidx, pr, kMask ? a.act : nullptr);
    } else {
      prune_tables(a.skey, R, Lf.depth, lane, pr, kMask ? a.act_pre : nullptr);
      cand_all = group_candidates(sub, pr, false);
      if (kMask) cand_act = group_candidates(sub, pr, true);
    }
    for (int32_t t0 = 0; t0 < n_t; t0 += kTPer) {
      const bool valid = t0 + t < n_t;
      const int32_t ti = a.tgt[t_lo + (valid ? t0 + t : 0)];
      // masked loops: a target outside the mask keeps its h and outputs; its
      // list at its current support only sends reverse pairs to the masked
      // particles (whose forces need every pair within either support)
      const bool on = valid && (!kMask || a.act[ti] != 0);
      const float4 reli = a.rel[ti];
      const int4 fi = a.fine[ti];
      const float3 pi = rel_to(g, reli, fi, kNoShift);
      const float4 vi = a.vel4[ti];
      const float Ri = a.lrad[ti];
      const float R2 = Ri * Ri;
      // (a target outside the mask lists the masked sources only)
      const bool all_src = !kMask || on;
      // 1. filter: sources with r < R_i into this lane's list.  A group that
      // does not fit one staging chunk stages, per round, only the children
      // of its 27 cells that some target of the round reaches: a child whose
      // box lies beyond R_i (with a margin far above the rounding of r) holds
      // no list entry of that target.
      int cnt = 0;
      if (one_chunk) {
        if (valid) {
          for (int k = sub; k < nsrc; k += kTreeTpp) {
            const float4 sk = spos[k];
            const float r2 = r2_of(pi, sk);
            const int at = min(cnt, kTreeList) * 32 + lane;
            lr2[at] = r2;
            lje[at] = sidx[k];
            cnt += r2 < R2 && (all_src || sk.w != 0.0f);
          }
        }
      } else {
        int nh = 0;
        const int total = prune_round_fast(valid, sub, lane, pi, R2 * (1.0f + 0x1p-10f), g.side, cside, pr, nh,
                                           all_src ? cand_all : cand_act);
        for (int u0 = 0; u0 < total; u0 += kTCap) {
          const int c = tstage_union(u0, total, nh, pr, lane, g, a.rel, a.fine, spos, sidx, kMask ? a.act : nullptr);
          if (valid) {
            for (int k = sub; k < c; k += kTreeTpp) {
              const float4 sk = spos[k];
              const float r2 = r2_of(pi, sk);
              const int at = min(cnt, kTreeList) * 32 + lane;
              lr2[at] = r2;
              lje[at] = sidx[k];
              cnt += r2 < R2 && (all_src || sk.w != 0.0f);
            }
          }
          __syncwarp();
        }
      }
      // a target whose list overflowed, or whose support outgrows R_i, leaves
      // the group: it is queued for the per-target kernel, which solves it at
      // its own level with all 32 lanes of a warp over its 27 cells (so the
      // other targets of its round do not wait for it).  The flag is shared by
      // the target's lanes.
      bool queued = group_any(cnt > kTreeList, lane);
      // 2. Newton-Raphson passes
      float h = valid ? a.hs[ti] : hcap;
      if (on) {
        if (!(h > 0.0f)) h = 0.5f * hcap;
        if (h > hcap) h = hcap;
      }
      {
        // evaluated by every lane (a ballot), then merged
        const bool outgrown = group_any(valid && KernT<K>::gamma * h > Ri, lane);
        queued = queued || outgrown;
      }
      float hlo = 0.0f, hhi = INFINITY;
      bool done = !on || queued, atcap = false, conv = false;
      int it = 0, passes = 0;
      while (__any_sync(0xffffffffu, !done)) {
        const float H = KernT<K>::gamma * h;
        const float Hinv = 1.0f / H;
        float Sw = 0.f, Sdw = 0.f;
        if (!done)
          for (int e = 0; e < cnt; ++e) tnewton_pair<K>(lr2[e * 32 + lane], H, Hinv, Sw, Sdw);
        Sw = gsum(Sw);
        Sdw = gsum(Sdw);
        if (!done) {
          passes = it + 1;
          if (newton_update(Sw, Sdw, nwt, hcap, h, hlo, hhi, it, atcap, conv)) done = true;
        }
        // the list holds r < R_i: a support beyond it is queued
        const bool outgrown = group_any(valid && !queued && !atcap && KernT<K>::gamma * h > Ri, lane);
        if (outgrown) {
          queued = true;
          done = true;
        }
      }
      // 3. final pass at h
      const float H = KernT<K>::gamma * h;
      const float Hinv = 1.0f / H;
      const float H2 = H * H;
      TDSums s;
      tds_zero(s);
      // the list's reverse pairs are marked on the way (bit e: entry e; a
      // list holds at most kTreeList = 32), with j's threshold read with its
      // fine position
      TMark wm = 0;
      if (on && !queued) {
        for (int e = 0; e < cnt; ++e) {
          const uint32_t je = lje[e * 32 + lane];
          const int32_t j = unpack_j(je);
          const float4 rj = a.rel[j];
          const int4 fj = a.fine[j];
          const float3 d = pair_vec(g, reli, fi, rj, fj, unpack_s(je));
          tdens_pair<K>(d.x, d.y, d.z, vi, a.vel4[j], rj.w, H, Hinv, s);
          if (!atcap && want_reverse_t(__int_as_float(fj.w), ti, j, lr2[e * 32 + lane], H2, H, g.side) &&
              (!kMask || a.act[j] != 0))
            wm |= (TMark)1 << e;
        }
      } else if (kMask && valid && !queued) {
        // outside the mask: the reverse pairs to its listed (masked) sources
        for (int e = 0; e < cnt; ++e) {
          const int32_t j = unpack_j(lje[e * 32 + lane]);
          if (want_reverse(a, ti, j, lr2[e * 32 + lane], H2, H, g.side)) wm |= (TMark)1 << e;
        }
      }
      // reverse pairs from the lists: the warp takes one slot range for the
      // whole round
      emit_marked(a, wm, lje, ti, lane);
      tcombine(s);
      // 4. publish the list for the force loop: the target's lanes' lists
      // packed one after another (lane sub's entries after those of the
      // lanes below it), so that the force reads them in whole sectors
      {
        int incl = on && !queued ? cnt : 0;
#pragma unroll
        for (int o = 1; o < kTreeTpp; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o, kTreeTpp);
          if (sub >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, kTreeTpp - 1, kTreeTpp);
        if (on) {
          if (sub == 0) a.list_cnt[ti] = (uint16_t)(atcap || queued ? kListFallback : total);
          if (!queued) {
            uint32_t* dst = a.lists + (int64_t)ti * kTreeListTarget + (incl - cnt);
            for (int e = 0; e < cnt; ++e) dst[e] = lje[e * 32 + lane];
          }
        }
      }
      if (valid && sub == 0) {
        if (queued) {
          // solved at its own level by the per-target kernel
          const int32_t k = atomicAdd(a.fb_count, 1);
          if (k < a.n_total) a.fb_list[k] = ti | kFbOwnLevel | (on ? 0 : kFbPassive);
          free_acc += on ? 1ull : 0ull;
        } else if (on) {
          tdens_write<K>(a, ph, ti, h, s, vi.w, passes, !conv && !atcap);
          if (atcap) {
            // the support outgrew this level: re-solved at a coarser one
            const int32_t k = atomicAdd(a.fb_count, 1);
            if (k < a.n_total) a.fb_list[k] = ti;
          } else {
            pair_acc += (unsigned long long)s.npair;
          }
        }
      }
      __syncwarp();
    }
    __syncwarp();
  }
  if (ph.count_pairs) {
    unsigned long long v = pair_acc, w = free_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v += __shfl_xor_sync(0xffffffffu, v, o);
      w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if (lane == 0 && v) atomicAdd(a.pairs, v);
    if (lane == 0 && w) atomicAdd(a.list_free, w);
  }
}

// Reverse pairs -> per-receiver segments: rev_start holds the exclusive scan
// of the counts; each pair takes a slot of its receiver's segment.
__global__ void k_rev_scatter(const uint64_t* __restrict__ raw, const unsigned long long* __restrict__ count,
                              int64_t cap, const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                              uint32_t* __restrict__ rev) {
  const int64_t m = (int64_t)min(*count, (unsigned long long)cap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t e = raw[k];
    const int32_t r = (int32_t)(e >> 32);
    const int32_t pos = start[r] + atomicAdd(&fill[r], 1);
    rev[pos] = (uint32_t)(e & 0xffffffffu);
  }
}

// A segment of at most N entries sorted in registers: a bitonic network
// (every index fixed at compile time), padded with the largest key.
template <int N>
__device__ __forceinline__ void sort_segment_regs(uint32_t* __restrict__ rev, int32_t b, int32_t len) {
  uint32_t v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = k < len ? rev[b + k] : 0xffffffffu;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t x = v[i], y = v[l];
          const bool up = (i & k) == 0;
          v[i] = up ? min(x, y) : max(x, y);
          v[l] = up ? max(x, y) : min(x, y);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k < len) rev[b + k] = v[k];
}

// Sorts each receiver's segment by packed source (the slot order above is
// arbitrary), so the force sums run in a fixed order: up to 32 entries in
// registers, longer segments by insertion.
__global__ void k_rev_sort(int64_t n, const int32_t* __restrict__ start, uint32_t* __restrict__ rev) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = start[i], e = start[i + 1], len = e - b;
    if (len <= 1) continue;
    if (len <= 8) {
      sort_segment_regs<8>(rev, b, len);
    } else if (len <= 16) {
      sort_segment_regs<16>(rev, b, len);
    } else if (len <= 32) {
      sort_segment_regs<32>(rev, b, len);
    } else {
      for (int32_t k = b + 1; k < e; ++k) {
        const uint32_t v = rev[k];
        int32_t q = k - 1;
        while (q >= b && rev[q] > v) {
          rev[q + 1] = rev[q];
          --q;
        }
        rev[q + 1] = v;
      }
    }
  }
}

// ---- force ------------------------------------------------------------------

struct TFSums {
  float ax, ay, az, du, vsig;
  int npair;
};

// A source's force record, 64 bytes in source order (written by the force
// gather): q0 = (rel x, y, z, H), q1 = (fine x, y, z, rho as bits),
// q2 = (v, m), q3 = (f P / rho^2, f, c, B).  One record replaces six
// gathers from six arrays; 1/H is recomputed (correctly rounded, the value
// the arrays held).
struct TRec {
  float4 q0;
  int4 q1;
};

__device__ __forceinline__ TRec trec_head(const float4* __restrict__ rec, int32_t j) {
  const float4* r = rec + 4 * (int64_t)j;
  TRec t;
  t.q0 = r[0];
  t.q1 = *reinterpret_cast<const int4*>(r + 1);
  return t;
}

// Flavours of the force kernels: the "Minimal" force, the SPHENIX force and
// the SPHENIX gradient pass (Sec. 3.3; the terms are those of force.cu's
// flavours, with the fifth record E = (u, alpha_V, P, alpha_c) per source).
// The time-step limiter (kTLimit, Sec. 3.4) and the wake-up pass (kTWake)
// walk the same pairs with fE.x = each source's time bin.
enum : int { kTMin = 0, kTSphenix = 1, kTGradient = 2, kTLimit = 3, kTWake = 4 };

// One force pair with x_ij = (dx, dy, dz) (same terms as force.cu).  The
// gradient pass keeps only r < H_i (G_i = 0 beyond): the Laplacian sum
// (m_j / rho_j)(u_i - u_j) G_i in ax, the largest alpha_V in ay and the
// largest conduction speed v_c,ij in vsig.
template <int kFl, int K>
__device__ __forceinline__ void tforce_pair(float dx, float dy, float dz, const float4& vi, const float4& ci,
                                            const float4& ei, float Hi, float Hinv_i, float rho_i, const float4& vj,
                                            const float4& cj, const float4& ej, float Hj, float Hinv_j,
                                            float rho_j, const PhysDev& ph, TFSums& s) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  if constexpr (kFl == kTLimit) {
    // the largest bin among the force pairs (r < max(H_i, H_j)) in vsig
    const float Hm = fmaxf(Hi, Hj);
    const bool in = r2 < Hm * Hm;
    s.vsig = in ? fmaxf(s.vsig, ej.x) : s.vsig;
    s.npair += in;
    return;
  }
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  const float hi2 = Hinv_i * Hinv_i;
  const float Gi = kernel_g<K>(r * Hinv_i, Hi * rinv) * (hi2 * hi2 * Hinv_i);
  const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
  const float vdotx = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
  if constexpr (kFl == kTGradient) {
    s.ax = fmaf(__fdividef(vj.w, rho_j) * (ei.x - ej.x), Gi, s.ax);
    const float vc = fmaf(fabsf(vdotx), rinv, sqrtf(__fdividef(2.0f * fabsf(ei.z - ej.z), rho_i + rho_j)));
    const bool in = r2 < Hi * Hi;
    s.vsig = in ? fmaxf(s.vsig, vc) : s.vsig;
    s.ay = in ? fmaxf(s.ay, ej.y) : s.ay;
    s.npair += in;
    return;
  }
  const float hj2 = Hinv_j * Hinv_j;
  const float Gj = kernel_g<K>(r * Hinv_j, Hj * rinv) * (hj2 * hj2 * Hinv_j);
  const float mu = fminf(vdotx, 0.0f) * rinv;
  const float vs = fmaf(-ph.beta_v, mu, ci.z + cj.z);
  const float av = kFl == kTSphenix ? 0.5f * (ei.y + ej.y) : ph.alpha_v;
  const float nu = __fdividef(-av * (ci.w + cj.w) * mu * vs, rho_i + rho_j);
  const float piG = ci.x * Gi;
  const float visc = fmaf(ci.y, Gi, cj.y * Gj);
  const float mj = vj.w;
  const float sc = mj * fmaf(0.5f * nu, visc, fmaf(cj.x, Gj, piG));
  s.ax = fmaf(-sc, dx, s.ax);
  s.ay = fmaf(-sc, dy, s.ay);
  s.az = fmaf(-sc, dz, s.az);
  s.du = fmaf(mj * fmaf(0.25f * nu, visc, piG), vdotx, s.du);
  if constexpr (kFl == kTSphenix) {
    // conduction: zero beyond both supports (visc = 0) and for r = 0
    const float Ps = ei.z + ej.z, rs = rho_i + rho_j;
    const float ac = Ps > 0.0f ? __fdividef(fmaf(ei.z, ei.w, ej.z * ej.w), Ps) : 0.0f;
    const float vc = fmaf(fabsf(vdotx), rinv, sqrtf(__fdividef(2.0f * fabsf(ei.z - ej.z), rs)));
    s.du = fmaf(mj * ac * vc * (ei.x - ej.x) * r, __fdividef(visc, rs), s.du);
  }
  const float Hm = fmaxf(Hi, Hj);
  const bool in = r2 < Hm * Hm;
  s.vsig = in ? fmaxf(s.vsig, vs) : s.vsig;
  s.npair += in;
}

// tforce_pair with source j's data from its record (head already loaded) and,
// for the flavours with one, its fifth record.  The wake-up pass raises the
// wake-up bin of a source outside the mask within r < max(H_i, H_j) whose bin
// lies below the target's bin - 2 (Saitoh & Makino's limiter, Sec. 3.4).
template <int kFl, int K>
__device__ __forceinline__ void tforce_rec(float dx, float dy, float dz, const float4& vi, const float4& ci,
                                           const float4& ei, float Hi, float Hinv_i, float rho_i,
                                           const sphh::TreeForceArgs& a, int32_t j, const TRec& h, const PhysDev& ph,
                                           TFSums& s) {
  if constexpr (kFl == kTWake) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float Hm = fmaxf(Hi, h.q0.w);
    const int w = (int)ei.x - 2;
    if (r2 < Hm * Hm && a.act[j] == 0 && w > (int)a.fE[j].x) atomicMax(a.wake + a.perm[j], w);
    return;
  }
  const float4* r = a.rec + 4 * (int64_t)j;
  const float4 ej = kFl != kTMin ? a.fE[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (kFl == kTLimit) {
    tforce_pair<kFl, K>(dx, dy, dz, vi, ci, ei, Hi, Hinv_i, rho_i, vi, ci, ej, h.q0.w, 0.0f, 0.0f, ph, s);
  } else {
    tforce_pair<kFl, K>(dx, dy, dz, vi, ci, ei, Hi, Hinv_i, rho_i, r[2], r[3], ej, h.q0.w, __frcp_rn(h.q0.w),
                        __int_as_float(h.q1.w), ph, s);
  }
}

// The result of a target: the force, or the gradient pass's conduction
// parameter (the Euler step of eq. "artconddt" and its limiters, as in
// force.cu) and Laplacian.
template <int kFl>
__device__ __forceinline__ void tforce_write(const sphh::TreeForceArgs& a, const SphenixDev& x, float dt,
                                             int32_t ti, float Hi, const float4& ei, const TFSums& s) {
  const int32_t p = a.perm[ti];
  if constexpr (kFl == kTLimit) {
    // a step at most 4 times the smallest neighbour step: at most two bins
    // below the largest neighbour bin
    const int own = (int)ei.x, nb = (int)s.vsig - 2;
    a.bins_out[p] = own > nb ? own : nb;
  } else if constexpr (kFl == kTWake) {
    // the wake-up pass writes per source
  } else if constexpr (kFl == kTGradient) {
    const float lap = 2.0f * s.ax;
    const float src = ei.x > 0.0f ? x.beta_c * Hi * lap / sqrtf(ei.x) : 0.0f;
    const float rate = src - (ei.w - x.ac_min) * s.vsig / Hi;
    float an = fmaf(dt, rate, ei.w);
    an = fminf(an, x.ac_max * (1.0f - s.ay / x.av_max));
    an = fmaxf(an, x.ac_min);
    a.alpha_c_out[p] = an;
    if (a.lap_u != nullptr) a.lap_u[p] = lap;
  } else {
    a.ax[p] = s.ax;
    a.ay[p] = s.ay;
    a.az[p] = s.az;
    a.du_dt[p] = s.du;
    a.v_sig[p] = s.vsig;
  }
}

__device__ __forceinline__ float3 rec_rel_to(const TGeo& g, const TRec& h, int sc) {
  return rel_to(g, h.q0, h.q1, sc);
}

template <int kFl, int K>
__global__ void __launch_bounds__(kTWarps * 32) k_tree_force(sphh::TreeForceArgs a, PhysDev ph, SphenixDev x) {
  const int lane = threadIdx.x & 31;
  const int t = lane / kTreeTpp, sub = lane % kTreeTpp;
  const int32_t nl = *a.n_leaves;
  unsigned long long pair_acc = 0;
  for (int32_t li = next_group(a.work, lane); li < nl; li = next_group(a.work, lane)) {
    const TreeLeaf Lf = a.leaves[li];
    const int32_t t_lo = Lf.start, n_t = a.leaves[li + 1].start - Lf.start;
    const int sim = sim_of_cell(a.grid, a.n_sims, Lf.cell);
    const GridDev G = a.grid[sim];
    const TGeo g = leaf_geo(Lf, G);
    const float dt = kFl == kTGradient ? (float)(x.dt_dev != nullptr ? x.dt_dev[sim] : x.dt) : 0.0f;
    if (a.act != nullptr) {
      // masked loops: skip a group without a masked target
      bool any = false;
      for (int32_t k = lane; k < n_t; k += 32) any = any || a.act[a.tgt[t_lo + k]] != 0;
      if (!__any_sync(0xffffffffu, any)) continue;
    }
    for (int32_t t0 = 0; t0 < n_t; t0 += kTPer) {
      const bool valid = t0 + t < n_t;
      const int32_t ti = a.tgt[t_lo + (valid ? t0 + t : 0)];
      TFSums s;
      s.ax = s.ay = s.az = s.du = s.vsig = 0.f;
      s.npair = 0;
      const int lc = (int)a.list_cnt[ti];   // the target's packed list
      const bool fb = lc == kListFallback;  // written by k_tree_force_fb
      const float4 ei = kFl != kTMin ? a.fE[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      if (kFl == kTGradient) s.ay = ei.y;  // alpha_V,max starts at the target's
      const TRec hi = trec_head(a.rec, ti);
      const float Hi = hi.q0.w;
      const bool on = valid && !fb && (a.act == nullptr || a.act[ti] != 0);
      if (on) {
        const float4 reli = hi.q0;
        const int4 fi = hi.q1;
        const float3 pi = rel_to(g, reli, fi, kNoShift);
        const float4 vi = a.rec[4 * (int64_t)ti + 2];
        const float4 ci = a.rec[4 * (int64_t)ti + 3];
        const float2 di = make_float2(__int_as_float(hi.q1.w), __frcp_rn(hi.q0.w));
        // own reach: the list radius (a target without a complete list went
        // to the per-target kernel, kListFallback)
        const float C = a.lrad[ti];
        const float C2 = C * C;
        const uint32_t* lst = a.lists + (int64_t)ti * kTreeListTarget;
        for (int e = sub; e < lc; e += kTreeTpp) {
          const uint32_t je = lst[e];
          const int32_t j = unpack_j(je);
          if (j == ti) continue;
          const TRec hj = trec_head(a.rec, j);
          const float3 d = pair_vec(g, reli, fi, hj.q0, hj.q1, unpack_s(je));
          tforce_rec<kFl, K>(d.x, d.y, d.z, vi, ci, ei, Hi, di.y, di.x, a, j, hj, ph, s);
        }
        // reverse pairs beyond the own reach, split between the lanes (the
        // gradient pass reaches only H_i <= the own reach: none of them)
        if (kFl != kTGradient) {
          const int32_t r0 = a.rev_start[ti], r1 = a.rev_start[ti + 1];
          for (int32_t k = r0 + sub; k < r1; k += kTreeTpp) {
            const uint32_t je = a.rev[k];
            const int32_t j = unpack_j(je);
            const TRec hj = trec_head(a.rec, j);
            const float3 pj = rec_rel_to(g, hj, unpack_s(je));
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= C2)
              tforce_rec<kFl, K>(dx, dy, dz, vi, ci, ei, Hi, di.y, di.x, a, j, hj, ph, s);
          }
        }
      }
      s.ax = gsum(s.ax);
      s.ay = kFl == kTGradient ? gmax(s.ay) : gsum(s.ay);
      s.az = gsum(s.az);
      s.du = gsum(s.du);
      s.vsig = gmax(s.vsig);
      s.npair = gsumi(s.npair);
      if (on && sub == 0) {
        tforce_write<kFl>(a, x, dt, ti, Hi, ei, s);
        pair_acc += (unsigned long long)s.npair;
      }
    }
  }
  if (ph.count_pairs && a.pairs != nullptr) {
    unsigned long long v = pair_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(a.pairs, v);
  }
}

// ---- fallback: targets whose support outgrew the cells of their level ------
//
// One warp per queued target, all 32 lanes over its candidates: the 27 cells
// one level coarser (twice the side) around it, then coarser still while the
// solve keeps hitting the cap.  A target that needs more than its top cell
// sets SPH_ST_REBUILD: the top grid itself is too fine.

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int wsumi(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The 27 ranges of cell L (lanes 0..26) as a TRanges record.
__device__ __forceinline__ TRanges cell_ranges(const GridDev& G, const TreeLeaf& L,
                                               const uint64_t* __restrict__ skey,
                                               const int32_t* __restrict__ cell_start, int lane) {
  TRanges R;
  int32_t len = 0;
  R.lo = 0;
  R.sc = kNoShift;
  if (lane < 27) {
    const TreeRange t = neighbour_range(G, L, lane, skey, cell_start);
    R.lo = t.lo;
    len = t.hi - t.lo;
    R.sc = t.shift;
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  R.cum = incl - len;
  R.nsrc = __shfl_sync(0xffffffffu, incl, 31);
  return R;
}

template <int K>
__global__ void __launch_bounds__(kTWarps * 32) k_tree_density_fb(sphh::TreeDensityArgs a, PhysDev ph) {
  extern __shared__ __align__(16) unsigned char tsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const NewtonConst nwt = newton_const<K>(ph);
  unsigned char* base = tsm + (size_t)warp * kTWarpSmem;
  float4* spos = reinterpret_cast<float4*>(base);
  uint32_t* sidx = reinterpret_cast<uint32_t*>(spos + kTCap);
  TPrune* pr = reinterpret_cast<TPrune*>(sidx + kTCap + kTRows * 32 * 2);
  const int32_t nq = min(*a.fb_count, (int32_t)a.n_total);
  unsigned long long pair_acc = 0;
  for (int32_t q = next_group(a.fb_work, lane); q < nq; q = next_group(a.fb_work, lane)) {
    const int32_t qe = a.fb_list[q];
    const bool own = (qe & kFbOwnLevel) != 0;
    const int32_t ti = qe & kFbIndex;
    const uint64_t key = a.skey[ti];
    const GridDev G = a.grid[sim_of_cell(a.grid, a.n_sims, (int32_t)(key >> 30))];
    const float4 reli = a.rel[ti];
    const int4 fi = a.fine[ti];
    const float4 vi = a.vel4[ti];
    if (qe & kFbPassive) {
      // outside the mask: the reverse pairs of its current support H to the
      // masked particles, from the finest level whose 27 cells hold it (the
      // top cells hold every support)
      const float hp = a.hs[ti];
      const float H = KernT<K>::gamma * hp;
      int dp = (int)a.level[ti];
      TreeLeaf Lp = cell_at_depth(key, dp);
      TGeo gp = leaf_geo(Lp, G);
      while (dp > 0 && hp > h_cap<K>(gp.side_d, gp.L)) {
        --dp;
        Lp = cell_at_depth(key, dp);
        gp = leaf_geo(Lp, G);
      }
      const float3 pp = rel_to(gp, reli, fi, kNoShift);
      const TRanges Rr = cell_ranges(G, Lp, a.skey, a.cell_start, lane);
      prune_tables(a.skey, Rr, Lp.depth, lane, pr);
      const float cs = Lp.depth < kTreeDepth ? 0.5f * gp.side : gp.side;
      const float H2 = H * H;
      int nhp = 0;
      const int tot = prune_round(true, lane % kTreeTpp, lane, pp, H2 * (1.0f + 0x1p-10f), gp.side, cs, pr, nhp);
      for (int v0 = 0; v0 < tot; v0 += kTCap) {
        const int c = tstage_union(v0, tot, nhp, pr, lane, gp, a.rel, a.fine, spos, sidx);
        for (int k0 = 0; k0 < c; k0 += 32) {
          const int k = k0 + lane;
          bool want = false;
          uint64_t rec = 0;
          if (k < c) {
            const float r2 = r2_of(pp, spos[k]);
            const uint32_t je = sidx[k];
            const int32_t j = unpack_j(je);
            want = a.act[j] != 0 && want_reverse(a, ti, j, r2, H2, H, gp.side);
            rec = reverse_rec(j, ti, unpack_s(je));
          }
          emit_warp(a, want, rec, lane);
        }
        __syncwarp();
      }
      continue;
    }
    // a target queued from its group starts at its own level from its
    // starting h; one that hit its level's cap one level coarser from the
    // capped h of the first solve
    float h = own ? a.hs[ti] : a.h[a.perm[ti]];
    bool conv = false, atcap = true;
    int passes = 0, d = (int)a.level[ti] - (own ? 0 : 1);
    if (d < 0) {
      // already at its top cell: the caller rebuilds the top grid from twice
      // the capped h; the first solve's other outputs stand
      if (lane == 0) {
        atomicOr(a.status, SPH_ST_REBUILD);
        a.fb_level[ti] = 0;
        a.h[a.perm[ti]] = 2.0f * h;
      }
      __syncwarp();
      continue;
    }
    TGeo g;
    TRanges R;
    float3 pi;
    bool one_chunk = true;
    int nh = 0, total = 0;
    float Rp = 0.0f, cside = 0.0f;
    // the sources: the children of the 27 cells whose box lies within the
    // selection radius Rp (with a margin far above the rounding of r), staged
    // in chunks; Rp = min(cell side, 1.25 H) leaves room for the support to
    // grow, and a support beyond it selects again (H is warp-uniform)
#define TREE_FB_SELECT(Hsup)                                                                                   \
  if ((Hsup) > Rp) {                                                                                           \
    Rp = fminf(g.side, 1.25f * (Hsup));                                                                        \
    total = prune_round(true, lane % kTreeTpp, lane, pi, Rp * Rp * (1.0f + 0x1p-10f), g.side, cside, pr, nh); \
    one_chunk = total <= kTCap;                                                                                \
    if (one_chunk) tstage_union(0, total, nh, pr, lane, g, a.rel, a.fine, spos, sidx);                         \
  }
    for (; d >= 0; --d) {
      const TreeLeaf Lc = cell_at_depth(key, d);
      g = leaf_geo(Lc, G);
      R = cell_ranges(G, Lc, a.skey, a.cell_start, lane);
      pi = rel_to(g, reli, fi, kNoShift);
      const float hcap = h_cap<K>(g.side_d, g.L);
      prune_tables(a.skey, R, Lc.depth, lane, pr);
      cside = Lc.depth < kTreeDepth ? 0.5f * g.side : g.side;
      Rp = 0.0f;  // nothing selected at this level yet
      float hlo = 0.0f, hhi = INFINITY;
      int it = 0;
      if (h > hcap) h = hcap;
      bool done = false;
      while (!done) {  // warp-uniform: every lane holds the same reduced sums
        const float H = KernT<K>::gamma * h;
        TREE_FB_SELECT(H)
        const float Hinv = 1.0f / H;
        float Sw = 0.f, Sdw = 0.f;
        for (int v0 = 0; v0 < total; v0 += kTCap) {
          const int c = one_chunk ? total : tstage_union(v0, total, nh, pr, lane, g, a.rel, a.fine, spos, sidx);
          for (int k = lane; k < c; k += 32) tnewton_pair<K>(r2_of(pi, spos[k]), H, Hinv, Sw, Sdw);
          if (!one_chunk) __syncwarp();
        }
        Sw = wsum(Sw);
        Sdw = wsum(Sdw);
        ++passes;
        done = newton_update(Sw, Sdw, nwt, hcap, h, hlo, hhi, it, atcap, conv);
      }
      if (!atcap) break;
    }
    if (d < 0) {
      // even the top cell is too small: the caller rebuilds the top grid
      if (lane == 0) atomicOr(a.status, SPH_ST_REBUILD);
      d = 0;
    }
    // final pass at h, reverse pairs of this target
    const float H = KernT<K>::gamma * h;
    TREE_FB_SELECT(H)
#undef TREE_FB_SELECT
    const float Hinv = 1.0f / H;
    const float H2 = H * H;
    TDSums s;
    tds_zero(s);
    for (int v0 = 0; v0 < total; v0 += kTCap) {
      const int c = one_chunk ? total : tstage_union(v0, total, nh, pr, lane, g, a.rel, a.fine, spos, sidx);
      for (int k0 = 0; k0 < c; k0 += 32) {
        const int k = k0 + lane;
        bool want = false;
        uint64_t rec = 0;
        if (k < c) {
          const float4 pj = spos[k];
          const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (r2 < H2) {
            const uint32_t je = sidx[k];
            const int32_t j = unpack_j(je);
            tdens_pair<K>(dx, dy, dz, vi, a.vel4[j], pj.w, H, Hinv, s);
            want = want_reverse(a, ti, j, r2, H2, H, g.side);
            rec = reverse_rec(j, ti, unpack_s(je));
          }
        }
        emit_warp(a, want, rec, lane);
      }
      if (!one_chunk) __syncwarp();
    }
    s.w = wsum(s.w);
    s.dw = wsum(s.dw);
    s.mw = wsum(s.mw);
    s.mdw = wsum(s.mdw);
    s.div = wsum(s.div);
    s.cx = wsum(s.cx);
    s.cy = wsum(s.cy);
    s.cz = wsum(s.cz);
    s.npair = wsumi(s.npair);
    if (lane == 0) {
      tdens_write<K>(a, ph, ti, h, s, vi.w, passes, !conv && !atcap);
      if (atcap) a.h[a.perm[ti]] = 2.0f * h;  // next starting guess
      a.fb_level[ti] = (int8_t)d;
      pair_acc += (unsigned long long)s.npair;
    }
    __syncwarp();
  }
  if (ph.count_pairs && lane == 0 && pair_acc) atomicAdd(a.pairs, pair_acc);
}

template <int kFl, int K>
__global__ void __launch_bounds__(kTWarps * 32) k_tree_force_fb(sphh::TreeForceArgs a, PhysDev ph, SphenixDev x) {
  const int lane = threadIdx.x & 31;
  const int32_t nq = min(*a.fb_count, (int32_t)a.n_total);
  unsigned long long pair_acc = 0;
  for (int32_t q = next_group(a.fb_work, lane); q < nq; q = next_group(a.fb_work, lane)) {
    const int32_t qe = a.fb_list[q];
    if (qe & kFbPassive) continue;  // outside the mask: no force
    const int32_t ti = qe & kFbIndex;
    const uint64_t key = a.skey[ti];
    const int sim = sim_of_cell(a.grid, a.n_sims, (int32_t)(key >> 30));
    const GridDev G = a.grid[sim];
    const TreeLeaf Lc = cell_at_depth(key, (int)a.fb_level[ti]);
    const TGeo g = leaf_geo(Lc, G);
    const float dt = kFl == kTGradient ? (float)(x.dt_dev != nullptr ? x.dt_dev[sim] : x.dt) : 0.0f;
    const TRec hi = trec_head(a.rec, ti);
    const float3 pi = rec_rel_to(g, hi, kNoShift);
    const float4 vi = a.rec[4 * (int64_t)ti + 2];
    const float4 ci = a.rec[4 * (int64_t)ti + 3];
    const float4 ei = kFl != kTMin ? a.fE[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 di = make_float2(__int_as_float(hi.q1.w), __frcp_rn(hi.q0.w));
    const float Hi = hi.q0.w;
    // own reach: the list radius, or the support where it outgrew the list
    // (both within the cell of the fallback level, whose 27 cells hold every
    // source closer than that); the sources beyond it with a larger support
    // sent their pairs as reverse pairs (each emitted from r >= the list radius)
    const float C = fmaxf(a.lrad[ti], Hi);
    const float C2 = C * C;
    TFSums s;
    s.ax = s.ay = s.az = s.du = s.vsig = 0.f;
    s.npair = 0;
    if (kFl == kTGradient) s.ay = ei.y;
    const float cside = Lc.depth < kTreeDepth ? 0.5f * g.side : g.side;
    const float Cb2 = C2 * (1.0f + 0x1p-10f);
    for (int r = 0; r < 27; ++r) {
      const TreeRange Rg = neighbour_range(G, Lc, r, a.skey, a.cell_start);
      if (Rg.hi <= Rg.lo) continue;
      // the range's 8 children (contiguous in Morton order; a cell of the
      // deepest level is its own single child): lane c < 8 finds child c's
      // start and tests its box against the reach (with a margin far above
      // the rounding of r)
      int32_t c0 = Rg.lo;
      if (Lc.depth < kTreeDepth && lane > 0 && lane < 8) {
        const int sh = 3 * (kTreeDepth - Lc.depth - 1);
        const uint64_t base = (a.skey[Rg.lo] >> (sh + 3)) << (sh + 3);
        c0 = (int32_t)lower_bound64(a.skey, Rg.lo, Rg.hi, base + ((uint64_t)lane << sh));
      }
      if (Lc.depth >= kTreeDepth && lane > 0) c0 = Rg.hi;
      const int32_t nx = __shfl_down_sync(0xffffffffu, c0, 1);  // every lane takes part
      const int32_t c1 = lane < 7 ? nx : Rg.hi;
      const bool hit = lane < 8 && c1 > c0 && child_dist2(r * 8 + lane, g.side, cside, pi) < Cb2;
      unsigned hm = __ballot_sync(0xffffffffu, hit);
      while (hm) {
        const int ch = __ffs((int)hm) - 1;
        hm &= hm - 1u;
        const int32_t lo = __shfl_sync(0xffffffffu, c0, ch), hi = __shfl_sync(0xffffffffu, c1, ch);
        for (int32_t j = lo + lane; j < hi; j += 32) {
          if (j == ti) continue;
          const TRec hj = trec_head(a.rec, j);
          const float3 pj = rec_rel_to(g, hj, Rg.shift);
          const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
          if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < C2)
            tforce_rec<kFl, K>(dx, dy, dz, vi, ci, ei, Hi, di.y, di.x, a, j, hj, ph, s);
        }
      }
    }
    if (kFl != kTGradient) {
      const int32_t r0 = a.rev_start[ti], r1 = a.rev_start[ti + 1];
      for (int32_t k = r0 + lane; k < r1; k += 32) {
        const uint32_t je = a.rev[k];
        const int32_t j = unpack_j(je);
        const TRec hj = trec_head(a.rec, j);
        const float3 pj = rec_rel_to(g, hj, unpack_s(je));
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= C2)
          tforce_rec<kFl, K>(dx, dy, dz, vi, ci, ei, Hi, di.y, di.x, a, j, hj, ph, s);
      }
    }
    s.ax = wsum(s.ax);
    if (kFl == kTGradient) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s.ay = fmaxf(s.ay, __shfl_xor_sync(0xffffffffu, s.ay, o));
    } else {
      s.ay = wsum(s.ay);
    }
    s.az = wsum(s.az);
    s.du = wsum(s.du);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s.vsig = fmaxf(s.vsig, __shfl_xor_sync(0xffffffffu, s.vsig, o));
    s.npair = wsumi(s.npair);
    if (lane == 0) {
      tforce_write<kFl>(a, x, dt, ti, Hi, ei, s);
      pair_acc += (unsigned long long)s.npair;
    }
  }
  if (ph.count_pairs && a.pairs != nullptr && lane == 0 && pair_acc) atomicAdd(a.pairs, pair_acc);
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

__global__ void k_tree_mask(int64_t n, const int32_t* __restrict__ perm, const uint8_t* __restrict__ active,
                            uint8_t* __restrict__ out, int32_t* __restrict__ pre) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t v = k < n && active[perm[k]] != 0 ? 1 : 0;
    if (k < n) out[k] = v;
    if (pre != nullptr) pre[k] = v;
  }
}

static int tree_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

template <int K>
static cudaError_t launch_tree_density_k(const TreeDensityArgs& a, const PhysDev& ph, cudaStream_t st) {
  static int bps = 0;
  if (!bps) {
    cudaError_t e = cudaFuncSetAttribute(k_tree_density<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTDensSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tree_density<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTDensSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tree_density_fb<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTDensSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_tree_density<K, false>, kTWarps * 32, kTDensSmem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  const int64_t n = a.n_total;
  cudaError_t e = cudaMemsetAsync(a.rev_count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.fb_count, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.fb_work, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.rev_start, 0, sizeof(int32_t) * (n + 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.rev_fill, 0, sizeof(int32_t) * (n > 0 ? n : 1), st);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  if (a.act != nullptr)
    k_tree_density<K, true><<<a.num_sms * bps, kTWarps * 32, kTDensSmem, st>>>(a, ph);
  else
    k_tree_density<K, false><<<a.num_sms * bps, kTWarps * 32, kTDensSmem, st>>>(a, ph);
  k_tree_density_fb<K><<<a.num_sms * bps, kTWarps * 32, kTDensSmem, st>>>(a, ph);
  e = scan_exclusive_host_n(a.rev_start, n + 1, a.scan_tmp, st);
  if (e != cudaSuccess) return e;
  k_rev_scatter<<<a.num_sms * 4, 256, 0, st>>>(a.rev_raw, a.rev_count, a.rev_cap, a.rev_start, a.rev_fill, a.rev);
  k_rev_sort<<<tree_blocks(n), 256, 0, st>>>(n, a.rev_start, a.rev);
  return cudaGetLastError();
}

template <int kFl, int K>
static cudaError_t launch_tree_force_k(const TreeForceArgs& a, const PhysDev& ph, const SphenixDev& x,
                                       cudaStream_t st) {
  static int bps = 0;
  if (!bps) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_tree_force<kFl, K>, kTWarps * 32, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.fb_work, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_tree_force<kFl, K><<<a.num_sms * bps, kTWarps * 32, 0, st>>>(a, ph, x);
  k_tree_force_fb<kFl, K><<<a.num_sms * bps, kTWarps * 32, 0, st>>>(a, ph, x);
  return cudaGetLastError();
}

template <int kFl>
static cudaError_t launch_tree_force_fl(const TreeForceArgs& a, const PhysDev& ph, const SphenixDev& x,
                                        cudaStream_t st) {
  switch (ph.kernel) {
    case kKernQuartic:
      return launch_tree_force_k<kFl, kKernQuartic>(a, ph, x, st);
    case kKernWendlandC2:
      return launch_tree_force_k<kFl, kKernWendlandC2>(a, ph, x, st);
    default:
      return launch_tree_force_k<kFl, kKernCubic>(a, ph, x, st);
  }
}

cudaError_t launch_tree_sphenix_force(const TreeForceArgs& a, const PhysDev& ph, const SphenixDev& x,
                                      cudaStream_t st) {
  if (a.fE == nullptr) return cudaErrorInvalidValue;
  return launch_tree_force_fl<kTSphenix>(a, ph, x, st);
}

cudaError_t launch_tree_sphenix_gradient(const TreeForceArgs& a, const PhysDev& ph, const SphenixDev& x,
                                         cudaStream_t st) {
  if (a.fE == nullptr || a.alpha_c_out == nullptr) return cudaErrorInvalidValue;
  return launch_tree_force_fl<kTGradient>(a, ph, x, st);
}

cudaError_t launch_tree_density(const TreeDensityArgs& a, const PhysDev& ph, cudaStream_t st) {
  switch (ph.kernel) {
    case kKernQuartic:
      return launch_tree_density_k<kKernQuartic>(a, ph, st);
    case kKernWendlandC2:
      return launch_tree_density_k<kKernWendlandC2>(a, ph, st);
    default:
      return launch_tree_density_k<kKernCubic>(a, ph, st);
  }
}

cudaError_t launch_tree_force(const TreeForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  return launch_tree_force_fl<kTMin>(a, ph, SphenixDev{}, st);
}

cudaError_t launch_tree_limit(const TreeForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  if (a.fE == nullptr || a.bins_out == nullptr) return cudaErrorInvalidValue;
  return launch_tree_force_fl<kTLimit>(a, ph, SphenixDev{}, st);
}

cudaError_t launch_tree_wake(const TreeForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  if (a.fE == nullptr || a.act == nullptr || a.wake == nullptr) return cudaErrorInvalidValue;
  return launch_tree_force_fl<kTWake>(a, ph, SphenixDev{}, st);
}

cudaError_t launch_tree_mask(int64_t n, const int32_t* perm, const uint8_t* active, uint8_t* out, int32_t* pre,
                             int32_t* tmp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_tree_mask<<<tree_blocks(n + 1), 256, 0, st>>>(n, perm, active, out, pre);
  if (pre != nullptr) {
    const cudaError_t e = scan_exclusive_host_n(pre, n + 1, tmp, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace sphh
