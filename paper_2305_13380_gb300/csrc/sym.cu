// sym.cu -- the force loop with each pair evaluated once (Sec. 2.1: the pair
// terms of the symmetrised equations of motion are antisymmetric, so one
// evaluation serves both particles), for the "Minimal" flavour with the cubic
// spline on the uniform grid (SPH_FLAG_SYMMETRIC).
//
// Phase 1, k_force_sym: the blocks, rounds and lanes of k_force_min, but the
// density published only the sources later in sorted order (j > i), so each
// pair within reach is met once.  The target keeps its own side and emits the
// partner's side as a record (receiver j, source i, a_j, du_j/dt, v_sig):
//   B      = [P~_i t_i + P~_j t_j + nu/2 (F~_i t_i + F~_j t_j)] / r
//   a_i   += m_j B x_ij                a_j   -= m_i B x_ij
//   du_i  -= m_j/r [P~_i t_i + nu/4 F] v_ij . x_ij
//   du_j  -= m_i/r [P~_j t_j + nu/4 F] v_ij . x_ij
// (F = F~_i t_i + F~_j t_j; the factors and t(q) as in k_force_min).  Each
// warp reserves one record slot per list entry of its round with one atomic
// (entries beyond reach leave holes marked with receiver -1); lanes without a
// list take a slot per record.  Record order is not deterministic.
// Phase 2: counts per receiver are scanned, the records are scattered into
// per-receiver segments, and k_sym_reduce sorts each segment by source before
// adding it to the receiver's own sums, so the result does not depend on the
// order of the atomics and a simulation's result is the same alone or in a
// pool (sources are compared by sorted index, which keeps its order there).
// Blocks whose neighbourhood exceeds the staging buffer are done in place, one
// lane per target over the 27 cells read from global memory.
#include "blocks.cuh"
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "stencil.cuh"

namespace sphk {

constexpr float kSymKappa = 15.278874536821951f;  // 48 / pi
constexpr int kSymCap = kBlkStageCap;
constexpr int kSymListCap = 48;  // the density's published region
constexpr int kSymSeg = 64;      // largest per-receiver segment the reduction sorts

struct SymTarget {
  float x, y, z, Hinv, vx, vy, vz, m, P, F, c, B, rho;
  int32_t ti;
};

struct SymSums {
  float ax, ay, az, du, vsig;
  int npair;
};

// The pair (target T, source j at A, V, C, rho_j): the target's side into s,
// the partner's side returned (a_j in ax, ay, az, du_j in du, v_sig,ij) when
// the pair is within reach.
__device__ __forceinline__ bool sym_pair(const SymTarget& T, const float4& A, const float4& V, const float4& C,
                                         float rho_j, float beta, SymSums& s, float4& pa, float& pvs) {
  const float dx = T.x - A.x, dy = T.y - A.y, dz = T.z - A.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  const float qi = r * T.Hinv, qj = r * A.w;
  const float ai = __saturatef(1.0f - qi), bi = __saturatef(fmaf(-2.0f, qi, 1.0f));
  const float aj = __saturatef(1.0f - qj), bj = __saturatef(fmaf(-2.0f, qj, 1.0f));
  const float ti = fmaf(ai, ai, -bi * bi), tj = fmaf(aj, aj, -bj * bj);
  const float vx = T.vx - V.x, vy = T.vy - V.y, vz = T.vz - V.z;
  const float vdotx = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
  const float mu = fminf(vdotx, 0.0f) * rinv;
  const float vs = fmaf(-beta, mu, T.c + C.z);
  const float nu2 = __fdividef(-(T.B + C.w) * mu * vs, T.rho + rho_j);
  const float piT = T.P * ti, pjT = C.x * tj;
  const float Ft = fmaf(T.F, ti, C.y * tj);
  const float Bk = rinv * fmaf(nu2, Ft, piT + pjT);
  const float mj = V.w * Bk, mi = T.m * Bk;
  s.ax = fmaf(mj, dx, s.ax);
  s.ay = fmaf(mj, dy, s.ay);
  s.az = fmaf(mj, dz, s.az);
  const float hn = 0.5f * nu2;
  s.du = fmaf(-V.w * rinv * fmaf(hn, Ft, piT), vdotx, s.du);
  const bool in = ti + tj > 0.0f;
  s.vsig = in ? fmaxf(s.vsig, vs) : s.vsig;
  s.npair += in ? 2 : 0;
  pa = make_float4(-mi * dx, -mi * dy, -mi * dz, -T.m * rinv * fmaf(hn, Ft, pjT) * vdotx);
  pvs = vs;
  return in;
}

// Emits the partner's side of a pair (lanes of the current active set).
__device__ __forceinline__ void sym_emit(const sphh::SymArgs& y, bool in, int32_t recv, int32_t src,
                                         const float4& pa, float pvs, int lane) {
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, in);
  if (!in) return;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(y.counter, __popc(m));
  base = __shfl_sync(m, base, leader);
  const int64_t pos = (int64_t)base + __popc(m & ((1u << lane) - 1u));
  if (pos < y.cap) {
    y.rec_a[pos] = pa;
    y.rec_b[pos] = make_int2(__float_as_int(pvs), src);
    y.recv[pos] = recv;
    atomicAdd(y.cnt + recv, 1);
  } else {
    atomicOr(y.status, SPH_ST_CAPACITY);
  }
}

__device__ __forceinline__ void sym_write(const sphh::ForceArgs& a, int32_t ti, const SymSums& s) {
  const int32_t p = a.perm[ti];
  a.ax[p] = s.ax;
  a.ay[p] = s.ay;
  a.az[p] = s.az;
  a.du_dt[p] = s.du;
  a.v_sig[p] = s.vsig;
}

// A target of a block whose neighbourhood does not fit the staging buffer:
// its 27 cells straight from the sorted copies (positions relative to the
// target's cell), sources later in sorted order only.
__device__ __forceinline__ void sym_global_target(const sphh::ForceArgs& a, const sphh::SymArgs& y,
                                                  const NbLane& nb, const SymTarget& T, float half_alpha,
                                                  float beta, bool valid, int lane, SymSums& s) {
  for (int c = 0; c < 27; ++c) {
    const int32_t st = __shfl_sync(0xffffffffu, nb.start, c);
    const int32_t len = __shfl_sync(0xffffffffu, nb.len, c);
    const float ox = __shfl_sync(0xffffffffu, nb.ox, c), oy = __shfl_sync(0xffffffffu, nb.oy, c),
                oz = __shfl_sync(0xffffffffu, nb.oz, c);
    if (!valid) continue;
    for (int32_t j = st; j < st + len; ++j) {
      if (j <= T.ti) continue;
      const float4 A0 = a.fA[j];
      const float4 C0 = a.fC[j];
      const float2 D = a.fD[j];
      const float h2 = D.y * D.y;
      const float kap = kSymKappa * h2 * h2;
      const float4 A = make_float4(A0.x + ox, A0.y + oy, A0.z + oz, D.y);
      const float4 C = make_float4(kap * C0.x, kap * C0.y, C0.z, half_alpha * C0.w);
      float4 pa;
      float pvs;
      const bool in = sym_pair(T, A, a.fB[j], C, D.x, beta, s, pa, pvs);
      sym_emit(y, in, j, T.ti, pa, pvs, lane);
    }
  }
}

template <bool kCount>
__global__ void __launch_bounds__(kBlkThreads, 2) k_force_sym(sphh::ForceArgs a, sphh::SymArgs y, PhysDev ph) {
  extern __shared__ __align__(16) unsigned char ssm_raw[];
  float4* sA = reinterpret_cast<float4*>(ssm_raw);  // (x, y, z, 1/H)
  float4* sB = sA + kSymCap;                        // (vx, vy, vz, m)
  float4* sC = sB + kSymCap;                        // (P~, F~, c, B~)
  float* sR = reinterpret_cast<float*>(sC + kSymCap);
  int32_t* sJ = reinterpret_cast<int32_t*>(sR + kSymCap);  // sorted index
  StageTable& T = *reinterpret_cast<StageTable*>(sJ + kSymCap);
  BlockTargets& BT = *reinterpret_cast<BlockTargets*>(&T + 1);
  uint16_t* tgt_slot = reinterpret_cast<uint16_t*>(&BT + 1);
  uint8_t* tgt_cell = reinterpret_cast<uint8_t*>(tgt_slot + kSymCap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t total = a.misc_ro[kTotalBlocks];
  const float half_alpha = 0.5f * ph.alpha_v, beta = ph.beta_v;
  unsigned long long pair_acc = 0;

  for (int32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const BlockGeom g = block_geom(a.grid, a.n_sims, b);
    const int32_t nsrc = build_stage_table(g, a.cell_start, T);
    if (nsrc > kSymCap) {
      // one warp per cell of the block, one lane per target
      int tx, ty, tz;
      if (warp_cell(g, warp, tx, ty, tz)) {
        const int32_t nc = g.G.n_c;
        const int32_t cx = g.c0x + tx, cy = g.c0y + ty, cz = g.c0z + tz;
        const int32_t cid = g.G.cell_base + cx + nc * (cy + nc * cz);
        const int32_t ts = a.cell_start[cid], te = a.cell_start[cid + 1];
        const NbLane nb = neighbour_lane(lane, g.G.cell_base, cx, cy, cz, nc, g.G.cell_f, a.cell_start);
        for (int32_t t0 = ts; t0 < te; t0 += 32) {
          const int32_t ti = t0 + lane;
          const bool valid = ti < te;
          const int32_t tl = valid ? ti : ts;
          SymTarget Tg;
          {
            const float4 A = a.fA[tl], V = a.fB[tl], C = a.fC[tl];
            const float2 D = a.fD[tl];
            const float h2 = D.y * D.y, kap = kSymKappa * h2 * h2;
            Tg.x = A.x; Tg.y = A.y; Tg.z = A.z; Tg.Hinv = D.y;
            Tg.vx = V.x; Tg.vy = V.y; Tg.vz = V.z; Tg.m = V.w;
            Tg.P = kap * C.x; Tg.F = kap * C.y; Tg.c = C.z; Tg.B = half_alpha * C.w;
            Tg.rho = D.x;
            Tg.ti = tl;
          }
          SymSums s;
          s.ax = s.ay = s.az = s.du = s.vsig = 0.0f;
          s.npair = 0;
          sym_global_target(a, y, nb, Tg, half_alpha, beta, valid, lane, s);
          if (valid) {
            sym_write(a, ti, s);
            if (kCount) pair_acc += (unsigned long long)s.npair;
          }
        }
      }
      __syncthreads();
      continue;
    }
    build_targets<kKernCubic>(g, T, BT, tgt_slot, tgt_cell, nullptr, ph.lanes);  // ends with a barrier
    for (int32_t v = threadIdx.x; v < nsrc; v += kBlkThreads) {
      const int k = staged_cell_of(T, v);
      float ox, oy, oz;
      staged_offset(g, k, ox, oy, oz);
      const int32_t j = T.gstart[k] + (v - T.start[k]);
      const float4 A = a.fA[j];
      const float4 C = a.fC[j];
      const float2 D = a.fD[j];
      const float h2 = D.y * D.y;
      const float kap = kSymKappa * h2 * h2;
      sA[v] = make_float4(A.x + ox, A.y + oy, A.z + oz, D.y);
      sB[v] = a.fB[j];
      sC[v] = make_float4(kap * C.x, kap * C.y, C.z, half_alpha * C.w);
      sR[v] = D.x;
      sJ[v] = j;
    }
    __syncthreads();

    const int tpp = BT.tpp, lg = BT.lg, per = BT.per;
    const int sub = lane & (tpp - 1);
    for (int rd = warp; rd < BT.rounds; rd = next_round(BT, lane)) {
      const int t = lane >> lg;
      const int32_t e_t = rd * per + t;
      const bool valid = (t < per) && (e_t < BT.n);
      int slot = 0, kc = BT.cell_k[0];
      if (valid) {
        slot = tgt_slot[e_t];
        kc = BT.cell_k[tgt_cell[e_t]];
      }
      const int32_t ti = T.gstart[kc] + (slot - T.start[kc]);
      int cnt = valid ? 0xffff : 0;
      const uint16_t* lst = nullptr;
      if (valid && a.lists != nullptr) {
        const int64_t col = (int64_t)ti * 4 + sub;
        cnt = (int)a.list_cnt[col];
        lst = a.lists + col * kListRegion;
      }
      SymTarget Tg;
      {
        const float4 A = sA[slot], V = sB[slot], C = sC[slot];
        Tg.x = A.x; Tg.y = A.y; Tg.z = A.z; Tg.Hinv = A.w;
        Tg.vx = V.x; Tg.vy = V.y; Tg.vz = V.z; Tg.m = V.w;
        Tg.P = C.x; Tg.F = C.y; Tg.c = C.z; Tg.B = C.w;
        Tg.rho = sR[slot];
        Tg.ti = ti;
      }
      SymSums s;
      s.ax = s.ay = s.az = s.du = s.vsig = 0.0f;
      s.npair = 0;
      // one record slot per list entry, reserved with one atomic per warp;
      // entries beyond reach leave a hole (receiver -1)
      const int n_list = (valid && cnt <= kSymListCap) ? cnt : 0;
      int ex = n_list;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, ex, o);
        if (lane >= o) ex += u;
      }
      const int w_total = __shfl_sync(0xffffffffu, ex, 31);
      int base = 0;
      if (lane == 0 && w_total > 0) base = atomicAdd(y.counter, w_total);
      base = __shfl_sync(0xffffffffu, base, 0);
      const int64_t my0 = (int64_t)base + ex - n_list;
      if (n_list > 0 && my0 + n_list > y.cap) atomicOr(y.status, SPH_ST_CAPACITY);
      if (n_list > 0 && my0 + n_list <= y.cap) {
        // the upper list: every entry is later in sorted order
        for (int e = 0; e < n_list; ++e) {
          const int k = lst[e];
          float4 pa;
          float pvs;
          const bool in = sym_pair(Tg, sA[k], sB[k], sC[k], sR[k], beta, s, pa, pvs);
          const int32_t j = sJ[k];
          y.rec_a[my0 + e] = pa;
          y.rec_b[my0 + e] = make_int2(__float_as_int(pvs), ti);
          y.recv[my0 + e] = in ? j : -1;
          if (in) atomicAdd(y.cnt + j, 1);
        }
      } else if (valid && cnt > kSymListCap) {
        // no list, or the density list overflowed: the runs, later sources only
        const int tx = kc % g.ex - 1, ty = (kc / g.ex) % g.ey - 1, tz = kc / (g.ex * g.ey) - 1;
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
          for (int32_t k = A0 + sub; k < B0; k += tpp) {
            if (sJ[k] <= ti) continue;
            float4 pa;
            float pvs;
            const bool in = sym_pair(Tg, sA[k], sB[k], sC[k], sR[k], beta, s, pa, pvs);
            sym_emit(y, in, sJ[k], ti, pa, pvs, lane);
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int o = 1; o < 4; o <<= 1) {
        if (o < tpp) {
          s.ax += __shfl_xor_sync(0xffffffffu, s.ax, o);
          s.ay += __shfl_xor_sync(0xffffffffu, s.ay, o);
          s.az += __shfl_xor_sync(0xffffffffu, s.az, o);
          s.du += __shfl_xor_sync(0xffffffffu, s.du, o);
          s.vsig = fmaxf(s.vsig, __shfl_xor_sync(0xffffffffu, s.vsig, o));
          if (kCount) s.npair += __shfl_xor_sync(0xffffffffu, s.npair, o);
        }
      }
      if (valid && sub == 0) {
        sym_write(a, ti, s);
        if (kCount) pair_acc += (unsigned long long)s.npair;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (kCount && a.pairs != nullptr) {
    unsigned long long v = pair_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(a.pairs, v);
  }
}

constexpr size_t kSymSmem = (size_t)kSymCap * (3 * sizeof(float4) + sizeof(float) + sizeof(int32_t)) +
                            sizeof(StageTable) + sizeof(BlockTargets) +
                            (size_t)kSymCap * (sizeof(uint16_t) + sizeof(uint8_t));

// Exclusive scan of the per-receiver counts (n entries) into off[0..n]:
// tiles of kScanItems, their sums scanned by one block, then added back.
constexpr int kSymScanThreads = 1024;
constexpr int kSymScanItems = 4 * kSymScanThreads;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    sh[lane] = w;
  }
  __syncthreads();
  const int32_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kSymScanThreads) k_sym_scan_tiles(int64_t n, const int32_t* __restrict__ cnt,
                                                                  int32_t* __restrict__ off,
                                                                  int32_t* __restrict__ tile_sum) {
  __shared__ int32_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kSymScanItems + 4 * threadIdx.x;
  int32_t v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = base + q < n ? cnt[base + q] : 0;
  const int32_t t = v[0] + v[1] + v[2] + v[3];
  int32_t total;
  int32_t run = block_excl_scan(t, sh, total);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (base + q < n) off[base + q] = run;
    run += v[q];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kSymScanThreads) k_sym_scan_sums(int32_t n_tiles, int32_t* __restrict__ tile_sum) {
  __shared__ int32_t sh[32];
  int32_t carry = 0;
  for (int32_t t0 = 0; t0 < n_tiles; t0 += kSymScanThreads) {
    const int32_t i = t0 + threadIdx.x;
    const int32_t v = i < n_tiles ? tile_sum[i] : 0;
    int32_t total;
    const int32_t ex = block_excl_scan(v, sh, total);
    if (i < n_tiles) tile_sum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) tile_sum[n_tiles] = carry;
}

__global__ void k_sym_scan_add(int64_t n, int32_t* __restrict__ off, const int32_t* __restrict__ tile_sum,
                               int32_t n_tiles) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == n) off[n] = tile_sum[n_tiles];
    else off[i] += tile_sum[i / kSymScanItems];
  }
}

// Record r into its receiver's segment (slot order within a segment is not
// deterministic; the reduction sorts it).
__global__ void k_sym_scatter(sphh::SymArgs y) {
  const int64_t n_rec = min((int64_t)*y.counter, y.cap);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rec; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = y.recv[r];
    if (j < 0) continue;  // a list entry beyond reach
    const int32_t p = y.off[j] + atomicAdd(y.cursor + j, 1);
    y.order[p] = (int32_t)r;
  }
}

// Receiver j: its segment in order of source (the sources of a segment are
// distinct: a pair is met once), summed onto the receiver's own sums.  Up to
// kSymSeg records are sorted by insertion; a longer segment (a wide support
// over a dense region) takes its records by repeated selection of the next
// source, slow but in the same order.
__global__ void k_sym_reduce(sphh::ForceArgs a, sphh::SymArgs y, int64_t n) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s0 = y.off[j], len = y.off[j + 1] - s0;
    if (len == 0) continue;
    const int32_t p = a.perm[j];
    if (len > kSymSeg) {
      float ax = a.ax[p], ay = a.ay[p], az = a.az[p], du = a.du_dt[p], vs = a.v_sig[p];
      int32_t prev = -1;
      for (int e = 0; e < len; ++e) {
        int32_t best = 0x7fffffff, bi = -1;
        for (int q = 0; q < len; ++q) {
          const int32_t r = y.order[s0 + q];
          const int32_t k = y.rec_b[r].y;
          if (k > prev && k < best) {
            best = k;
            bi = r;
          }
        }
        if (bi < 0) break;
        const float4 ra = y.rec_a[bi];
        ax += ra.x;
        ay += ra.y;
        az += ra.z;
        du += ra.w;
        vs = fmaxf(vs, __int_as_float(y.rec_b[bi].x));
        prev = best;
      }
      a.ax[p] = ax;
      a.ay[p] = ay;
      a.az[p] = az;
      a.du_dt[p] = du;
      a.v_sig[p] = vs;
      continue;
    }
    int32_t idx[kSymSeg], key[kSymSeg];
    for (int e = 0; e < len; ++e) {
      const int32_t r = y.order[s0 + e];
      const int32_t k = y.rec_b[r].y;
      int q = e;
      while (q > 0 && key[q - 1] > k) {
        key[q] = key[q - 1];
        idx[q] = idx[q - 1];
        --q;
      }
      key[q] = k;
      idx[q] = r;
    }
    float ax = a.ax[p], ay = a.ay[p], az = a.az[p], du = a.du_dt[p], vs = a.v_sig[p];
    for (int e = 0; e < len; ++e) {
      const float4 ra = y.rec_a[idx[e]];
      ax += ra.x;
      ay += ra.y;
      az += ra.z;
      du += ra.w;
      vs = fmaxf(vs, __int_as_float(y.rec_b[idx[e]].x));
    }
    a.ax[p] = ax;
    a.ay[p] = ay;
    a.az[p] = az;
    a.du_dt[p] = du;
    a.v_sig[p] = vs;
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int grid_sym(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

int64_t sym_tiles(int64_t n) { return (n + kSymScanItems - 1) / kSymScanItems; }

cudaError_t launch_force_sym(const ForceArgs& a, const SymArgs& y, const PhysDev& ph, int64_t n, cudaStream_t st) {
  static int bps = 0;
  if (!bps) {
    cudaError_t e = cudaFuncSetAttribute(k_force_sym<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSymSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_force_sym<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSymSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_force_sym<false>, kBlkThreads, kSymSmem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  cudaError_t e = cudaMemsetAsync(y.counter, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(y.cnt, 0, sizeof(int32_t) * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(y.cursor, 0, sizeof(int32_t) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  if (ph.count_pairs)
    k_force_sym<true><<<a.num_sms * bps, kBlkThreads, kSymSmem, st>>>(a, y, ph);
  else
    k_force_sym<false><<<a.num_sms * bps, kBlkThreads, kSymSmem, st>>>(a, y, ph);
  if (n > 0) {
    const int64_t tiles = sym_tiles(n);
    k_sym_scan_tiles<<<(int)tiles, kSymScanThreads, 0, st>>>(n, y.cnt, y.off, y.tile_sum);
    k_sym_scan_sums<<<1, kSymScanThreads, 0, st>>>((int32_t)tiles, y.tile_sum);
    k_sym_scan_add<<<grid_sym(n + 1, 256), 256, 0, st>>>(n, y.off, y.tile_sum, (int32_t)tiles);
    k_sym_scatter<<<a.num_sms * 8, 256, 0, st>>>(y);
    k_sym_reduce<<<grid_sym(n, 128), 128, 0, st>>>(a, y, n);
  }
  return cudaGetLastError();
}

}  // namespace sphh
