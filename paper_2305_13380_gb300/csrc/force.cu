// force.cu -- the SPH force loop (Sec. 3.2): pressure gradient of the
// "Minimal" density-energy equations of motion, artificial viscosity with the
// Balsara switch, du/dt and the signal velocity.
//
// k_force: the block layout of the density loop (blocks.cuh) with tpp lanes
// per target.  A filter pass keeps, per lane, the staged sources with
// r_ij < max(H_i, H_j), j != i (the force neighbour set); the pair pass then
// walks only that list.  Per pair, with x_ij = x_i - x_j, v_ij = v_i - v_j,
// and G = g(q) / H^5 (so that grad_i W(r_ij, h) = G x_ij) evaluated once with
// h_i and once with h_j:
//   mu     = min(v_ij . x_ij, 0) / r
//   vsig   = c_i + c_j - beta mu
//   nu     = -alpha_V (B_i + B_j)/2 mu vsig / ((rho_i + rho_j)/2)
//   a_i   -= m_j [ fP_i G_i + fP_j G_j + nu/2 (f_i G_i + f_j G_j) ] x_ij
//   du_i  += m_j [ fP_i G_i + nu/4 (f_i G_i + f_j G_j) ] v_ij . x_ij
// with fP = f P / rho^2; v_sig,i is the maximum of vsig over the list.
// Blocks whose neighbourhood does not fit are done by k_force_overflow.
//
// The SPHENIX flavour (Sec. 3.3) runs the same kernels with a fifth record
// per source, E = (u, alpha_V, P, alpha_c):
//  - kFlSphenix, the force: alpha_V (B_i + B_j)/2 becomes
//    (alpha_V,i + alpha_V,j)/2 (B_i + B_j)/2 (eq. "av_ij"), and du_i gains the
//    conduction term (eq. "art_cond") over the same pairs,
//      alpha_c,ij v_c,ij m_j (u_i - u_j) r (f_i G_i + f_j G_j) / (rho_i + rho_j),
//    alpha_c,ij = (P_i alpha_c,i + P_j alpha_c,j) / (P_i + P_j),
//    v_c,ij = |v_ij . x_ij| / r + sqrt(2 |P_i - P_j| / (rho_i + rho_j));
//  - kFlGradient, the gradient pass over r < H_i: lap u_i =
//    2 sum_j (m_j / rho_j)(u_i - u_j) G_i, v_c,i = max_j v_c,ij and the largest
//    alpha_V of the target and its neighbours, then the conduction parameter's
//    Euler step (eq. "artconddt") and its limiters (eqs. "condshocklimiter",
//    "conductionlimiter").
// The fifth record costs 16 bytes of shared memory per staged source, so the
// SPHENIX kernels stage at most 1200 sources per block, the most that keeps
// two blocks per SM (a 2.29-lattice-points-per-cell grid stages up to ~1050);
// larger neighbourhoods go to the overflow kernel.
#include "blocks.cuh"
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "stencil.cuh"

namespace sphk {

enum : int { kFlMinimal = 0, kFlSphenix = 1, kFlGradient = 2, kFlLimit = 3 };

template <int kFl, int K>
__host__ __device__ constexpr int force_cap() {
  return kFl == kFlMinimal ? stage_cap<K>() : (stage_cap<K>() < 1200 ? stage_cap<K>() : 1200);
}
template <int kFl>
__host__ __device__ constexpr size_t rec_bytes() {  // staged bytes per source
  return 3 * sizeof(float4) + sizeof(float2) + (kFl != kFlMinimal ? sizeof(float4) : 0);
}
constexpr int kFListCap = 48;
constexpr int kFListEager = 4;  // 16-byte list words loaded before the count is known
// per source: A (x, y, z, H), B (vx, vy, vz, m), C (fP, f, c, B), D (rho, 1/H),
// and for SPHENIX E (u, alpha_V, P, alpha_c)
template <int kFl, int K>
__host__ __device__ constexpr size_t force_blk_smem() {
  return (size_t)force_cap<kFl, K>() * rec_bytes<kFl>() + (size_t)kBlkWarps * kFListCap * 32 * sizeof(uint16_t) +
         sizeof(StageTable) + sizeof(BlockTargets) + (size_t)force_cap<kFl, K>() * (sizeof(uint16_t) + sizeof(uint8_t));
}
static_assert(2 * (force_blk_smem<kFlSphenix, kKernCubic>() + 1024) <= 228 * 1024, "two SPHENIX blocks per SM");
static_assert(2 * (force_blk_smem<kFlMinimal, kKernQuartic>() + 1024) <= 228 * 1024, "two quartic blocks per SM");
constexpr int kFOvfCap = 160;
template <int kFl>
__host__ __device__ constexpr size_t fovf_smem() {
  return (size_t)kWarpsPerBlock * kFOvfCap * rec_bytes<kFl>();
}

struct ForceSums {
  float ax, ay, az, du, vsig;
  int npair;
};

struct ForceTarget {
  float4 A, B, C, E;
  float2 D;
  float Hinv5;
};

__device__ __forceinline__ void fsums_zero(ForceSums& s) {
  s.ax = s.ay = s.az = s.du = s.vsig = 0.f;
  s.npair = 0;
}

template <int kFl, int K>
__device__ __forceinline__ void force_pair(const ForceTarget& T, const float4& Aj, const float4& Bj,
                                           const float4& Cj, const float2& Dj, const float4& Ej,
                                           const PhysDev& ph, bool counted, ForceSums& s) {
  if constexpr (kFl == kFlLimit) {
    // the first time-step limiter: the largest bin among the force pairs
    s.vsig = counted ? fmaxf(s.vsig, Ej.x) : s.vsig;
    s.npair += counted;
    return;
  }
  const float dx = T.A.x - Aj.x, dy = T.A.y - Aj.y, dz = T.A.z - Aj.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  const float Gi = kernel_g<K>(r * T.D.y, T.A.w * rinv) * T.Hinv5;
  const float vx = T.B.x - Bj.x, vy = T.B.y - Bj.y, vz = T.B.z - Bj.z;
  const float vdotx = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
  if constexpr (kFl == kFlGradient) {
    // zero beyond H_i (G_i = 0) and for the self pair (u_i - u_j = 0)
    s.ax = fmaf(__fdividef(Bj.w, Dj.x) * (T.E.x - Ej.x), Gi, s.ax);
    const float vc = fmaf(fabsf(vdotx), rinv, sqrtf(__fdividef(2.0f * fabsf(T.E.z - Ej.z), T.D.x + Dj.x)));
    s.vsig = counted ? fmaxf(s.vsig, vc) : s.vsig;
    s.ay = counted ? fmaxf(s.ay, Ej.y) : s.ay;
    s.npair += counted;
    return;
  }
  const float Hj2 = Dj.y * Dj.y;
  const float Gj = kernel_g<K>(r * Dj.y, Aj.w * rinv) * (Hj2 * Hj2 * Dj.y);
  const float mu = fminf(vdotx, 0.0f) * rinv;
  const float vs = fmaf(-ph.beta_v, mu, T.C.z + Cj.z);
  const float av = kFl == kFlSphenix ? 0.5f * (T.E.y + Ej.y) : ph.alpha_v;
  const float nu = __fdividef(-av * (T.C.w + Cj.w) * mu * vs, T.D.x + Dj.x);
  const float piG = T.C.x * Gi;
  const float visc = fmaf(T.C.y, Gi, Cj.y * Gj);
  const float sc = Bj.w * fmaf(0.5f * nu, visc, fmaf(Cj.x, Gj, piG));
  s.ax = fmaf(-sc, dx, s.ax);
  s.ay = fmaf(-sc, dy, s.ay);
  s.az = fmaf(-sc, dz, s.az);
  s.du = fmaf(Bj.w * fmaf(0.25f * nu, visc, piG), vdotx, s.du);
  if constexpr (kFl == kFlSphenix) {
    // conduction: zero beyond both supports (visc = 0) and for r = 0
    const float Ps = T.E.z + Ej.z, rs = T.D.x + Dj.x;
    const float ac = Ps > 0.0f ? __fdividef(fmaf(T.E.z, T.E.w, Ej.z * Ej.w), Ps) : 0.0f;
    const float vc = fmaf(fabsf(vdotx), rinv, sqrtf(__fdividef(2.0f * fabsf(T.E.z - Ej.z), rs)));
    s.du = fmaf(Bj.w * ac * vc * (T.E.x - Ej.x) * r, __fdividef(visc, rs), s.du);
  }
  s.vsig = counted ? fmaxf(s.vsig, vs) : s.vsig;
  s.npair += counted;
}

__device__ __forceinline__ void finish_target(ForceTarget& T) {
  const float h2 = T.D.y * T.D.y;
  T.Hinv5 = h2 * h2 * T.D.y;
}

// The gradient pass's result: the Euler step of eq. "artconddt" over dt,
//   alpha_c += dt [beta_c H lap_u / sqrt(u) - (alpha_c - alpha_c,min) v_c / H]
// (no source where u <= 0), limited to
// [alpha_c,min, alpha_c,max (1 - alpha_V,max,i / alpha_V,max)].
__device__ __forceinline__ void gradient_write(const sphh::ForceArgs& a, const SphenixDev& x, float dt, int32_t ti,
                                               const ForceTarget& T, const ForceSums& s) {
  const int32_t p = a.perm[ti];
  const float lap = 2.0f * s.ax;
  const float H = T.A.w, u = T.E.x, ac = T.E.w;
  const float src = u > 0.0f ? x.beta_c * H * lap / sqrtf(u) : 0.0f;
  const float rate = src - (ac - x.ac_min) * s.vsig / H;
  float an = fmaf(dt, rate, ac);
  an = fminf(an, x.ac_max * (1.0f - s.ay / x.av_max));
  an = fmaxf(an, x.ac_min);
  a.alpha_c_out[p] = an;
  if (a.lap_u != nullptr) a.lap_u[p] = lap;
}

// The limiter's result: a step at most 4 times the smallest neighbour step,
// i.e. at most two bins below the largest neighbour bin (the sums' v_sig
// field holds that largest bin).
__device__ __forceinline__ void limit_write(const sphh::ForceArgs& a, int32_t ti, const ForceTarget& T,
                                            const ForceSums& s) {
  const int own = (int)T.E.x, nb = (int)s.vsig - 2;
  a.bins_out[a.perm[ti]] = own > nb ? own : nb;
}

__device__ __forceinline__ float block_dt(const sphh::ForceArgs& a, const SphenixDev& x, int32_t b) {
  return (float)(x.dt_dev != nullptr ? x.dt_dev[sim_of_block(a.grid, a.n_sims, b)] : x.dt);
}

__device__ __forceinline__ void force_write(const sphh::ForceArgs& a, int32_t ti, const ForceSums& s) {
  const int32_t p = a.perm[ti];
  a.ax[p] = s.ax;
  a.ay[p] = s.ay;
  a.az[p] = s.az;
  a.du_dt[p] = s.du;
  a.v_sig[p] = s.vsig;
}

// The gradient pass's SPHENIX sums in the force sums' fields: ax = the
// Laplacian sum, ay = the largest alpha_V (a maximum), vsig = the largest
// v_c,ij.
template <int kFl>
__device__ __forceinline__ void fsums_add(ForceSums& s, const ForceSums& t) {
  s.ax += t.ax;
  s.ay = kFl == kFlGradient ? fmaxf(s.ay, t.ay) : s.ay + t.ay;
  s.az += t.az;
  s.du += t.du;
  s.vsig = fmaxf(s.vsig, t.vsig);
  s.npair += t.npair;
}

template <int kFl>
__device__ __forceinline__ void fcombine(ForceSums& s, int tpp) {
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    if (o < tpp) {
      s.ax += __shfl_xor_sync(0xffffffffu, s.ax, o);
      const float ay = __shfl_xor_sync(0xffffffffu, s.ay, o);
      s.ay = kFl == kFlGradient ? fmaxf(s.ay, ay) : s.ay + ay;
      s.az += __shfl_xor_sync(0xffffffffu, s.az, o);
      s.du += __shfl_xor_sync(0xffffffffu, s.du, o);
      s.vsig = fmaxf(s.vsig, __shfl_xor_sync(0xffffffffu, s.vsig, o));
      s.npair += __shfl_xor_sync(0xffffffffu, s.npair, o);
    }
  }
}

// The density loop's list of this lane for round rd (same build, same
// rounds): its count (0xffff if it overflowed or the lane has no target) and
// its entries as 16-byte words.  The first kFListEager words (which hold the
// typical list) are loaded without waiting on the count, so that they
// overlap other memory traffic; the rest only when the count needs them.
// Words beyond the count are never used.
__device__ __forceinline__ void fetch_list(const sphh::ForceArgs& a, const BlockTargets& BT,
                                           const StageTable& T, const uint16_t* tgt_slot,
                                           const uint8_t* tgt_cell, int rd, int lane, int& lc,
                                           uint4 (&w)[kFListCap / 8]) {
  const int t = lane >> BT.lg, sub = lane & (BT.tpp - 1);
  const int32_t e_t = rd * BT.per + t;
  lc = 0xffff;
  if (t >= BT.per || e_t >= BT.n) return;
  const int kc = BT.cell_k[tgt_cell[e_t]];
  const int32_t ti = T.gstart[kc] + (tgt_slot[e_t] - T.start[kc]);
  const int64_t col = (int64_t)ti * 4 + sub;
  lc = (int)a.list_cnt[col];
  const uint4* src = reinterpret_cast<const uint4*>(a.lists + (int64_t)ti * (4 * kListRegion) +
                                                    list_offset(a.list_cnt, ti, sub));
#pragma unroll
  for (int q = 0; q < kFListEager; ++q) w[q] = src[q];
#pragma unroll
  for (int q = kFListEager; q < kFListCap / 8; ++q)
    if (8 * q < lc && lc <= kFListCap) w[q] = src[q];
}

// The reach of a pair: r < max(H_i, H_j) for the force, r < H_i for the
// gradient pass.
template <int kFl>
__device__ __forceinline__ float reach(float Hi, float Hj) {
  return kFl == kFlGradient ? Hi : fmaxf(Hi, Hj);
}

template <int kFl, int K>
__global__ void __launch_bounds__(kBlkThreads, 2) k_force(sphh::ForceArgs a, PhysDev ph, SphenixDev x) {
  constexpr int kCap = force_cap<kFl, K>();
  constexpr bool kE = kFl != kFlMinimal;
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  float4* sA = reinterpret_cast<float4*>(fsm_raw);
  float4* sB = sA + kCap;
  float4* sC = sB + kCap;
  float4* sE = sC + kCap;  // SPHENIX only
  float2* sD = reinterpret_cast<float2*>(sC + (kE ? 2 : 1) * kCap);
  uint16_t* lj_all = reinterpret_cast<uint16_t*>(sD + kCap);
  StageTable& T = *reinterpret_cast<StageTable*>(lj_all + kBlkWarps * kFListCap * 32);
  BlockTargets& BT = *reinterpret_cast<BlockTargets*>(&T + 1);
  uint16_t* tgt_slot = reinterpret_cast<uint16_t*>(&BT + 1);
  uint8_t* tgt_cell = reinterpret_cast<uint8_t*>(tgt_slot + kCap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* lj = lj_all + warp * (kFListCap * 32);
  const int32_t total = a.misc_ro[kTotalBlocks];
  unsigned long long pair_acc = 0;

  for (int32_t b = blockIdx.x; b < total; b += gridDim.x) {
    if (a.blk_any != nullptr && a.blk_any[b] == 0) continue;  // no active target
    const BlockGeom g = block_geom(a.grid, a.n_sims, b);
    const int32_t nsrc = build_stage_table(g, a.cell_start, T);
    if (nsrc > kCap) {
      if (threadIdx.x == 0) a.overflow[atomicAdd(&a.misc[kNumOverflow], 1)] = b;
      __syncthreads();
      continue;
    }
    const float dt = kFl == kFlGradient ? block_dt(a, x, b) : 0.0f;
    // the targets' rounds first (they need only the table), so that each
    // warp's first list is in flight together with the staging loads
    build_targets<K>(g, T, BT, tgt_slot, tgt_cell, a.act, ph.lanes);  // ends with a barrier
    if (BT.n == 0) continue;  // a masked block without active targets
    const int tpp = BT.tpp, lg = BT.lg, per = BT.per;
    const int sub = lane & (tpp - 1);
    int pre_lc = 0xffff;
    uint4 pre[kFListCap / 8];
    if (a.lists != nullptr && warp < BT.rounds) fetch_list(a, BT, T, tgt_slot, tgt_cell, warp, lane, pre_lc, pre);
    for (int32_t v = threadIdx.x; v < nsrc; v += kBlkThreads) {
      const int k = staged_cell_of(T, v);
      float ox, oy, oz;
      staged_offset(g, k, ox, oy, oz);
      const int32_t j = T.gstart[k] + (v - T.start[k]);
      float4 p = a.fA[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      sA[v] = p;
      sB[v] = a.fB[j];
      sC[v] = a.fC[j];
      sD[v] = a.fD[j];
      if (kE) sE[v] = a.fE[j];
    }
    __syncthreads();

    for (int rd = warp; rd < BT.rounds; rd = next_round(BT, lane)) {
      const int t = lane >> lg;
      const int32_t e_t = rd * per + t;
      const bool valid = (t < per) && (e_t < BT.n);
      int self_slot = 0, kc = BT.cell_k[0];
      if (valid) {
        self_slot = tgt_slot[e_t];
        kc = BT.cell_k[tgt_cell[e_t]];
      }
      const int tx = kc % g.ex - 1, ty = (kc / g.ex) % g.ey - 1, tz = kc / (g.ex * g.ey) - 1;
      const int32_t ti = T.gstart[kc] + (self_slot - T.start[kc]);
      if (a.lists != nullptr && rd != warp) fetch_list(a, BT, T, tgt_slot, tgt_cell, rd, lane, pre_lc, pre);
      ForceTarget Tg;
      Tg.A = sA[self_slot];
      Tg.B = sB[self_slot];
      Tg.C = sC[self_slot];
      Tg.D = sD[self_slot];
      Tg.E = kE ? sE[self_slot] : make_float4(0.f, 0.f, 0.f, 0.f);
      finish_target(Tg);
      ForceSums s0, s1;
      fsums_zero(s0);
      fsums_zero(s1);
      if (kFl == kFlGradient) s0.ay = s1.ay = Tg.E.y;  // alpha_V,max starts at the target's
      // the density loop's list of this lane (same build, same rounds): all
      // sources within the cell size, a superset of the pairs in reach
      int cnt = -1;
      if (a.lists != nullptr && valid) {
        const int lc = pre_lc;
        if (lc <= kFListCap) {
#pragma unroll
          for (int e8 = 0; e8 < kFListCap; e8 += 8) {
            if (e8 < lc) {
              const uint4 v = pre[e8 >> 3];
              const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int e0 = e8 + 2 * q;
                if (e0 < lc) lj[e0 * 32 + lane] = (uint16_t)(w[q] & 0xffffu);
                if (e0 + 1 < lc) lj[(e0 + 1) * 32 + lane] = (uint16_t)(w[q] >> 16);
              }
            }
          }
          cnt = lc;
        }
      }
      if (valid && cnt < 0) {
        // own filter (no list, or the density list overflowed)
        cnt = 0;
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
#pragma unroll 4
          for (int32_t k = A0 + sub; k < B0; k += tpp) {
            const float4 Aj = sA[k];
            const float dx = Tg.A.x - Aj.x, dy = Tg.A.y - Aj.y, dz = Tg.A.z - Aj.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float Hm = reach<kFl>(Tg.A.w, Aj.w);
            if (r2 < Hm * Hm && k != self_slot) {
              if (cnt < kFListCap) lj[cnt * 32 + lane] = (uint16_t)k;
              ++cnt;
            }
          }
        }
      }
      if (valid && cnt <= kFListCap) {
        // pairs beyond reach add exactly zero; the self pair and pairs beyond
        // reach do not enter the maxima or the pair count
        int e = 0;
        for (; e + 1 < cnt; e += 2) {
          const int ka = lj[e * 32 + lane], kb = lj[(e + 1) * 32 + lane];
          const float4 Aa = sA[ka], Ab = sA[kb];
          const float dxa = Tg.A.x - Aa.x, dya = Tg.A.y - Aa.y, dza = Tg.A.z - Aa.z;
          const float dxb = Tg.A.x - Ab.x, dyb = Tg.A.y - Ab.y, dzb = Tg.A.z - Ab.z;
          const float r2a = fmaf(dxa, dxa, fmaf(dya, dya, dza * dza));
          const float r2b = fmaf(dxb, dxb, fmaf(dyb, dyb, dzb * dzb));
          const float Hma = reach<kFl>(Tg.A.w, Aa.w), Hmb = reach<kFl>(Tg.A.w, Ab.w);
          const float4 Ea = kE ? sE[ka] : Tg.E, Eb = kE ? sE[kb] : Tg.E;
          force_pair<kFl, K>(Tg, Aa, sB[ka], sC[ka], sD[ka], Ea, ph, r2a < Hma * Hma && ka != self_slot, s0);
          force_pair<kFl, K>(Tg, Ab, sB[kb], sC[kb], sD[kb], Eb, ph, r2b < Hmb * Hmb && kb != self_slot, s1);
        }
        if (e < cnt) {
          const int ka = lj[e * 32 + lane];
          const float4 Aa = sA[ka];
          const float dxa = Tg.A.x - Aa.x, dya = Tg.A.y - Aa.y, dza = Tg.A.z - Aa.z;
          const float r2a = fmaf(dxa, dxa, fmaf(dya, dya, dza * dza));
          const float Hma = reach<kFl>(Tg.A.w, Aa.w);
          const float4 Ea = kE ? sE[ka] : Tg.E;
          force_pair<kFl, K>(Tg, Aa, sB[ka], sC[ka], sD[ka], Ea, ph, r2a < Hma * Hma && ka != self_slot, s0);
        }
      } else if (valid) {
        // list overflow: walk the runs directly
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
          for (int32_t k = A0 + sub; k < B0; k += tpp) {
            const float4 Aj = sA[k];
            const float dx = Tg.A.x - Aj.x, dy = Tg.A.y - Aj.y, dz = Tg.A.z - Aj.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float Hm = reach<kFl>(Tg.A.w, Aj.w);
            if (r2 < Hm * Hm && k != self_slot)
              force_pair<kFl, K>(Tg, Aj, sB[k], sC[k], sD[k], kE ? sE[k] : Tg.E, ph, true, s0);
          }
        }
      }
      fsums_add<kFl>(s0, s1);
      fcombine<kFl>(s0, tpp);
      if (valid && sub == 0) {
        if (kFl == kFlGradient)
          gradient_write(a, x, dt, ti, Tg, s0);
        else if (kFl == kFlLimit)
          limit_write(a, ti, Tg, s0);
        else
          force_write(a, ti, s0);
        pair_acc += (unsigned long long)s0.npair;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (ph.count_pairs && a.pairs != nullptr) {
    unsigned long long v = pair_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(a.pairs, v);
  }
}

// ---------------------------------------------------------------------------
// k_force_min: the "Minimal" force with the cubic spline, the path of the
// plain and batched steps.  Same blocks, rounds, lanes and density lists as
// k_force, with the pair arithmetic reduced by folding the kernel gradient's
// constants into per-particle factors when the sources are staged.
//
// For the cubic spline, w'(q) = -(48/pi) [(1-q)_+^2 - (1-2q)_+^2], so
//   grad_i W(r_ij, h) = G x_ij,  G = -kappa t(q) / r,
//   kappa = (48/pi) / H^4,  t(q) = (1-q)_+^2 - (1-2q)_+^2 >= 0,
// and with the staged factors P~ = kappa f P / rho^2, F~ = kappa f and
// B~ = (alpha_V / 2) B the equations of k_force become
//   nu/2  = -(B~_i + B~_j) mu vsig / (rho_i + rho_j)
//   a_i  += m_j / r [P~_i t_i + P~_j t_j + nu/2 (F~_i t_i + F~_j t_j)] x_ij
//   du_i -= m_j / r [P~_i t_i + nu/4 (F~_i t_i + F~_j t_j)] v_ij . x_ij
// A pair beyond both supports has t_i = t_j = 0 and adds exactly zero, as
// does the target itself (r = 0, t = 0); neither enters v_sig,i or the pair
// count (t_i + t_j = 0).  So the lane walks its density list (all sources
// within one cell size) without testing the reach.  The list is read from
// global memory into registers, 16 bytes (8 entries) at a time with the next
// word in flight, so no shared memory is spent on lists and three blocks fit
// an SM.
// ---------------------------------------------------------------------------
constexpr float kKappaCubic = 15.278874536821951f;  // 48 / pi
constexpr int kMinBlocks = 3;

struct MinTarget {
  float x, y, z, Hinv, vx, vy, vz, P, F, c, B, rho;
};

struct MinSums {
  float ax, ay, az, du, vsig;
  int npair;
};

template <bool kCount>
__device__ __forceinline__ void min_pair(const MinTarget& T, const float4& A, const float4& V, const float4& C,
                                         float rho_j, float beta, MinSums& s) {
  const float dx = T.x - A.x, dy = T.y - A.y, dz = T.z - A.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  const float qi = r * T.Hinv, qj = r * A.w;
  // q >= 0, so max(1 - q, 0) and max(1 - 2q, 0) are saturations to [0, 1]
  const float ai = __saturatef(1.0f - qi), bi = __saturatef(fmaf(-2.0f, qi, 1.0f));
  const float aj = __saturatef(1.0f - qj), bj = __saturatef(fmaf(-2.0f, qj, 1.0f));
  const float ti = fmaf(ai, ai, -bi * bi), tj = fmaf(aj, aj, -bj * bj);
  const float vx = T.vx - V.x, vy = T.vy - V.y, vz = T.vz - V.z;
  const float vdotx = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
  const float mu = fminf(vdotx, 0.0f) * rinv;
  const float vs = fmaf(-beta, mu, T.c + C.z);
  const float nu2 = __fdividef(-(T.B + C.w) * mu * vs, T.rho + rho_j);
  const float piT = T.P * ti;
  const float Pt = fmaf(C.x, tj, piT);
  const float Ft = fmaf(T.F, ti, C.y * tj);
  const float mr = V.w * rinv;
  const float S = mr * fmaf(nu2, Ft, Pt);
  s.ax = fmaf(S, dx, s.ax);
  s.ay = fmaf(S, dy, s.ay);
  s.az = fmaf(S, dz, s.az);
  const float D = fmaf(0.5f * nu2, Ft, piT);
  s.du = fmaf(-mr * D, vdotx, s.du);
  const bool in = ti + tj > 0.0f;
  s.vsig = in ? fmaxf(s.vsig, vs) : s.vsig;
  if (kCount) s.npair += in ? 1 : 0;
}

// Staged slot of entry e (0..7) of a 16-byte list word.
__device__ __forceinline__ int list_entry(const uint4& w, int e) {
  const uint32_t v = e < 2 ? w.x : (e < 4 ? w.y : (e < 6 ? w.z : w.w));
  return (int)((e & 1) ? (v >> 16) : (v & 0xffffu));
}

template <bool kCount>
__global__ void __launch_bounds__(kBlkThreads, kMinBlocks) k_force_min(sphh::ForceArgs a, PhysDev ph) {
  constexpr int kCap = kBlkStageCap;
  constexpr int kSlots = kCap;
  extern __shared__ __align__(16) unsigned char msm_raw[];
  float4* sA = reinterpret_cast<float4*>(msm_raw);  // (x, y, z, 1/H)
  float4* sB = sA + kSlots;                         // (vx, vy, vz, m)
  float4* sC = sB + kSlots;                         // (P~, F~, c, B~)
  float* sR = reinterpret_cast<float*>(sC + kSlots);  // rho
  StageTable& T = *reinterpret_cast<StageTable*>(sR + kSlots);
  BlockTargets& BT = *reinterpret_cast<BlockTargets*>(&T + 1);
  uint16_t* tgt_slot = reinterpret_cast<uint16_t*>(&BT + 1);
  uint8_t* tgt_cell = reinterpret_cast<uint8_t*>(tgt_slot + kCap);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t total = a.misc_ro[kTotalBlocks];
  const float half_alpha = 0.5f * ph.alpha_v, beta = ph.beta_v;
  unsigned long long pair_acc = 0;

  for (int32_t b = blockIdx.x; b < total; b += gridDim.x) {
    if (a.blk_any != nullptr && a.blk_any[b] == 0) continue;  // no active target
    const BlockGeom g = block_geom(a.grid, a.n_sims, b);
    const int32_t nsrc = build_stage_table(g, a.cell_start, T);
    if (nsrc > kCap) {
      if (threadIdx.x == 0) a.overflow[atomicAdd(&a.misc[kNumOverflow], 1)] = b;
      __syncthreads();
      continue;
    }
    build_targets<kKernCubic>(g, T, BT, tgt_slot, tgt_cell, a.act, ph.lanes);  // ends with a barrier
    if (BT.n == 0) continue;
    for (int32_t v = threadIdx.x; v < nsrc; v += kBlkThreads) {
      const int k = staged_cell_of(T, v);
      float ox, oy, oz;
      staged_offset(g, k, ox, oy, oz);
      const int32_t j = T.gstart[k] + (v - T.start[k]);
      const float4 A = a.fA[j];
      const float4 C = a.fC[j];
      const float2 D = a.fD[j];
      const float h2 = D.y * D.y;
      const float kap = kKappaCubic * h2 * h2;
      sA[v] = make_float4(A.x + ox, A.y + oy, A.z + oz, D.y);
      sB[v] = a.fB[j];
      sC[v] = make_float4(kap * C.x, kap * C.y, C.z, half_alpha * C.w);
      sR[v] = D.x;
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
      const uint4* src = nullptr;
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (valid && a.lists != nullptr) {
        const int64_t col = (int64_t)ti * 4 + sub;
        cnt = (int)a.list_cnt[col];
        src = reinterpret_cast<const uint4*>(a.lists + (int64_t)ti * (4 * kListRegion) +
                                             list_offset(a.list_cnt, ti, sub));
        w = src[0];
      }
      const bool direct = cnt > kFListCap;
      const int nw = direct ? 0 : (cnt + 7) >> 3;
      MinTarget Tg;
      {
        const float4 A = sA[slot], V = sB[slot], C = sC[slot];
        Tg.x = A.x; Tg.y = A.y; Tg.z = A.z; Tg.Hinv = A.w;
        Tg.vx = V.x; Tg.vy = V.y; Tg.vz = V.z;
        Tg.P = C.x; Tg.F = C.y; Tg.c = C.z; Tg.B = C.w;
        Tg.rho = sR[slot];
      }
      MinSums s;
      s.ax = s.ay = s.az = s.du = s.vsig = 0.0f;
      s.npair = 0;
      for (int q = 0; q < nw; ++q) {
        const uint4 wn = q + 1 < nw ? src[q + 1] : w;  // the next word in flight
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (8 * q + e < cnt) {
            const int k = list_entry(w, e);
            min_pair<kCount>(Tg, sA[k], sB[k], sC[k], sR[k], beta, s);
          }
        }
        w = wn;
      }
      if (direct && valid) {
        // no list, or the density list overflowed: every source of the runs
        // (the pairs beyond reach add exactly zero)
        const int tx = kc % g.ex - 1, ty = (kc / g.ex) % g.ey - 1, tz = kc / (g.ex * g.ey) - 1;
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
          for (int32_t k = A0 + sub; k < B0; k += tpp) min_pair<kCount>(Tg, sA[k], sB[k], sC[k], sR[k], beta, s);
        }
      }
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
        const int32_t p = a.perm[ti];
        a.ax[p] = s.ax;
        a.ay[p] = s.ay;
        a.az[p] = s.az;
        a.du_dt[p] = s.du;
        a.v_sig[p] = s.vsig;
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

constexpr size_t kMinSmem = (size_t)kBlkStageCap * (3 * sizeof(float4) + sizeof(float)) + sizeof(StageTable) +
                            sizeof(BlockTargets) +
                            (size_t)kBlkStageCap * (sizeof(uint16_t) + sizeof(uint8_t));
static_assert(kMinBlocks * (kMinSmem + 1024) <= 228 * 1024, "three k_force_min blocks per SM");

// Blocks whose neighbourhood exceeded the staging buffer: one warp per target
// cell, lane = target, the 27 cells streamed through a per-warp buffer with
// positions relative to the target cell.
template <int kFl, int K>
__global__ void __launch_bounds__(kThreads) k_force_overflow(sphh::ForceArgs a, PhysDev ph, SphenixDev x) {
  constexpr bool kE = kFl != kFlMinimal;
  extern __shared__ __align__(16) unsigned char fo_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = fo_raw + warp * (fovf_smem<kFl>() / kWarpsPerBlock);
  float4* sA = reinterpret_cast<float4*>(base);
  float4* sB = sA + kFOvfCap;
  float4* sC = sB + kFOvfCap;
  float4* sE = sC + kFOvfCap;  // SPHENIX only
  float2* sD = reinterpret_cast<float2*>(sC + (kE ? 2 : 1) * kFOvfCap);
  const int32_t n_items = a.misc_ro[kNumOverflow] * kBlkWarps;
  unsigned long long pair_acc = 0;
  for (int32_t item = blockIdx.x * kWarpsPerBlock + warp; item < n_items;
       item += gridDim.x * kWarpsPerBlock) {
    const int32_t b = a.overflow[item / kBlkWarps];
    const BlockGeom g = block_geom(a.grid, a.n_sims, b);
    int tx, ty, tz;
    if (!warp_cell(g, item % kBlkWarps, tx, ty, tz)) continue;
    const float dt = kFl == kFlGradient ? block_dt(a, x, b) : 0.0f;
    const int32_t nc = g.G.n_c;
    const int32_t cx = g.c0x + tx, cy = g.c0y + ty, cz = g.c0z + tz;
    const int32_t c = g.G.cell_base + cx + nc * (cy + nc * cz);
    const int32_t ts = a.cell_start[c], te = a.cell_start[c + 1];
    const NbLane nb = neighbour_lane(lane, g.G.cell_base, cx, cy, cz, nc, g.G.cell_f, a.cell_start);
    int incl = nb.len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int nsrc = __shfl_sync(0xffffffffu, incl, 31);
    const int self_base = __shfl_sync(0xffffffffu, incl - nb.len, 13);
    auto put = [&](int slot, int32_t j, float ox, float oy, float oz) {
      float4 p = a.fA[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      sA[slot] = p;
      sB[slot] = a.fB[j];
      sC[slot] = a.fC[j];
      sD[slot] = a.fD[j];
      if (kE) sE[slot] = a.fE[j];
    };
    for (int32_t t0 = ts; t0 < te; t0 += 32) {
      const int32_t ti = t0 + lane;
      const bool valid = ti < te && (a.act == nullptr || a.act[ti] != 0);
      const int32_t tl = valid ? ti : ts;
      ForceTarget Tg;
      Tg.A = a.fA[tl];
      Tg.B = a.fB[tl];
      Tg.C = a.fC[tl];
      Tg.D = a.fD[tl];
      Tg.E = kE ? a.fE[tl] : make_float4(0.f, 0.f, 0.f, 0.f);
      finish_target(Tg);
      ForceSums s;
      fsums_zero(s);
      if (kFl == kFlGradient) s.ay = Tg.E.y;
      for (int v0 = 0; v0 < nsrc; v0 += kFOvfCap) {
        const int cnt = stage_sources(v0, kFOvfCap, nb, lane, put);
        for (int k = 0; k < cnt; ++k) {
          const float4 Aj = sA[k];
          const float dx = Tg.A.x - Aj.x, dy = Tg.A.y - Aj.y, dz = Tg.A.z - Aj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float Hm = reach<kFl>(Tg.A.w, Aj.w);
          const bool self = (v0 + k == self_base + (ti - ts));
          if (r2 < Hm * Hm && !self) force_pair<kFl, K>(Tg, Aj, sB[k], sC[k], sD[k], kE ? sE[k] : Tg.E, ph, true, s);
        }
        __syncwarp();
      }
      if (valid) {
        if (kFl == kFlGradient)
          gradient_write(a, x, dt, ti, Tg, s);
        else if (kFl == kFlLimit)
          limit_write(a, ti, Tg, s);
        else
          force_write(a, ti, s);
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

}  // namespace sphk

namespace sphh {
using namespace sphk;

template <int kFl, int K>
static cudaError_t launch_force_fk(const ForceArgs& a, const PhysDev& ph, const SphenixDev& x, cudaStream_t st) {
  static int bps = 0, bps_o = 0;
  // the Minimal flavour with the cubic spline runs k_force_min
  constexpr bool kMin = kFl == kFlMinimal && K == kKernCubic;
  constexpr size_t kSmem = kMin ? kMinSmem : force_blk_smem<kFl, K>(), kSmemO = fovf_smem<kFl>();
  if (!bps) {
    cudaError_t e;
    if (kMin) {
      e = cudaFuncSetAttribute(k_force_min<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_force_min<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_force_min<false>, kBlkThreads, kSmem);
    } else {
      e = cudaFuncSetAttribute(k_force<kFl, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_force<kFl, K>, kBlkThreads, kSmem);
    }
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_force_overflow<kFl, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemO);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_o, k_force_overflow<kFl, K>, kThreads, kSmemO);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    if (bps_o < 1) bps_o = 1;
  }
  cudaError_t e = cudaMemsetAsync(a.misc + kNumOverflow, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (kMin && ph.count_pairs)
    k_force_min<true><<<a.num_sms * bps, kBlkThreads, kSmem, st>>>(a, ph);
  else if (kMin)
    k_force_min<false><<<a.num_sms * bps, kBlkThreads, kSmem, st>>>(a, ph);
  else
    k_force<kFl, K><<<a.num_sms * bps, kBlkThreads, kSmem, st>>>(a, ph, x);
  k_force_overflow<kFl, K><<<a.num_sms * bps_o, kThreads, kSmemO, st>>>(a, ph, x);
  return cudaGetLastError();
}

template <int kFl>
static cudaError_t launch_force_fl(const ForceArgs& a, const PhysDev& ph, const SphenixDev& x, cudaStream_t st) {
  switch (ph.kernel) {
    case kKernQuartic:
      return launch_force_fk<kFl, kKernQuartic>(a, ph, x, st);
    case kKernWendlandC2:
      return launch_force_fk<kFl, kKernWendlandC2>(a, ph, x, st);
    default:
      return launch_force_fk<kFl, kKernCubic>(a, ph, x, st);
  }
}

cudaError_t launch_force(const ForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  return launch_force_fl<kFlMinimal>(a, ph, SphenixDev{}, st);
}

cudaError_t launch_sphenix_force(const ForceArgs& a, const PhysDev& ph, const SphenixDev& x, cudaStream_t st) {
  if (a.fE == nullptr) return cudaErrorInvalidValue;
  return launch_force_fl<kFlSphenix>(a, ph, x, st);
}

cudaError_t launch_limit_bins(const ForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  if (a.fE == nullptr || a.bins_out == nullptr) return cudaErrorInvalidValue;
  return launch_force_fl<kFlLimit>(a, ph, SphenixDev{}, st);
}

cudaError_t launch_sphenix_gradient(const ForceArgs& a, const PhysDev& ph, const SphenixDev& x, cudaStream_t st) {
  if (a.fE == nullptr || a.alpha_c_out == nullptr) return cudaErrorInvalidValue;
  return launch_force_fl<kFlGradient>(a, ph, x, st);
}

}  // namespace sphh
