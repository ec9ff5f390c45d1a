// density.cu -- the SPH density loop with the per-particle smoothing-length
// solve (Sec. 3.1.1-3.1.2).
//
// k_density: one thread block per 2x2x2 block of cells (blocks.cuh), one warp
// per target cell, the block's 4x4x4 neighbourhood staged once in shared
// memory.  Each target is served by tpp lanes (threads per particle: 4 for
// cells of <= 8 particles, else 2) that split the sources between them.
//
//  1. filter: each lane keeps, in its own column of a shared-memory list, the
//     staged slots of the sources closer than the cell size (any support
//     H <= cell can only reach those);
//  2. Newton-Raphson passes run over the list only, accumulating
//        S_w = sum_j w(q),   S_dw = sum_j (3 w + q w'(q)),   q = r / H,
//     so that n_hat = S_w / H^3 and dn_hat/dh = -S_dw / (h H^3).  The
//     iteration of the paper, h <- h - f/f' with f = n_hat - (eta/h)^3 and
//     f' = dn_hat/dh + 3 eta^3 / h^4, is h <- h (1 - A/B) with
//     A = S_w/gamma_K^3 - eta^3, B = 3 eta^3 - S_dw/gamma_K^3 (newton_update:
//     the convergence test in FP64, the update in FP32); a target stops when
//     |A/B| <= h_tol, with that last correction applied (or at the cell cap
//     / max_h_iter);
//  3. a final pass at the converged h accumulates, in FP32,
//        S_mw = sum m_j w,  S_mdw = sum m_j (3 w + q w'),
//        S_div = sum m_j g (v_j - v_i) . x_ij,  S_curl = sum m_j g (v_i - v_j) x x_ij,
//     with g = w'(q)/q, so rho = S_mw / H^3, d rho/dh = -S_mdw / (h H^3) and
//     grad_i W_ij = g x_ij / H^5.
// The partial sums of the tpp lanes are combined with warp shuffles in a
// fixed order, so results do not depend on scheduling.  A target whose list
// overflows walks the staged sources directly.  A block whose neighbourhood
// does not fit the staging buffer is queued for k_density_overflow, which
// streams each target cell's 27 cells through a per-warp buffer.
#include "blocks.cuh"
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "stencil.cuh"

namespace sphk {

// staged sources per block
template <int K>
__host__ __device__ constexpr int dens_cap() {
  return stage_cap<K>();
}
// List entries per lane.  The cubic spline's rounds give a target two lanes
// (above 8 targets a round), each holding ~28 candidates at 13 particles per
// cell, but ~33 when the largest h makes cells 5 % wider (15 per cell): 56
// entries keep such lanes from overflowing into the direct path (which every
// warp holding one would then take), and still fit three blocks per SM.  The
// wider kernels always take four lanes per target.  Lists longer than the
// force's region (kListRegion) are not published: the force filters those
// lanes itself.
template <int K>
__host__ __device__ constexpr int list_cap() {
  return K == kKernCubic ? 56 : kLaneListCap;
}
template <int K>
__host__ __device__ constexpr int list_rows() {  // + one scratch row for the branch-free append
  return list_cap<K>() + 1;
}
// The list keeps each entry's r^2 for the Newton passes (kCacheR2), or only
// the slot, the passes then recomputing r^2 from the staged position.  The
// slots alone leave room for three resident blocks per SM instead of two
// (79 registers, 66 KB of shared memory per block), which was measured
// 10 % faster on the 2M lattice: the loop is latency-bound, and the
// recomputation costs less than the extra warps gain.
constexpr bool kCacheR2 = false;
constexpr int kDensMinBlocks = 3;  // resident blocks per SM the registers are sized for
// shared memory: staged sources (32 B each), per-warp lists (r^2, slot),
// the staging table, the block's target rounds and its target slots/cells
template <int K>
__host__ __device__ constexpr size_t dens_blk_smem() {
  return (size_t)dens_cap<K>() * 2 * sizeof(float4) +
                                (size_t)kBlkWarps * list_rows<K>() * 32 *
                                    ((kCacheR2 ? sizeof(float) : 0) + sizeof(uint16_t)) +
                                sizeof(StageTable) + sizeof(BlockTargets) +
                                (size_t)dens_cap<K>() * (sizeof(uint16_t) + sizeof(uint8_t));
}
constexpr int kOvfCap = 256;  // per-warp staging of the overflow kernel
constexpr size_t kOvfSmem = (size_t)kWarpsPerBlock * kOvfCap * 2 * sizeof(float4);

struct DensSums {
  float w, dw, mw, mdw, div, cx, cy, cz;
  int npair;
};

__device__ __forceinline__ void sums_zero(DensSums& s) {
  s.w = s.dw = s.mw = s.mdw = s.div = s.cx = s.cy = s.cz = 0.f;
  s.npair = 0;
}

// Full density sums of one pair (target at pi/vi, source pj/vj) at H.
template <int K>
__device__ __forceinline__ void dens_pair(const float4& pi, const float4& vi, const float4& pj,
                                          const float4& vj, float H, float Hinv, DensSums& s) {
  const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float q = r2 * rinv * Hinv;
  float w, g;
  kernel_w_g<K>(q, H * rinv, w, g);
  const float dw = fmaf(q * q, g, 3.0f * w);
  s.w += w;
  s.dw += dw;
  s.mw = fmaf(pj.w, w, s.mw);
  s.mdw = fmaf(pj.w, dw, s.mdw);
  const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;
  const float mg = pj.w * g;
  s.div = fmaf(mg, fmaf(ux, dx, fmaf(uy, dy, uz * dz)), s.div);
  s.cx = fmaf(mg, fmaf(uz, dy, -uy * dz), s.cx);
  s.cy = fmaf(mg, fmaf(ux, dz, -uz * dx), s.cy);
  s.cz = fmaf(mg, fmaf(uy, dx, -ux * dy), s.cz);
  s.npair += q < 1.0f;
}


// Terms of the Newton passes: w(q) and 3 w + q w'(q), up to the constant
// factors w_scale<K>() and dw_scale<K>() applied to the sums.  For the cubic
// spline, with a = (1-q)_+ and b = (1-2q)_+ (saturations, as q >= 0),
//   w = (8/pi)(2a^3 - b^3),  w'(q) = -(48/pi)(a^2 - b^2),
//   3w + q w' = (24/pi)(2a^3 - b^3 - 2q (a^2 - b^2)).
template <int K>
__device__ __forceinline__ void newton_terms(float q, float& w, float& dw) {
  if constexpr (K == kKernCubic) {
    const float a = __saturatef(1.0f - q), b = __saturatef(fmaf(-2.0f, q, 1.0f));
    const float a2 = a * a, b2 = b * b;
    w = fmaf(2.0f * a2, a, -b2 * b);
    dw = fmaf(-2.0f * q, a2 - b2, w);
  } else {
    kernel_w_dw<K>(q, w, dw);
  }
}
template <int K>
__host__ __device__ constexpr float w_scale() {
  return K == kKernCubic ? kWNorm : 1.0f;
}
template <int K>
__host__ __device__ constexpr float dw_scale() {
  return K == kKernCubic ? 3.0f * kWNorm : 1.0f;
}

// Sums of the final pass at the converged h.
struct FinSums {
  float mw, mdw, div, cx, cy, cz;
  int npair;
};

__device__ __forceinline__ void fin_zero(FinSums& s) {
  s.mw = s.mdw = s.div = s.cx = s.cy = s.cz = 0.f;
  s.npair = 0;
}

// One pair of the final pass.  Cubic spline: the bracketed terms of
// newton_terms and g~ = (a^2 - b^2)/r, where w'(q)/q = -(48/pi) H g~; the
// constants are applied once per target by fin_scale.  Other kernels: w,
// 3w + q w' and g = w'(q)/q.
template <int K>
__device__ __forceinline__ void fin_pair(const float4& pi, const float4& vi, const float4& pj, const float4& vj,
                                         float mj, float H, float Hinv, FinSums& s) {
  const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float q = r2 * rinv * Hinv;
  float w, dw, g;
  if constexpr (K == kKernCubic) {
    const float a = __saturatef(1.0f - q), b = __saturatef(fmaf(-2.0f, q, 1.0f));
    const float a2 = a * a, b2 = b * b, t = a2 - b2;
    w = fmaf(2.0f * a2, a, -b2 * b);
    dw = fmaf(-2.0f * q, t, w);
    g = t * rinv;
  } else {
    kernel_w_g<K>(q, H * rinv, w, g);
    dw = fmaf(q * q, g, 3.0f * w);
  }
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

// The final-pass sums in the units of dens_write: sum m w, sum m (3w + q w')
// and the gradient sums with g = w'(q)/q.
template <int K>
__device__ __forceinline__ void fin_scale(FinSums& s, float H) {
  if constexpr (K == kKernCubic) {
    s.mw *= kWNorm;
    s.mdw *= 3.0f * kWNorm;
    const float gs = -6.0f * kWNorm * H;
    s.div *= gs;
    s.cx *= gs;
    s.cy *= gs;
    s.cz *= gs;
  }
}

__device__ __forceinline__ void fin_combine(FinSums& s, int tpp) {
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    if (o < tpp) {
      s.mw += __shfl_xor_sync(0xffffffffu, s.mw, o);
      s.mdw += __shfl_xor_sync(0xffffffffu, s.mdw, o);
      s.div += __shfl_xor_sync(0xffffffffu, s.div, o);
      s.cx += __shfl_xor_sync(0xffffffffu, s.cx, o);
      s.cy += __shfl_xor_sync(0xffffffffu, s.cy, o);
      s.cz += __shfl_xor_sync(0xffffffffu, s.cz, o);
      s.npair += __shfl_xor_sync(0xffffffffu, s.npair, o);
    }
  }
}

__device__ __forceinline__ float start_h(float h0, float hcap) {
  const float h = h0 > 0.0f ? h0 : 0.5f * hcap;
  return h > hcap ? hcap : h;
}

// Writes the outputs of one target (sorted index ti) from its sums at h.
template <int K>
__device__ __forceinline__ void dens_write(const sphh::DensityArgs& a, const PhysDev& ph, int32_t ti,
                                           float h, const FinSums& s, float u_i, int passes,
                                           bool conv, bool atcap) {
  const float H = KernT<K>::gamma * h;
  const float Hinv = 1.0f / H;
  const float H2inv = Hinv * Hinv;
  const int32_t p = a.perm[ti];
  const float rho = s.mw * H2inv * Hinv;
  const float fi = 1.0f / (1.0f - s.mdw / (3.0f * s.mw));
  const float div = s.div * H2inv / s.mw;
  const float curl = sqrtf(fmaf(s.cx, s.cx, fmaf(s.cy, s.cy, s.cz * s.cz))) * H2inv / s.mw;
  const float P = (ph.gamma - 1.0f) * u_i * rho;
  const float cs = sqrtf(ph.gamma * P / rho);
  const float hf = h;
  const float B_i = fabsf(div) / (fabsf(div) + curl + ph.eps_balsara * cs / hf);
  // a support that outgrew its cell: twice the cap is the next starting guess,
  // so that each rebuild at least doubles the cells it needs
  a.h[p] = atcap ? 2.0f * hf : hf;
  a.rho[p] = rho;
  a.f[p] = fi;
  a.div_v[p] = div;
  a.curl_v[p] = curl;
  a.P[p] = P;
  a.c[p] = cs;
  a.B[p] = B_i;
  if (a.n_iter) a.n_iter[p] = passes;
  if (atcap) atomicOr(a.status, SPH_ST_REBUILD);
  else if (!conv) atomicOr(a.status, SPH_ST_H_NOCONV);
}

// r^2 of list entry `at` of a lane: cached, or recomputed (same operands,
// same result) from the staged position.
__device__ __forceinline__ float list_r2(const float* lr2, const uint16_t* lj, const float4* spos,
                                         const float4& pi, int at) {
  if (kCacheR2) return lr2[at];
  const float4 pj = spos[lj[at]];
  const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

template <int K>
__global__ void __launch_bounds__(kBlkThreads, kDensMinBlocks) k_density(sphh::DensityArgs a, PhysDev ph) {
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  float4* spos = reinterpret_cast<float4*>(dsm_raw);
  float4* svel = spos + dens_cap<K>();
  // per-lane list entries (r^2, staged slot), column layout [entry][lane]
  float* lr2_all = reinterpret_cast<float*>(svel + dens_cap<K>());
  uint16_t* lj_all = reinterpret_cast<uint16_t*>(lr2_all + (kCacheR2 ? kBlkWarps * list_rows<K>() * 32 : 0));
  StageTable& T = *reinterpret_cast<StageTable*>(lj_all + kBlkWarps * list_rows<K>() * 32);
  BlockTargets& BT = *reinterpret_cast<BlockTargets*>(&T + 1);
  uint16_t* tgt_slot = reinterpret_cast<uint16_t*>(&BT + 1);
  uint8_t* tgt_cell = reinterpret_cast<uint8_t*>(tgt_slot + dens_cap<K>());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* lr2 = lr2_all + warp * (list_rows<K>() * 32);
  uint16_t* lj = lj_all + warp * (list_rows<K>() * 32);
  const int32_t total = a.misc_ro[kTotalBlocks];
  const NewtonConst nwt = newton_const<K>(ph);
  unsigned long long pair_acc = 0;

  for (int32_t b = blockIdx.x; b < total; b += gridDim.x) {
    if (a.blk_any != nullptr && a.blk_any[b] == 0) continue;  // no active target
    const BlockGeom g = block_geom(a.grid, a.n_sims, b);
    const int32_t nsrc = build_stage_table(g, a.cell_start, T);
    if (nsrc > dens_cap<K>()) {
      if (threadIdx.x == 0) a.overflow[atomicAdd(&a.misc[kNumOverflow], 1)] = b;
      __syncthreads();
      continue;
    }
    if (a.act != nullptr) {
      // masked: the block's active targets first, and nothing to stage
      // when it has none
      build_targets<K>(g, T, BT, tgt_slot, tgt_cell, a.act, ph.lanes);
      if (BT.n == 0) continue;
    }
    for (int32_t v = threadIdx.x; v < nsrc; v += kBlkThreads) {
      const int k = staged_cell_of(T, v);
      float ox, oy, oz;
      staged_offset(g, k, ox, oy, oz);
      const int32_t j = T.gstart[k] + (v - T.start[k]);
      float4 p = a.pos4[j];
      const float4 v4 = a.vel4[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      // staged: the position about the block centre (|p| < 2 sqrt(3) cells)
      // with |p|^2 for the filter's expanded distance, the velocity with the
      // mass (the target's u is read from vel4)
      spos[v] = make_float4(p.x, p.y, p.z, fmaf(p.x, p.x, fmaf(p.y, p.y, p.z * p.z)));
      svel[v] = make_float4(v4.x, v4.y, v4.z, p.w);
    }
    if (a.act == nullptr)
      build_targets<K>(g, T, BT, tgt_slot, tgt_cell, nullptr, ph.lanes);  // ends with a barrier
    else
      __syncthreads();  // the staging

    const float hcap = h_cap<K>((double)g.G.reach_f, g.G.L);
    const float R2 = g.G.cell_f * g.G.cell_f;
    const int tpp = BT.tpp, lg = BT.lg, per = BT.per;
    const int sub = lane & (tpp - 1);
    for (int rd = warp; rd < BT.rounds; rd = next_round(BT, lane)) {
      const int t = lane >> lg;
      const int32_t e_t = rd * per + t;
      const bool valid = (t < per) && (e_t < BT.n);
      int slot_i = 0, kc = BT.cell_k[0];
      if (valid) {
        slot_i = tgt_slot[e_t];
        kc = BT.cell_k[tgt_cell[e_t]];
      }
      const int tx = kc % g.ex - 1, ty = (kc / g.ex) % g.ey - 1, tz = kc / (g.ex * g.ey) - 1;
      const int32_t ti = T.gstart[kc] + (slot_i - T.start[kc]);  // sorted index
      const float4 pi = spos[slot_i];
      const float4 vi = svel[slot_i];
      // the starting h and u, loaded now so that their latency hides behind
      // the filter
      const float h_start = valid ? a.hs[ti] : 0.0f;
      const float u_i = valid ? a.vel4[ti].w : 0.0f;
      // 1. filter into the lane's own list column
      int cnt = 0;
      if (valid && a.axis_order != nullptr) {
        // sorted interactions (Sec. 2.2): each neighbour cell is walked along
        // the axis linking it to the target's cell, nearest particles first,
        // up to the first one whose distance along that axis reaches the
        // search radius; the rest of the cell lies farther along the axis
        const float Rn[4] = {0.0f, g.G.cell_f, g.G.cell_f * 1.41421356f, g.G.cell_f * 1.73205081f};
#pragma unroll 1
        for (int nb = 0; nb < 27; ++nb) {
          const int ox = nb % 3 - 1, oy = (nb / 3) % 3 - 1, oz = nb / 9 - 1;
          const int k = (tx + 1 + ox) + g.ex * ((ty + 1 + oy) + g.ey * (tz + 1 + oz));
          const int32_t s0 = T.start[k], len = T.len[k];
          if (nb == 13) {  // the own cell: every particle
            for (int32_t r = sub; r < len; r += tpp) {
              const float4 pj = spos[s0 + r];
              const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              const int at = min(cnt, list_cap<K>()) * 32 + lane;
              if (kCacheR2) lr2[at] = r2;
              lj[at] = (uint16_t)(s0 + r);
              cnt += r2 < R2;
            }
            continue;
          }
          int sense;
          const int q = axis_of(ox, oy, oz, sense);
          const uint16_t* ord = a.axis_order + (int64_t)q * a.axis_stride + T.gstart[k];
          // |x_ij . delta| <= r |delta|: beyond R |delta| (with a margin far
          // above FP32 rounding) no pair is within R
          const float bound = Rn[ox * ox + oy * oy + oz * oz] * 1.00001f;
          const float sf = (float)sense;
          const float p_i = sf * axis_proj(pi.x, pi.y, pi.z, q);
          for (int32_t r = sub; r < len; r += tpp) {
            const int32_t kk = s0 + (int32_t)ord[sense > 0 ? r : len - 1 - r];
            const float4 pj = spos[kk];
            if (sf * axis_proj(pj.x, pj.y, pj.z, q) - p_i >= bound) break;
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const int at = min(cnt, list_cap<K>()) * 32 + lane;
            if (kCacheR2) lr2[at] = r2;
            lj[at] = (uint16_t)kk;
            cnt += r2 < R2;
          }
        }
      } else if (valid) {
        // r^2 = |p_i|^2 + |p_j|^2 - 2 p_i . p_j: three FMAs from the staged
        // |p_j|^2 against R^2 - |p_i|^2.  Its rounding (a few 1e-6 R^2 at
        // |p| < 2 sqrt(3) cells) lies far inside the 2e-5 R^2 margin, so every
        // source within R is listed (a listed source just beyond R adds
        // nothing: the passes recompute r^2 exactly, and the force tests
        // its own reach)
        static_assert(!kCacheR2, "the expanded filter keeps no r^2");
        const float mx = -2.0f * pi.x, my = -2.0f * pi.y, mz = -2.0f * pi.z;
        const float cthr = fmaf(R2, 2e-5f, R2) - pi.w;
#pragma unroll 1
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
#pragma unroll 4
          for (int32_t k = A0 + sub; k < B0; k += tpp) {
            const float4 pj = spos[k];
            const float tq = fmaf(mz, pj.z, fmaf(my, pj.y, fmaf(mx, pj.x, pj.w)));
            const int at = min(cnt, list_cap<K>()) * 32 + lane;
            lj[at] = (uint16_t)k;
            cnt += tq < cthr;
          }
        }
      }
      bool direct = cnt > list_cap<K>();
      if (a.axis_order != nullptr) {
        // the sorted walk splits a target's sources between its lanes by rank
        // along each axis, the direct walk by position in the runs: a target
        // whose list overflowed in any lane sends all its lanes direct, so
        // that its lanes never mix the two splits (here, or in the force loop
        // through the published lists)
        const unsigned m = __ballot_sync(0xffffffffu, direct);
        const unsigned grp = ((1u << tpp) - 1u) << (lane & ~(tpp - 1));
        direct = (m & grp) != 0u;
      }
      // publish the list for the force loop of this build: 16-byte vectors
      // into this lane's region (the force loop rebuilds the same rounds)
      bool pub = valid && !direct && cnt <= kListRegion;
      if (a.axis_order != nullptr) {
        // the force's own filter splits by run position: under the sorted
        // walk a target's lanes are published all together or not at all
        const unsigned m = __ballot_sync(0xffffffffu, valid && !pub);
        const unsigned grp = ((1u << tpp) - 1u) << (lane & ~(tpp - 1));
        pub = pub && (m & grp) == 0u;
      }
      // a target's lanes' lists are published one after another, each from a
      // 16-byte word: lane sub's after the lower lanes' counts rounded up to
      // words (the force reads the target's counts and finds its offset), so
      // that the lists move in whole sectors
      int poff = 0;
      {
        const int mine = (a.lists != nullptr && valid && !a.upper && pub) ? ((cnt + 7) & ~7) : 0;
        int incl = mine;
        for (int o = 1; o < tpp; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o, tpp);
          if (sub >= o) incl += v;
        }
        poff = incl - mine;
      }
      if (a.lists != nullptr && valid && a.upper) {
        // symmetric force pairs: only the sources later in sorted order, so
        // that each pair is met by one of its two particles
        const int64_t col = (int64_t)ti * 4 + sub;
        int kept = 0;
        if (pub) {
          uint16_t* dst = a.lists + col * kListRegion;
          // without a periodic wrap the staged order of a block is the sorted
          // order (cells z, y, x major to minor in both), so the slot decides
          const bool wraps = g.c0x == 0 || g.c0y == 0 || g.c0z == 0 || g.c0x + g.wx >= g.G.n_c ||
                             g.c0y + g.wy >= g.G.n_c || g.c0z + g.wz >= g.G.n_c;
          for (int e = 0; e < cnt; ++e) {
            const int slot = lj[e * 32 + lane];
            bool later = slot > slot_i;
            if (wraps) {
              const int kk = staged_cell_of(T, slot);
              later = T.gstart[kk] + (slot - T.start[kk]) > ti;
            }
            if (later) dst[kept++] = (uint16_t)slot;
          }
        }
        a.list_cnt[col] = (uint16_t)(pub ? kept : 0xffff);
      } else if (a.lists != nullptr && valid) {
        const int64_t col = (int64_t)ti * 4 + sub;
        a.list_cnt[col] = (uint16_t)(pub ? cnt : 0xffff);
        if (pub) {
          uint4* dst = reinterpret_cast<uint4*>(a.lists + (int64_t)ti * (4 * kListRegion) + poff);
          for (int e8 = 0; e8 < cnt; e8 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int e0 = e8 + 2 * q, e1 = e0 + 1;
              const uint32_t lo = e0 < list_cap<K>() ? lj[e0 * 32 + lane] : 0u;
              const uint32_t hi = e1 < list_cap<K>() ? lj[e1 * 32 + lane] : 0u;
              w[q] = lo | (hi << 16);
            }
            dst[e8 >> 3] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
      // 2. Newton-Raphson passes over the list (or over all runs if it overflowed)
      float h = valid ? start_h(h_start, hcap) : hcap;
      float lo = 0.0f, hi = INFINITY;
      bool done = !valid, atcap = false, conv = false;
      int it = 0, passes = 0;
      while (__any_sync(0xffffffffu, !done)) {
        const float H = KernT<K>::gamma * h;
        const float Hinv = 1.0f / H;
        float Sw0 = 0.f, Sdw0 = 0.f, Sw1 = 0.f, Sdw1 = 0.f;
        const int n_l = (!done && !direct) ? cnt : 0;
        int e = 0;
        for (; e + 1 < n_l; e += 2) {
          const float r2a = list_r2(lr2, lj, spos, pi, e * 32 + lane);
          const float r2b = list_r2(lr2, lj, spos, pi, (e + 1) * 32 + lane);
          const float ria = rsqrtf(fmaxf(r2a, 1e-30f)), rib = rsqrtf(fmaxf(r2b, 1e-30f));
          const float qa = r2a * ria * Hinv, qb = r2b * rib * Hinv;
          float wa, dwa, wb, dwb;
          newton_terms<K>(qa, wa, dwa);
          newton_terms<K>(qb, wb, dwb);
          Sw0 += wa;
          Sw1 += wb;
          Sdw0 += dwa;
          Sdw1 += dwb;
        }
        if (e < n_l) {
          const float r2a = list_r2(lr2, lj, spos, pi, e * 32 + lane);
          const float ria = rsqrtf(fmaxf(r2a, 1e-30f));
          float wa, dwa;
          newton_terms<K>(r2a * ria * Hinv, wa, dwa);
          Sw0 += wa;
          Sdw0 += dwa;
        }
        if (!done && direct) {
          for (int r = 0; r < 9; ++r) {
            int32_t A0, B0;
            warp_run(g, T, tx, ty, tz, r, A0, B0);
            for (int32_t k = A0 + sub; k < B0; k += tpp) {
              const float4 pj = spos[k];
              const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              const float ri = rsqrtf(fmaxf(r2, 1e-30f));
              const float q = r2 * ri * Hinv;
              float w, dw;
              newton_terms<K>(q, w, dw);
              Sw0 += w;
              Sdw0 += dw;
            }
          }
        }
        float Sw = w_scale<K>() * (Sw0 + Sw1), Sdw = dw_scale<K>() * (Sdw0 + Sdw1);
        Sw += __shfl_xor_sync(0xffffffffu, Sw, 1);
        Sdw += __shfl_xor_sync(0xffffffffu, Sdw, 1);
        if (tpp == 4) {
          Sw += __shfl_xor_sync(0xffffffffu, Sw, 2);
          Sdw += __shfl_xor_sync(0xffffffffu, Sdw, 2);
        }
        if (!done) {
          passes = it + 1;
          if (newton_update(Sw, Sdw, nwt, hcap, h, lo, hi, it, atcap, conv)) done = true;
        }
      }
      // 3. final pass at the converged h
      const float H = KernT<K>::gamma * h;
      const float Hinv = 1.0f / H;
      FinSums s0;
      fin_zero(s0);
      if (valid && !direct) {
        for (int e = 0; e < cnt; ++e) {
          const int ka = (int)lj[e * 32 + lane];
          const float4 vk = svel[ka];
          fin_pair<K>(pi, vi, spos[ka], vk, vk.w, H, Hinv, s0);
        }
      }
      if (valid && direct) {
        for (int r = 0; r < 9; ++r) {
          int32_t A0, B0;
          warp_run(g, T, tx, ty, tz, r, A0, B0);
          for (int32_t k = A0 + sub; k < B0; k += tpp) {
            const float4 pj = spos[k];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R2) {
              const float4 vk = svel[k];
              fin_pair<K>(pi, vi, pj, vk, vk.w, H, Hinv, s0);
            }
          }
        }
      }
      fin_combine(s0, tpp);
      fin_scale<K>(s0, H);
      if (valid && sub == 0) {
        dens_write<K>(a, ph, ti, h, s0, u_i, passes, conv, atcap);
        pair_acc += (unsigned long long)s0.npair;
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (ph.count_pairs) {
    unsigned long long v = pair_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(a.pairs, v);
  }
}

// Blocks whose neighbourhood exceeded the staging buffer: one warp per target
// cell; each lane owns a target and walks the 27 cells, streamed through a
// per-warp shared buffer, with positions relative to the target cell.
template <int K>
__global__ void __launch_bounds__(kThreads) k_density_overflow(sphh::DensityArgs a, PhysDev ph) {
  extern __shared__ float4 osm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* spos = osm + warp * (2 * kOvfCap);
  float4* svel = spos + kOvfCap;
  const int32_t n_items = a.misc_ro[kNumOverflow] * kBlkWarps;
  const NewtonConst nwt = newton_const<K>(ph);
  unsigned long long pair_acc = 0;
  for (int32_t item = blockIdx.x * kWarpsPerBlock + warp; item < n_items;
       item += gridDim.x * kWarpsPerBlock) {
    const BlockGeom g = block_geom(a.grid, a.n_sims, a.overflow[item / kBlkWarps]);
    int tx, ty, tz;
    if (!warp_cell(g, item % kBlkWarps, tx, ty, tz)) continue;
    const int32_t nc = g.G.n_c;
    const int32_t cx = g.c0x + tx, cy = g.c0y + ty, cz = g.c0z + tz;
    const int32_t c = g.G.cell_base + cx + nc * (cy + nc * cz);
    const int32_t ts = a.cell_start[c], te = a.cell_start[c + 1];
    const NbLane nb = neighbour_lane(lane, g.G.cell_base, cx, cy, cz, nc, g.G.cell_f, a.cell_start);
    const int nsrc = warp_sum_int(nb.len);
    auto put = [&](int slot, int32_t j, float ox, float oy, float oz) {
      float4 p = a.pos4[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      spos[slot] = p;
      svel[slot] = a.vel4[j];
    };
    const float hcap = h_cap<K>((double)g.G.reach_f, g.G.L);
    for (int32_t t0 = ts; t0 < te; t0 += 32) {
      const int32_t ti = t0 + lane;
      const bool valid = ti < te && (a.act == nullptr || a.act[ti] != 0);
      const float4 pi = valid ? a.pos4[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 vi = valid ? a.vel4[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      float h = valid ? start_h(a.hs[ti], hcap) : hcap;
      float lo = 0.0f, hi = INFINITY;
      bool done = !valid, atcap = false, conv = false;
      int it = 0;
      int passes = 0;
      while (__any_sync(0xffffffffu, !done)) {
        const float H = KernT<K>::gamma * h;
        const float Hinv = 1.0f / H;
        DensSums s;
        sums_zero(s);
        for (int v0 = 0; v0 < nsrc; v0 += kOvfCap) {
          const int cnt = stage_sources(v0, kOvfCap, nb, lane, put);
          for (int k = 0; k < cnt; ++k) dens_pair<K>(pi, vi, spos[k], svel[k], H, Hinv, s);
          __syncwarp();
        }
        if (!done) {
          passes = it + 1;
          if (newton_update(s.w, s.dw, nwt, hcap, h, lo, hi, it, atcap, conv)) done = true;
        }
      }
      // final pass at the converged h
      {
        const float H = KernT<K>::gamma * h;
        const float Hinv = 1.0f / H;
        FinSums s;
        fin_zero(s);
        for (int v0 = 0; v0 < nsrc; v0 += kOvfCap) {
          const int cnt = stage_sources(v0, kOvfCap, nb, lane, put);
          for (int k = 0; k < cnt; ++k) fin_pair<K>(pi, vi, spos[k], svel[k], spos[k].w, H, Hinv, s);
          __syncwarp();
        }
        fin_scale<K>(s, H);
        if (valid) {
          dens_write<K>(a, ph, ti, h, s, vi.w, passes, conv, atcap);
          pair_acc += (unsigned long long)s.npair;
        }
      }
    }
  }
  if (ph.count_pairs) {
    unsigned long long v = pair_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(a.pairs, v);
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

template <int K>
static cudaError_t launch_density_k(const DensityArgs& a, const PhysDev& ph, cudaStream_t st) {
  static int bps = 0, bps_o = 0;
  if (!bps) {
    cudaError_t e = cudaFuncSetAttribute(k_density<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dens_blk_smem<K>());
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_density<K>, kBlkThreads, dens_blk_smem<K>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_density_overflow<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kOvfSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps_o, k_density_overflow<K>, kThreads, kOvfSmem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    if (bps_o < 1) bps_o = 1;
  }
  cudaError_t e = cudaMemsetAsync(a.misc + kNumOverflow, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_density<K><<<a.num_sms * bps, kBlkThreads, dens_blk_smem<K>(), st>>>(a, ph);
  k_density_overflow<K><<<a.num_sms * bps_o, kThreads, kOvfSmem, st>>>(a, ph);
  return cudaGetLastError();
}

cudaError_t launch_density(const DensityArgs& a, const PhysDev& ph, cudaStream_t st) {
  switch (ph.kernel) {
    case kKernQuartic:
      return launch_density_k<kKernQuartic>(a, ph, st);
    case kKernWendlandC2:
      return launch_density_k<kKernWendlandC2>(a, ph, st);
    default:
      return launch_density_k<kKernCubic>(a, ph, st);
  }
}

}  // namespace sphh
