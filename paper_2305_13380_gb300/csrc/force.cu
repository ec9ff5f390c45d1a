// force.cu -- the SPH force loop (Sec. 3.2): pressure gradient of the
// "Minimal" density-energy equations of motion, artificial viscosity with the
// Balsara switch, du/dt and the signal velocity.
//
// Same layout as the density loop: one warp per target cell, the 27
// neighbour cells staged in shared memory, one lane per target.  Per pair,
// with x_ij = x_i - x_j, v_ij = v_i - v_j, G = g(q) / H^5 (so that
// grad_i W(r_ij, h) = G x_ij) evaluated once with h_i and once with h_j:
//   mu     = min(v_ij . x_ij, 0) / r
//   vsig   = c_i + c_j - beta mu
//   nu     = -alpha_V (B_i + B_j)/2 mu vsig / ((rho_i + rho_j)/2)
//   a_i   -= m_j [ fP_i G_i + fP_j G_j + nu/2 (f_i G_i + f_j G_j) ] x_ij
//   du_i  += m_j [ fP_i G_i + nu/4 (f_i G_i + f_j G_j) ] v_ij . x_ij
// with fP = f P / rho^2.  Both kernel gradients vanish beyond their support,
// so candidates outside max(H_i, H_j) contribute exactly zero; only the
// signal-velocity maximum needs the explicit r < max(H_i, H_j), j != i test.
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "stencil.cuh"

namespace sphk {

constexpr int kForceCap = 384;
// per source: pos4 (x, y, z, m), vel4 (vx, vy, vz, 1/H), th4 (fP, f, c, B),
// rh4 (rho, H, 1/H^5, -), index
constexpr size_t kForceSmem = (size_t)kWarpsPerBlock * kForceCap * (4 * sizeof(float4) + sizeof(int32_t));

__global__ void __launch_bounds__(kThreads) k_force(sphh::ForceArgs a, PhysDev ph) {
  extern __shared__ float4 fsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* spos = fsm + warp * (4 * kForceCap);
  float4* svel = spos + kForceCap;
  float4* sth = svel + kForceCap;
  float4* srh = sth + kForceCap;
  int32_t* sidx = reinterpret_cast<int32_t*>(fsm + kWarpsPerBlock * 4 * kForceCap) + warp * kForceCap;
  const int32_t total = a.misc_ro[kTotalCells];
  const float half_alpha = 0.5f * ph.alpha_v;
  unsigned long long pair_acc = 0;

  for (int32_t c = blockIdx.x * kWarpsPerBlock + warp; c < total; c += gridDim.x * kWarpsPerBlock) {
    const int32_t ts = a.cell_start[c], te = a.cell_start[c + 1];
    if (ts >= te) continue;
    const GridDev G = a.grid[sim_of_cell(a.grid, a.n_sims, c)];
    const int32_t local = c - G.cell_base, nc = G.n_c;
    const int32_t cx = local % nc, cy = (local / nc) % nc, cz = local / (nc * nc);
    const NbLane nb = neighbour_lane(lane, G.cell_base, cx, cy, cz, nc, G.cell_f, a.cell_start);
    const int nsrc = warp_sum_int(nb.len);
    const bool fits = nsrc <= kForceCap;
    auto put = [&](int slot, int32_t j, float ox, float oy, float oz) {
      float4 p = a.pos4[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      spos[slot] = p;
      const float4 v = a.vel4[j];
      svel[slot] = v;
      sth[slot] = a.th4[j];
      const float Hinv = v.w;
      const float H2 = Hinv * Hinv;
      srh[slot] = make_float4(a.rho_s[j], 1.0f / Hinv, H2 * H2 * Hinv, 0.0f);
      sidx[slot] = j;
    };
    if (fits) stage_sources(0, kForceCap, nb, lane, put);

    for (int32_t t0 = ts; t0 < te; t0 += 32) {
      const int32_t ti = t0 + lane;
      const bool valid = ti < te;
      const int32_t tl = valid ? ti : ts;
      const float4 pi = a.pos4[tl];
      const float4 vi = a.vel4[tl];
      const float4 thi = a.th4[tl];
      const float rhoi = a.rho_s[tl];
      const float Hinv_i = vi.w;
      const float H_i = 1.0f / Hinv_i;
      const float Hinv5_i = Hinv_i * Hinv_i * Hinv_i * Hinv_i * Hinv_i;
      float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f, vsig = 0.f;
      int npair = 0;
      for (int v0 = 0; v0 < nsrc; v0 += kForceCap) {
        const int cnt = fits ? nsrc : stage_sources(v0, kForceCap, nb, lane, put);
#pragma unroll 2
        for (int k = 0; k < cnt; ++k) {
          const float4 pj = spos[k];
          const float4 vj = svel[k];
          const float4 thj = sth[k];
          const float4 rhj = srh[k];
          const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
          const float r = r2 * rinv;
          const float Gi = kernel_g(r * Hinv_i, H_i * rinv) * Hinv5_i;
          const float Gj = kernel_g(r * vj.w, rhj.y * rinv) * rhj.z;
          const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
          const float vdotx = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
          const float mu = fminf(vdotx, 0.0f) * rinv;
          const float vs = fmaf(-ph.beta_v, mu, thi.z + thj.z);
          const float nu = __fdividef(-half_alpha * (thi.w + thj.w) * mu * vs, 0.5f * (rhoi + rhj.x));
          const float piG = thi.x * Gi;
          const float visc = fmaf(thi.y, Gi, thj.y * Gj);
          const float s = pj.w * fmaf(0.5f * nu, visc, fmaf(thj.x, Gj, piG));
          ax = fmaf(-s, dx, ax);
          ay = fmaf(-s, dy, ay);
          az = fmaf(-s, dz, az);
          du = fmaf(pj.w * fmaf(0.25f * nu, visc, piG), vdotx, du);
          const float Hm = fmaxf(H_i, rhj.y);
          const bool in = (r2 < Hm * Hm) && (sidx[k] != ti);
          vsig = in ? fmaxf(vsig, vs) : vsig;
          npair += in;
        }
        __syncwarp();
      }
      if (valid) {
        const int32_t p = a.perm[ti];
        a.ax[p] = ax;
        a.ay[p] = ay;
        a.az[p] = az;
        a.du_dt[p] = du;
        a.v_sig[p] = vsig;
        pair_acc += (unsigned long long)npair;
      }
    }
    __syncwarp();
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

cudaError_t launch_force(const ForceArgs& a, const PhysDev& ph, cudaStream_t st) {
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_force, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kForceSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_force, kThreads, kForceSmem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  k_force<<<a.num_sms * blocks_per_sm, kThreads, kForceSmem, st>>>(a, ph);
  return cudaGetLastError();
}

}  // namespace sphh
