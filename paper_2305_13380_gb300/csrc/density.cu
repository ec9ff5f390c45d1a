// density.cu -- the SPH density loop with the per-particle smoothing-length
// solve (Sec. 3.1.1-3.1.2).
//
// One warp owns one target cell at a time (persistent grid over the cells of
// every simulation).  The particles of the 27 neighbour cells are staged in
// shared memory with positions relative to the target cell; each lane owns a
// target particle and walks the staged sources (a broadcast read).  For each
// pass at the lane's current h the lane accumulates, in FP32,
//   S_w   = sum_j w(q),            S_dw  = sum_j (3 w + q w'(q)),
//   S_mw  = sum_j m_j w(q),        S_mdw = sum_j m_j (3 w + q w'(q)),
//   S_div = sum_j m_j g(q) (v_j - v_i) . x_ij,
//   S_curl= sum_j m_j g(q) (v_i - v_j) x x_ij,      g(q) = w'(q)/q,
// so that n_hat = S_w / H^3, dn_hat/dh = -S_dw / (h H^3), rho = S_mw / H^3,
// d rho/dh = -S_mdw / (h H^3), grad_i W_ij = g(q) x_ij / H^5.  Newton-Raphson
// on n_hat(h) - (eta/h)^3 (the paper's iteration, with dn_hat/dh) is taken in
// FP64: h <- h (1 - A/B) with A = S_w/gamma_K^3 - eta^3 and
// B = 3 eta^3 - S_dw/gamma_K^3; the lane stops when |A/B| <= h_tol and
// writes the quantities of the last pass.
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "stencil.cuh"

namespace sphk {

constexpr int kDensCap = 448;  // staged sources per warp
constexpr size_t kDensSmem = (size_t)kWarpsPerBlock * kDensCap * 2 * sizeof(float4);

__global__ void __launch_bounds__(kThreads) k_density(sphh::DensityArgs a, PhysDev ph) {
  extern __shared__ float4 dsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* spos = dsm + warp * (2 * kDensCap);
  float4* svel = spos + kDensCap;
  const int32_t total = a.misc_ro[kTotalCells];
  const double g3 = kGammaKd * kGammaKd * kGammaKd;
  const double eta3 = (double)ph.eta3;
  unsigned long long pair_acc = 0;

  for (int32_t c = blockIdx.x * kWarpsPerBlock + warp; c < total; c += gridDim.x * kWarpsPerBlock) {
    const int32_t ts = a.cell_start[c], te = a.cell_start[c + 1];
    if (ts >= te) continue;
    const GridDev G = a.grid[sim_of_cell(a.grid, a.n_sims, c)];
    const int32_t local = c - G.cell_base, nc = G.n_c;
    const int32_t cx = local % nc, cy = (local / nc) % nc, cz = local / (nc * nc);
    const NbLane nb = neighbour_lane(lane, G.cell_base, cx, cy, cz, nc, G.cell_f, a.cell_start);
    const int nsrc = warp_sum_int(nb.len);
    const bool fits = nsrc <= kDensCap;
    auto put = [&](int slot, int32_t j, float ox, float oy, float oz) {
      float4 p = a.pos4[j];
      p.x += ox;
      p.y += oy;
      p.z += oz;
      spos[slot] = p;
      svel[slot] = a.vel4[j];
    };
    if (fits) stage_sources(0, kDensCap, nb, lane, put);
    // H may not exceed the cell: every neighbour must lie in the 27 cells.
    const double hcap = (double)G.cell_f * (1.0 - 1e-5) / kGammaKd;

    for (int32_t t0 = ts; t0 < te; t0 += 32) {
      const int32_t ti = t0 + lane;
      const bool valid = ti < te;
      const float4 pi = valid ? a.pos4[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 vi = valid ? a.vel4[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
      double h = valid ? (double)a.hs[ti] : hcap;
      if (!(h > 0.0)) h = 0.5 * hcap;
      if (h > hcap) h = hcap;
      double lo = 0.0, hi = INFINITY;
      bool done = !valid;
      int it = 0;
      while (__any_sync(0xffffffffu, !done)) {
        const float H = kGammaK * (float)h;
        const float Hinv = 1.0f / H;
        float Sw = 0.f, Sdw = 0.f, Smw = 0.f, Smdw = 0.f, Sdiv = 0.f, Scx = 0.f, Scy = 0.f, Scz = 0.f;
        int npair = 0;
        for (int v0 = 0; v0 < nsrc; v0 += kDensCap) {
          const int cnt = fits ? nsrc : stage_sources(v0, kDensCap, nb, lane, put);
#pragma unroll 4
          for (int k = 0; k < cnt; ++k) {
            const float4 pj = spos[k];
            const float4 vj = svel[k];
            const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
            const float q = r2 * rinv * Hinv;
            float w, g;
            kernel_w_g(q, H * rinv, w, g);
            const float dw = fmaf(q * q, g, 3.0f * w);
            Sw += w;
            Sdw += dw;
            Smw = fmaf(pj.w, w, Smw);
            Smdw = fmaf(pj.w, dw, Smdw);
            const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;
            const float mg = pj.w * g;
            Sdiv = fmaf(mg, fmaf(ux, dx, fmaf(uy, dy, uz * dz)), Sdiv);
            Scx = fmaf(mg, fmaf(uz, dy, -uy * dz), Scx);
            Scy = fmaf(mg, fmaf(ux, dz, -uz * dx), Scy);
            Scz = fmaf(mg, fmaf(uy, dx, -ux * dy), Scz);
            npair += q < 1.0f;
          }
          if (!fits) __syncwarp();
        }
        if (!done) {
          const double A = (double)Sw / g3 - eta3;
          const double B = 3.0 * eta3 - (double)Sdw / g3;
          if (A < 0.0) lo = h; else hi = h;
          const bool conv = (B > 0.0) && (fabs(A) <= ph.h_tol * B);
          const bool atcap = (h >= hcap) && (A < 0.0);
          const bool last = it + 1 >= ph.max_h_iter;
          if (conv || atcap || last) {
            const int32_t p = a.perm[ti];
            const float H2inv = Hinv * Hinv;
            const float rho = Smw * H2inv * Hinv;
            const float fi = 1.0f / (1.0f - Smdw / (3.0f * Smw));
            const float div = Sdiv * H2inv / Smw;
            const float curl = sqrtf(fmaf(Scx, Scx, fmaf(Scy, Scy, Scz * Scz))) * H2inv / Smw;
            const float P = (ph.gamma - 1.0f) * vi.w * rho;
            const float cs = sqrtf(ph.gamma * P / rho);
            const float hf = (float)h;
            const float B_i = fabsf(div) / (fabsf(div) + curl + ph.eps_balsara * cs / hf);
            a.h[p] = hf;
            a.rho[p] = rho;
            a.f[p] = fi;
            a.div_v[p] = div;
            a.curl_v[p] = curl;
            a.P[p] = P;
            a.c[p] = cs;
            a.B[p] = B_i;
            if (a.n_iter) a.n_iter[p] = it + 1;
            if (atcap) atomicOr(a.status, SPH_ST_REBUILD);
            else if (!conv) atomicOr(a.status, SPH_ST_H_NOCONV);
            pair_acc += (unsigned long long)npair;
            done = true;
          } else {
            double hn = (B > 0.0) ? h * (1.0 - A / B) : 2.0 * h;
            hn = fmin(fmax(hn, 0.5 * h), 2.0 * h);
            if (!(B > 0.0) || !(hn > lo) || !(hn < hi)) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
            if (hn > hcap) hn = hcap;
            h = hn;
            ++it;
          }
        }
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

cudaError_t launch_density(const DensityArgs& a, const PhysDev& ph, cudaStream_t st) {
  static int blocks_per_sm = 0;
  if (!blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_density, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDensSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_density, kThreads, kDensSmem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  k_density<<<a.num_sms * blocks_per_sm, kThreads, kDensSmem, st>>>(a, ph);
  return cudaGetLastError();
}

}  // namespace sphh
