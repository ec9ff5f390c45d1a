// sphenix.cu -- the per-particle steps of the SPHENIX flavour (Sec. 3.3); its
// neighbour loops (the gradient pass and the force) are the templates of
// force.cu.
//
// Viscosity update (eqs. "sphenix_visc1" to "sphenix_visc4"), per particle,
// after the density loop of this evaluation and before the gradient pass:
//   rate     = (div_v - div_v_prev) / dt        (0 when dt = 0)
//   S        = H^2 max(0, -rate)
//   alpha_loc = alpha_V,max S / (v_sig^2 + S)    (0 when S = 0)
//   alpha_V  = alpha_loc                         if alpha_loc > alpha_V
//            = alpha_loc + (alpha_V - alpha_loc) exp(-ell c dt / H)  otherwise
// with v_sig the signal velocity of the previous force evaluation.
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__global__ void k_sphenix_alpha_v(sphh::SphenixAlphaArgs a, SphenixDev x) {
  const WarpRange wr = warp_range(a.n_total);
  SimCursor sc;
  for (int64_t i = wr.lo + (threadIdx.x & 31); i < wr.hi; i += 32) {
    const float dt = (float)(x.dt_dev != nullptr ? x.dt_dev[sc.at(a.sim_offset, a.n_sims, i)] : x.dt);
    const float H = a.gamma_k * a.h[i];
    const float div = a.div_v[i];
    const float rate = dt > 0.0f ? (div - a.div_v_prev[i]) / dt : 0.0f;
    const float S = H * H * fmaxf(-rate, 0.0f);
    const float vs = a.v_sig[i];
    const float loc = S > 0.0f ? x.av_max * S / fmaf(vs, vs, S) : 0.0f;
    const float al = a.alpha_v[i];
    a.alpha_v[i] = loc > al ? loc : fmaf(al - loc, expf(-x.ell * a.c[i] * dt / H), loc);
    a.div_v_prev[i] = div;
  }
}

__global__ void k_gather_sphenix(int64_t n_total, const int32_t* __restrict__ perm, const float* __restrict__ u,
                                 const float* __restrict__ alpha_v, const float* __restrict__ P,
                                 const float* __restrict__ alpha_c, float4* __restrict__ fE) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[s];
    fE[s] = make_float4(u[p], alpha_v[p], P[p], alpha_c[p]);
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_sphenix_alpha_v(const SphenixAlphaArgs& a, const SphenixDev& x, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  k_sphenix_alpha_v<<<grid_of(a.n_total), 256, 0, st>>>(a, x);
  return cudaGetLastError();
}

cudaError_t launch_gather_sphenix(int64_t n_total, const int32_t* perm, const float* u, const float* alpha_v,
                                  const float* P, const float* alpha_c, float4* fE, cudaStream_t st) {
  if (n_total <= 0) return cudaSuccess;
  k_gather_sphenix<<<grid_of(n_total), 256, 0, st>>>(n_total, perm, u, alpha_v, P, alpha_c, fE);
  return cudaGetLastError();
}

}  // namespace sphh
