// hier.cu -- sub-steps of the power-of-two time-step hierarchy (Sec. 2.4,
// "Local time-step optimisations"): an integer timeline of 2^max_bin ticks per
// dt_max; a particle in bin b takes steps of 2^(max_bin - b) ticks, aligned to
// multiples of that length.  Each particle runs its own kick-drift-kick: its
// velocity and energy are kept half-kicked for the current step, every
// particle drifts with it, and at the end of its step it gets the second half
// kick with the new acceleration, a new bin, and the first half kick of the
// next step.
#include <climits>

#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__device__ __forceinline__ int64_t step_ticks(int32_t bin, int max_bin) { return (int64_t)1 << (max_bin - bin); }

// The next tick at which some particle's step ends.
__global__ void k_hier_next(int64_t n, const int32_t* __restrict__ bin, const int64_t* __restrict__ t_begin,
                            int max_bin, unsigned long long* __restrict__ t_next) {
  unsigned long long m = ~0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long e = (unsigned long long)(t_begin[i] + step_ticks(bin[i], max_bin));
    m = e < m ? e : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v < m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(t_next, m);
}

// Drift of every particle from t_now to t_next (FP64 positions, one periodic
// wrap), the velocity and energy predicted at t_next for the loops,
// v(t) = v_half + a (t - t_begin - step/2) tau, and the active mask: the
// particles whose step ends at t_next.  With predict, h and rho follow the
// last divergence over the drift, h e^(div_v dt / 3) and rho e^(-div_v dt)
// (continuity), and P and c the equation of state at that rho and the
// predicted u (the density loop replaces them for the active particles).
__global__ void k_hier_drift(sphh::HierArgs a) {
  const int64_t tn = (int64_t)*a.t_next;
  const int64_t t_now = a.t_now_dev != nullptr ? *a.t_now_dev : a.t_now;
  const double dt = (double)(tn - t_now) * a.tau;
  const double L = *a.box;
  float v2max = 0.0f, hmax = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    v2max = fmaxf(v2max, fmaf(a.vx[i], a.vx[i], fmaf(a.vy[i], a.vy[i], a.vz[i] * a.vz[i])));
    const int64_t s = step_ticks(a.bin[i], a.max_bin);
    double x = fma((double)a.vx[i], dt, a.x[i]), y = fma((double)a.vy[i], dt, a.y[i]),
           z = fma((double)a.vz[i], dt, a.z[i]);
    x = x < 0.0 ? x + L : x;
    x = x >= L ? x - L : x;
    y = y < 0.0 ? y + L : y;
    y = y >= L ? y - L : y;
    z = z < 0.0 ? z + L : z;
    z = z >= L ? z - L : z;
    a.x[i] = x;
    a.y[i] = y;
    a.z[i] = z;
    const float w = (float)(((double)(tn - a.t_begin[i]) - 0.5 * (double)s) * a.tau);
    a.vpx[i] = fmaf(a.ax[i], w, a.vx[i]);
    a.vpy[i] = fmaf(a.ay[i], w, a.vy[i]);
    a.vpz[i] = fmaf(a.az[i], w, a.vz[i]);
    const float up = fmaf(a.du_dt[i], w, a.u[i]);
    a.up[i] = up;
    a.act[i] = (uint8_t)(a.t_begin[i] + s == tn);
    if (a.predict) {
      const float dv = (float)((double)a.div_v[i] * dt);
      a.h[i] *= expf(dv * (1.0f / 3.0f));
      const float rho = a.rho[i] * expf(-dv);
      const float P = (a.gamma - 1.0f) * up * rho;
      a.rho[i] = rho;
      a.P[i] = P;
      a.c[i] = sqrtf(a.gamma * P / rho);
    }
    hmax = fmaxf(hmax, a.h[i]);
  }
  if (a.vmax2_bits != nullptr) {
    // non-negative floats order like their bits
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v2max = fmaxf(v2max, __shfl_xor_sync(0xffffffffu, v2max, o));
      hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(a.vmax2_bits, __float_as_uint(v2max));
      atomicMax(a.hmax_bits, __float_as_uint(hmax));
    }
  }
}

// The limiter's input: the CFL proposal of an active particle (and of one
// flagged for synchronisation, which starts a step at t_next too), the bin
// that another inactive particle holds for its current step (the step it
// takes in the force loops until it ends).
__global__ void k_hier_held_bins(int64_t n, const uint8_t* __restrict__ act, const uint8_t* __restrict__ sync,
                                 const int32_t* __restrict__ bin, int32_t* __restrict__ prop) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!act[i] && !(sync != nullptr && sync[i])) prop[i] = bin[i];
}

__device__ __forceinline__ int32_t wrap_cell(int32_t k, int32_t nc) {
  k += k < 0 ? nc : 0;
  return k >= nc ? k - nc : k;
}

// Per cell, the smallest bin among its inactive particles (the wake-up pass
// walks only around active particles whose new bin is more than two above the
// smallest bin in their 27 cells).
__global__ void k_hier_cellmin_init(int32_t* __restrict__ cellmin, const int32_t* __restrict__ total_cells) {
  const int32_t nc = *total_cells;
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) cellmin[c] = INT_MAX;
}
__global__ void k_hier_cellmin(sphh::WakeArgs a) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += (int64_t)gridDim.x * blockDim.x) {
    if (a.act_s[s]) continue;
    const int32_t p = a.perm[s];
    atomicMin(&a.cellmin[a.key[p]], a.bin[p]);
  }
}

// The wake-up limiter's neighbour pass (Sec. 3.4, after Saitoh & Makino
// 2009): once the active particles hold their new bins, every inactive
// force-loop neighbour j of an active i (r_ij < max(H_i, H_j), minimum image,
// decided in FP64) whose step is more than 4 times longer, bin_j < bin_i - 2,
// gets wake[j] = max(wake[j], bin_i - 2).  A warp takes 32 particles of the
// sorted order at a time and walks the cells around each active one, a lane
// per candidate (sorted, so the loads of a cell's candidates coalesce): the
// inactive ones within max(H_i, H_j) by the loops' FP32 cell-relative
// positions, with a margin far above their rounding, get the bin test and
// then the FP64 decision.  The cells are at least as wide as every H, so the
// 27 cells around i's (the distinct ones when n_c < 3, without the FP32 test)
// hold all its neighbours.
__global__ void k_hier_wake(sphh::WakeArgs a) {
  const GridDev G = a.grid[0];
  const int32_t nc = G.n_c;
  const int d0 = nc >= 3 ? -1 : 0, d1 = nc >= 3 ? 1 : nc - 1;
  const bool pre = nc >= 3;
  const double L = G.L;
  const float cs = G.cell_f;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (((int64_t)gridDim.x * blockDim.x) >> 5) << 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) << 5; base < a.n; base += stride) {
    const int64_t me = base + lane;
    unsigned m = __ballot_sync(0xffffffffu, me < a.n && a.act_s[me] != 0);
    while (m != 0u) {
      const int64_t si = base + (__ffs((int)m) - 1);
      m &= m - 1u;
      const int32_t i = a.perm[si];
      const int32_t w = a.bin[i] - 2;
      if (w <= 0) continue;  // no bin lies below
      const int32_t c = a.key[i] - G.cell_base;
      const int32_t kx = c % nc, ky = (c / nc) % nc, kz = c / (nc * nc);
      {
        // skip when no inactive particle of the 27 cells steps in a bin below w
        const int nd = d1 - d0 + 1;
        int32_t lo = INT_MAX;
        if (lane < nd * nd * nd) {
          const int dx = d0 + lane % nd, dy = d0 + (lane / nd) % nd, dz = d0 + lane / (nd * nd);
          lo = a.cellmin[G.cell_base + wrap_cell(kx + dx, nc) +
                         nc * (wrap_cell(ky + dy, nc) + nc * wrap_cell(kz + dz, nc))];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        if (lo >= w) continue;
      }
      const float4 Pi = a.pos4[si];
      const double xi = a.x[i], yi = a.y[i], zi = a.z[i];
      const double Hi = a.gamma * (double)a.h[i];
      for (int dz = d0; dz <= d1; ++dz)
        for (int dy = d0; dy <= d1; ++dy)
          for (int dx = d0; dx <= d1; ++dx) {
            const int32_t cn =
                G.cell_base + wrap_cell(kx + dx, nc) + nc * (wrap_cell(ky + dy, nc) + nc * wrap_cell(kz + dz, nc));
            const float ox = (float)dx * cs, oy = (float)dy * cs, oz = (float)dz * cs;
            const int32_t t1 = a.cell_start[cn + 1];
            for (int32_t t = a.cell_start[cn] + lane; t < t1; t += 32) {
              if (a.act_s[t]) continue;
              if (pre) {
                const float4 Pj = a.pos4[t];
                const float fx = Pi.x - (Pj.x + ox), fy = Pi.y - (Pj.y + oy), fz = Pi.z - (Pj.z + oz);
                const float Hm = fmaxf(Pi.w, Pj.w);
                if (fmaf(fx, fx, fmaf(fy, fy, fz * fz)) >= Hm * Hm * (1.0f + 1e-4f)) continue;
              }
              const int32_t j = a.perm[t];
              if (a.bin[j] >= w) continue;
              double ex = a.x[j] - xi, ey = a.y[j] - yi, ez = a.z[j] - zi;
              ex -= L * rint(ex / L);
              ey -= L * rint(ey / L);
              ez -= L * rint(ez / L);
              const double Hm = fmax(Hi, a.gamma * (double)a.h[j]);
              if (ex * ex + ey * ey + ez * ez < Hm * Hm) atomicMax(&a.wake[j], w);
            }
          }
    }
  }
}

// The steps that end early (Sec. 3.4, second and third limiters): an
// inactive particle that is woken (wake[i] > bin[i]) or flagged for
// synchronisation ends its current step at t_next, where its velocity and
// energy are the predicted ones (its last a and du/dt over the part of the
// step it ran), and starts a new step there: the flagged one in its CFL bin
// (adapt) or its held bin, either raised to the wake-up bin, shortened until
// the step divides t_next, with the first half kick.  Every flag is cleared.
__global__ void k_hier_interrupt(sphh::HierArgs a) {
  const int64_t tn = (int64_t)*a.t_next;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool fl = a.sync != nullptr && a.sync[i] != 0;
    if (fl) a.sync[i] = 0;
    if (a.act[i]) continue;
    const int32_t held = a.bin[i], wk = a.wake != nullptr ? a.wake[i] : -1;
    const bool woken = wk > held;
    if (!fl && !woken) continue;
    int32_t b = fl ? (a.bin_new != nullptr ? a.bin_new[i] : held) : wk;
    b = woken && wk > b ? wk : b;
    b = b < 0 ? 0 : (b > a.max_bin ? a.max_bin : b);
    while (b < a.max_bin && tn % step_ticks(b, a.max_bin) != 0) ++b;
    const float h_new = (float)(0.5 * (double)step_ticks(b, a.max_bin) * a.tau);
    a.vx[i] = fmaf(a.ax[i], h_new, a.vpx[i]);
    a.vy[i] = fmaf(a.ay[i], h_new, a.vpy[i]);
    a.vz[i] = fmaf(a.az[i], h_new, a.vpz[i]);
    const float u = a.up[i], un = fmaf(a.du_dt[i], h_new, u);
    a.u[i] = un;
    if (u < 0.0f || un < 0.0f) atomicOr(a.status, SPH_ST_NEG_U);
    a.bin[i] = b;
    a.t_begin[i] = tn;
  }
}

// The end of an active particle's step: second half kick over the old step,
// the new bin (the proposed one, shortened until the new step is aligned with
// t_next), first half kick over the new step.
__global__ void k_hier_kick(sphh::HierArgs a) {
  const int64_t tn = (int64_t)*a.t_next;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!a.act[i]) continue;
    const float h_old = (float)(0.5 * (double)step_ticks(a.bin[i], a.max_bin) * a.tau);
    int32_t b = a.bin_new != nullptr ? a.bin_new[i] : a.bin[i];
    b = b < 0 ? 0 : (b > a.max_bin ? a.max_bin : b);
    while (b < a.max_bin && tn % step_ticks(b, a.max_bin) != 0) ++b;
    const float h_new = (float)(0.5 * (double)step_ticks(b, a.max_bin) * a.tau);
    const float vx = fmaf(a.ax[i], h_old, a.vx[i]), vy = fmaf(a.ay[i], h_old, a.vy[i]),
                vz = fmaf(a.az[i], h_old, a.vz[i]), u = fmaf(a.du_dt[i], h_old, a.u[i]);
    a.vx[i] = fmaf(a.ax[i], h_new, vx);
    a.vy[i] = fmaf(a.ay[i], h_new, vy);
    a.vz[i] = fmaf(a.az[i], h_new, vz);
    const float un = fmaf(a.du_dt[i], h_new, u);
    a.u[i] = un;
    if (u < 0.0f || un < 0.0f) atomicOr(a.status, SPH_ST_NEG_U);
    a.bin[i] = b;
    a.t_begin[i] = tn;
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int grid_h(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_hier_next(const HierArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.t_next, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess || a.n <= 0) return e;
  k_hier_next<<<grid_h(a.n), 256, 0, st>>>(a.n, a.bin, a.t_begin, a.max_bin, a.t_next);
  return cudaGetLastError();
}

cudaError_t launch_hier_drift(const HierArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_hier_drift<<<grid_h(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_hier_held_bins(const HierArgs& a, int32_t* prop, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_hier_held_bins<<<grid_h(a.n), 256, 0, st>>>(a.n, a.act, a.sync, a.bin, prop);
  return cudaGetLastError();
}

cudaError_t launch_hier_wake(const WakeArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.wake, 0xff, (size_t)a.n * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  k_hier_cellmin_init<<<grid_h(a.n), 256, 0, st>>>(a.cellmin, a.total_cells);
  k_hier_cellmin<<<grid_h(a.n), 256, 0, st>>>(a);
  k_hier_wake<<<grid_h(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_hier_interrupt(const HierArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_hier_interrupt<<<grid_h(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_hier_kick(const HierArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_hier_kick<<<grid_h(a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sphh
