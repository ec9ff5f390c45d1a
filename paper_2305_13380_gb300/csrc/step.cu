// step.cu -- kick-drift-kick time integration with one global time-step per
// simulation (Sec. 2.4 leapfrog; Sec. 5.4 kick and drift operators with the
// scale factor a = 1, so every operator's time interval is dt), and the FP64
// conservation sums.
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// dt_s = C_CFL min_i H_i / v_sig,i over simulation s, as C_CFL gamma_K
// min_i (h_i / v_sig,i): each quotient is one correctly rounded FP32
// division (FP64 division is slow on this GPU), the minimum is exact, and the
// scaling by C_CFL gamma_K is FP64.  Non-negative floats order like their bit
// patterns, so the minimum is taken with an integer atomicMin on the bits:
// each thread keeps a running minimum for the simulation it is in, lanes of
// one simulation combine with shuffles, and one lane per group publishes.
// Particles with v_sig = 0 do not limit dt; a simulation without any signal
// velocity gets dt = 0.
constexpr unsigned kInfBits32 = 0x7f800000u;

__global__ void k_dt_init(unsigned* __restrict__ bits, int n_sims) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sims; s += gridDim.x * blockDim.x)
    bits[s] = kInfBits32;
}

__global__ void k_dt_min(const int64_t* __restrict__ sim_offset, int n_sims, int64_t n_total,
                         const float* __restrict__ h, const float* __restrict__ v_sig,
                         unsigned* __restrict__ bits) {
  const WarpRange wr = warp_range(n_total);
  SimCursor sc;
  int cur = -1;
  float m = INFINITY;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(sim_offset, n_sims, p);
    if (s != cur) {
      if (cur >= 0 && m < INFINITY) atomicMin(&bits[cur], __float_as_uint(m));
      cur = s;
      m = INFINITY;
    }
    const float vs = v_sig[p];
    if (vs > 0.0f) m = fminf(m, __fdiv_rn(h[p], vs));
  }
  // lanes holding the same simulation combine, then one of them publishes
  const unsigned grp = __match_any_sync(0xffffffffu, cur);
  const int lane = threadIdx.x & 31;
  for (int o = 0; o < 32; ++o) {
    const float other = __shfl_sync(0xffffffffu, m, o);
    if ((grp >> o) & 1u) m = fminf(m, other);
  }
  if (cur >= 0 && m < INFINITY && lane == __ffs(grp) - 1) atomicMin(&bits[cur], __float_as_uint(m));
}

__global__ void k_dt_final(const unsigned* __restrict__ bits, int n_sims, double cfl, double gamma_k,
                           double* __restrict__ dt, float* __restrict__ dt_f) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sims; s += gridDim.x * blockDim.x) {
    const float m = __uint_as_float(bits[s]);
    const double d = isinf(m) ? 0.0 : cfl * gamma_k * (double)m;
    dt[s] = d;
    dt_f[2 * s] = (float)(0.5 * d);
    dt_f[2 * s + 1] = (float)(d / 3.0);
  }
}

// One periodic wrap: x < 0 -> x + L, then x >= L -> x - L.  The tests use
// the bit patterns (integer compares instead of FP64 ones: non-negative
// doubles order like their bits, and -0.0 counts as not negative), with the
// same results for every input including NaN.
__device__ __forceinline__ double wrap1(double x, double L) {
  long long b = __double_as_longlong(x);
  if (b < 0 && (b << 1) != 0) {
    x += L;
    b = __double_as_longlong(x);
  }
  if (b >= __double_as_longlong(L)) x -= L;
  return x;
}

// Widening of a float to double (exact): a normal float's sign, exponent
// rebiased from 127 to 1023 and its 23 fraction bits at the top of the 52,
// built with integer operations (this GPU's FP64 pipe, which a conversion
// instruction would use, is slow); zero, subnormals, infinities and NaN take
// the native conversion.
__device__ __forceinline__ double widen(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// First half kick, drift (FP64, one periodic wrap), prediction for the loops.
__global__ void k_kick_drift(sphh::StepArgs a) {
  int cur = -1;
  double dt = 0.0, L = 0.0;
  float hdt = 0.0f, dt3 = 0.0f;
  const WarpRange wr = warp_range(a.n_total);
  SimCursor sc;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(a.sim_offset, a.n_sims, p);
    if (s != cur) {  // the simulation's dt and box (0.5 dt and dt / 3 in FP32)
      cur = s;
      dt = a.dt[s];
      L = a.box[s];
      hdt = a.dt_f[2 * s];
      dt3 = a.dt_f[2 * s + 1];
    }
    const float vx = fmaf(hdt, a.ax[p], a.vx[p]);
    const float vy = fmaf(hdt, a.ay[p], a.vy[p]);
    const float vz = fmaf(hdt, a.az[p], a.vz[p]);
    const float u = fmaf(hdt, a.du_dt[p], a.u[p]);
    a.vx[p] = vx;
    a.vy[p] = vy;
    a.vz[p] = vz;
    a.u[p] = u;
    a.x[p] = wrap1(fma(widen(vx), dt, a.x[p]), L);
    a.y[p] = wrap1(fma(widen(vy), dt, a.y[p]), L);
    a.z[p] = wrap1(fma(widen(vz), dt, a.z[p]), L);
    a.vpx[p] = fmaf(hdt, a.ax[p], vx);
    a.vpy[p] = fmaf(hdt, a.ay[p], vy);
    a.vpz[p] = fmaf(hdt, a.az[p], vz);
    const float up = fmaf(hdt, a.du_dt[p], u);
    a.up[p] = up;
    if (u < 0.0f || up < 0.0f) atomicOr(a.status, SPH_ST_NEG_U);
    if (a.h_guess != nullptr) {
      // the smoothing length follows the density, rho ~ h^-3, whose rate is
      // -rho div v: h (1 + div_v dt / 3) starts the next solve closer to its
      // root (clamped to [0.8, 1.25]; a NaN rate leaves the factor at 0.8)
      const float f = fmaf(dt3, a.div_v[p], 1.0f);
      a.h_guess[p] *= fminf(fmaxf(f, 0.8f), 1.25f);
    }
  }
}

// Second half kick with the new accelerations.
__global__ void k_kick(sphh::StepArgs a) {
  int cur = -1;
  float hdt = 0.0f;
  const WarpRange wr = warp_range(a.n_total);
  SimCursor sc;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(a.sim_offset, a.n_sims, p);
    if (s != cur) {
      cur = s;
      hdt = a.dt_f[2 * s];
    }
    a.vx[p] = fmaf(hdt, a.ax[p], a.vx[p]);
    a.vy[p] = fmaf(hdt, a.ay[p], a.vy[p]);
    a.vz[p] = fmaf(hdt, a.az[p], a.vz[p]);
    const float u = fmaf(hdt, a.du_dt[p], a.u[p]);
    a.u[p] = u;
    if (u < 0.0f) atomicOr(a.status, SPH_ST_NEG_U);
  }
}

// out[4 s + 0..2] = sum_i m_i a_i, out[4 s + 3] = sum_i m_i (v_i . a_i + du_i/dt)
// in FP64, one block per simulation.
__global__ void k_conservation(const int64_t* __restrict__ sim_offset, int n_sims,
                               const float* __restrict__ m, const float* __restrict__ vx,
                               const float* __restrict__ vy, const float* __restrict__ vz,
                               const float* __restrict__ ax, const float* __restrict__ ay,
                               const float* __restrict__ az, const float* __restrict__ du,
                               double* __restrict__ out) {
  const int s = blockIdx.x;
  if (s >= n_sims) return;
  double sx = 0, sy = 0, sz = 0, se = 0;
  for (int64_t p = sim_offset[s] + threadIdx.x; p < sim_offset[s + 1]; p += blockDim.x) {
    const double mi = m[p];
    sx += mi * ax[p];
    sy += mi * ay[p];
    sz += mi * az[p];
    se += mi * ((double)vx[p] * ax[p] + (double)vy[p] * ay[p] + (double)vz[p] * az[p] + du[p]);
  }
  __shared__ double red[4][32];
  sx = warp_sum_d(sx);
  sy = warp_sum_d(sy);
  sz = warp_sum_d(sz);
  se = warp_sum_d(se);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = sx;
    red[1][w] = sy;
    red[2][w] = sz;
    red[3][w] = se;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    out[4 * s + threadIdx.x] = t;
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_dt(const StepArgs& a, cudaStream_t st) {
  const int sb = (a.n_sims + 255) / 256;
  k_dt_init<<<sb, 256, 0, st>>>(a.dt_bits, a.n_sims);
  if (a.n_total > 0) {
    int64_t b = (a.n_total + 255) / 256;
    const int64_t cap = (int64_t)a.num_sms * 8;
    if (b > cap) b = cap;
    k_dt_min<<<(int)b, 256, 0, st>>>(a.sim_offset, a.n_sims, a.n_total, a.h, a.v_sig, a.dt_bits);
  }
  k_dt_final<<<sb, 256, 0, st>>>(a.dt_bits, a.n_sims, a.cfl, a.gamma_k, a.dt, a.dt_f);
  return cudaGetLastError();
}
cudaError_t launch_kick_drift(const StepArgs& a, cudaStream_t st) {
  if (a.n_total > 0) k_kick_drift<<<blocks_for(a.n_total), 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_kick(const StepArgs& a, cudaStream_t st) {
  if (a.n_total > 0) k_kick<<<blocks_for(a.n_total), 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_conservation(int n_sims, const int64_t* sim_offset, const float* m, const float* vx,
                                const float* vy, const float* vz, const float* ax, const float* ay,
                                const float* az, const float* du_dt, double* out, cudaStream_t st) {
  k_conservation<<<n_sims, 256, 0, st>>>(sim_offset, n_sims, m, vx, vy, vz, ax, ay, az, du_dt, out);
  return cudaGetLastError();
}

}  // namespace sphh
