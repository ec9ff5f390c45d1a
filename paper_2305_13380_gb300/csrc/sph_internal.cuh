// sph_internal.cuh -- device-side structures and helpers shared by the CUDA
// translation units of the SPH library (cell build, density, force, step).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sphk {

// H/h of the 3-D cubic spline in the Dehnen & Aly (2012) convention (Sec. 3.1).
constexpr double kGammaKd = 1.825742;
constexpr float kGammaK = 1.825742f;
// Normalisation of the cubic spline with support H: w(0) = 8/pi.
constexpr float kWNorm = 2.5464790894703255f;

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;

// Misc device words kept by a context.
enum MiscSlot {
  kStatus = 0,       // SPH_ST_* bits
  kTotalCells = 1,   // number of cells over all simulations of the last build
  kTreeWork = 2,     // group counter of the tree loops
  kTotalBlocks = 3,  // number of 2x2x2 blocks of cells over all simulations
  kNumOverflow = 4,  // blocks queued for the overflow kernel of a loop
  kTreeFbCount = 5,  // targets queued for the coarser-level solve of the tree loops
  kTreeFbWork = 6,   // queue counter of the tree fallback kernels
  kHierVmax = 7,     // largest |v| of a sub-step's drift (float bits)
  kHierHmax = 8,     // largest h after a sub-step's drift (float bits)
  kMiscWords = 10
};

// One simulation's grid, computed on the device by the build.
struct GridDev {
  double L;           // periodic box side
  double cell;        // cell side L / n_c (FP64)
  float cell_f;       // cell side (FP32)
  int32_t n_c;        // cells per side
  int32_t cell_base;  // first global cell id of this simulation
  int32_t blk_base;   // first global 2x2x2-block id of this simulation
  float scale_f;      // n_c / L in FP32 (estimates of cell coordinates)
  float reach_f;      // largest support the cells serve: cell_f after a build,
                      // less twice the drift since, while cells are kept
  int64_t part_base;  // first pool index of this simulation
  int64_t n;          // particles in this simulation
};

enum : int { kKernCubic = 0, kKernQuartic = 1, kKernWendlandC2 = 2, kNumKernels = 3 };

template <int K>
struct KernT;
template <>
struct KernT<kKernCubic> {
  static constexpr float gamma = 1.825742f;
  static constexpr double gammad = 1.825742;
};
template <>
struct KernT<kKernQuartic> {
  static constexpr float gamma = 2.018932f;
  static constexpr double gammad = 2.018932;
  static constexpr float c = 9.71404681957369f;  // 15625 / (512 pi)
};
template <>
struct KernT<kKernWendlandC2> {
  static constexpr float gamma = 1.936492f;
  static constexpr double gammad = 1.936492;
  static constexpr float c = 3.3422538049298023f;  // 21 / (2 pi)
};

// gamma_K of a kernel id (host and device; cubic for an unknown id).
__host__ __device__ inline double kernel_gamma(int k) {
  return k == kKernQuartic ? KernT<kKernQuartic>::gammad
                           : (k == kKernWendlandC2 ? KernT<kKernWendlandC2>::gammad : KernT<kKernCubic>::gammad);
}

// Physics constants passed by value to the loop kernels.
struct PhysDev {
  float gamma;
  float eta3;        // eta^3
  float alpha_v;
  float beta_v;
  float eps_balsara;
  double h_tol;
  int32_t max_h_iter;
  int32_t count_pairs;
  int32_t kernel;  // kKern*
  int32_t lanes;   // lanes per target of the uniform loops (0: automatic)
};

// Constants of the SPHENIX flavour (Sec. 3.3) and the step dt over which its
// parameters evolve: dt_dev[s] per simulation when given, else dt.
struct SphenixDev {
  float av_max = 2.0f;  // alpha_V,max
  float ell = 0.05f;    // viscosity decay length
  float beta_c = 1.0f;
  float ac_min = 0.0f;  // alpha_c,min
  float ac_max = 1.0f;  // alpha_c,max
  double dt = 0.0;
  const double* dt_dev = nullptr;
};

// One Newton-Raphson update of the smoothing length (Sec. 3.1): the root of
// f(h) = n_hat(h) - (eta / h)^3, from the sums of a pass at h,
//   S_w = sum_j w(q),   S_dw = sum_j (3 w + q w'(q)),   q = r / H,
// so that with A = S_w / gamma_K^3 - eta^3 and B = 3 eta^3 - S_dw / gamma_K^3
// the Newton step is h <- h (1 - A/B).
//
// The convergence test |A| <= h_tol B runs in FP64 on gamma_K^3 A and
// gamma_K^3 B (a positive scale changes neither the test nor the ratio A/B):
// those are one FP64 subtraction each from the FP32 sums.  The update itself
// runs in FP32, whose rounding (~1e-7 relative) is far below h_tol; this
// keeps FP64 division, slow on this GPU, out of the loop.  A finished target
// gets its last correction applied (Newton converges quadratically, so the
// result is within ~2 (A/B)^2 of the root).  Safeguards: the step is clamped
// to [h/2, 2h] and falls back to bisection of the bracket [lo, hi] when it
// leaves it or B <= 0; h never exceeds hcap.  Returns true when the target
// is done (converged, capped, or out of iterations); otherwise advances h.
struct NewtonConst {
  double a0;  // gamma_K^3 eta^3
  double b0;  // 3 gamma_K^3 eta^3
  double tol;
  int32_t max_it;
};

template <int K = 0>
__device__ __forceinline__ NewtonConst newton_const(const PhysDev& ph) {
  constexpr double gk = KernT<K>::gammad;
  const double g3 = gk * gk * gk;
  NewtonConst c;
  c.a0 = g3 * (double)ph.eta3;
  c.b0 = 3.0 * c.a0;
  c.tol = ph.h_tol;
  c.max_it = ph.max_h_iter;
  return c;
}

__device__ __forceinline__ bool newton_update(float Sw, float Sdw, const NewtonConst& nc, float hcap,
                                              float& h, float& lo, float& hi, int& it, bool& atcap,
                                              bool& conv) {
  const double A = (double)Sw - nc.a0;
  const double B = nc.b0 - (double)Sdw;
  if (A < 0.0) lo = h; else hi = h;
  conv = (B > 0.0) && (fabs(A) <= nc.tol * B);
  atcap = (h >= hcap) && (A < 0.0);
  const float d = (float)A / (float)B;
  if (conv) {
    h = h * (1.0f - d);
    if (h > hcap) {
      h = hcap;
      atcap = true;
    }
    return true;
  }
  if (atcap || it + 1 >= nc.max_it) return true;
  float hn = (B > 0.0) ? h * (1.0f - d) : 2.0f * h;
  hn = fminf(fmaxf(hn, 0.5f * h), 2.0f * h);
  if (!(B > 0.0) || !(hn > lo) || !(hn < hi)) hn = isinf(hi) ? 2.0f * h : 0.5f * (lo + hi);
  if (hn > hcap) hn = hcap;
  h = hn;
  ++it;
  return false;
}

// The largest h whose support gamma_K h stays below `side` (and half the box).
template <int K = 0>
__device__ __forceinline__ float h_cap(double side, double L) {
  return (float)(fmin(side, 0.5 * L) * (1.0 - 1e-5) / KernT<K>::gammad);
}

// Simulation owning a pool index (upper bound search over sim_offset).
__device__ __forceinline__ int sim_of_particle(const int64_t* __restrict__ sim_offset, int n_sims,
                                               int64_t p) {
  int lo = 0, hi = n_sims - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sim_offset[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Warp-contiguous split of [0, n) over the grid: warp w takes [lo, hi), runs
// of ceil(n / warps) rounded up to a multiple of 32, and lane l the indices
// lo + l + 32 k.  Loads stay coalesced, and a thread's indices stay in one
// simulation over long runs (a grid-stride loop jumps across many small
// simulations at every step).  blockDim.x is a multiple of 32.
struct WarpRange {
  int64_t lo, hi;
};
__device__ __forceinline__ WarpRange warp_range(int64_t n) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t run = ((n + nw - 1) / nw + 31) & ~(int64_t)31;
  const int64_t lo = w * run;
  return {lo, lo + run < n ? lo + run : n};
}

// Simulation of a pool index, searched again only when the index leaves the
// range of the last one found.
struct SimCursor {
  int s = -1;
  int64_t lo = 0, hi = 0;
  __device__ __forceinline__ int at(const int64_t* __restrict__ sim_offset, int n_sims, int64_t p) {
    if (p < lo || p >= hi) {
      s = sim_of_particle(sim_offset, n_sims, p);
      lo = sim_offset[s];
      hi = sim_offset[s + 1];
    }
    return s;
  }
};

// Offset of a position from the lower corner of the cell k it is filed in
// (FP64).  After a build it lies in [0, cell); while a sub-step keeps the
// cells of an earlier build a particle may have drifted a little out of its
// cell, and across the periodic boundary: the image nearest the cell is taken
// (no change to an offset within half a box of the cell's centre).
__device__ __forceinline__ double cell_offset(double x, int32_t k, const GridDev& G) {
  double d = x - (double)k * G.cell;
  if (G.reach_f < G.cell_f) {
    // cells kept from an earlier build (a fresh build's offsets need no test):
    // the test in FP32 (a wrapped offset is off by about a box; FP64 is slow
    // on this GPU), the shift in FP64
    const float o = (float)d - 0.5f * G.cell_f, half = 0.5f * (float)G.L;
    if (fabsf(o) > half) d += o > 0.0f ? -G.L : G.L;
  }
  return d;
}

// Global 2x2x2-block id of a global cell id of simulation G.
__device__ __forceinline__ int32_t block_of_cell(int32_t c, const GridDev& G) {
  const int32_t nc = G.n_c, nb = (nc + 1) >> 1;
  const int32_t local = c - G.cell_base;
  const int32_t kx = local % nc, ky = (local / nc) % nc, kz = local / (nc * nc);
  return G.blk_base + (kx >> 1) + nb * ((ky >> 1) + nb * (kz >> 1));
}

// Simulation owning a global cell id.
__device__ __forceinline__ int sim_of_cell(const GridDev* __restrict__ grid, int n_sims, int32_t c) {
  int lo = 0, hi = n_sims - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (grid[mid].cell_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Cell coordinate of one position component: k = floor(fl(fl(x n_c) / L)),
// clamped to [0, n_c - 1]; both roundings are IEEE round-to-nearest.
__device__ __forceinline__ int32_t cell_coord(double x, double L, int32_t n_c) {
  double s = __ddiv_rn(__dmul_rn(x, (double)n_c), L);
  int32_t k = (int32_t)floor(s);
  k = k < 0 ? 0 : k;
  return k > n_c - 1 ? n_c - 1 : k;
}

// The same k with FP64 work only near cell faces.  FP64 division is slow on
// this GPU, so an FP32 estimate comes first: x truncated to an FP32 value by
// integer operations on its bits (sign, exponent and the leading 20 mantissa
// bits: relative error below 2^-20) times scale_f = fl32(n_c / L).  Its
// relative error is below 2^-20 + 2^-23, i.e. under 1.1e-6 n_c in absolute
// terms over [0, L).  When the estimate lies farther than 4e-6 n_c from an
// integer, the exact quotient has the same floor; otherwise, and for x that
// is negative, zero, tiny, huge or not a number, the exact FP64 path decides.
// The result is bit-identical to cell_coord.
__device__ __forceinline__ int32_t cell_coord_fast(double x, double L, int32_t n_c, float scale_f) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (hi > 0 && e > 0 && e < 255) {
    const float s = __int_as_float((e << 23) | ((hi & 0xfffff) << 3)) * scale_f;
    const float k = floorf(s);
    const float fr = s - k;
    const float tol = 4e-6f * (float)n_c;
    if (fr >= tol && fr <= 1.0f - tol) {
      int32_t ki = (int32_t)k;
      ki = ki < 0 ? 0 : ki;
      return ki > n_c - 1 ? n_c - 1 : ki;
    }
  }
  return cell_coord(x, L, n_c);
}

// The 13 axes linking a cell to its neighbours (Sec. 2.2, sorted
// interactions): delta_q with components in {-1, 0, 1}, first non-zero
// component (z, then y, then x) positive; the other 13 neighbours lie along
// -delta_q.  q = 0: (1,0,0); q = 1..3: (q-2, 1, 0); q = 4..12:
// ((q-4)%3 - 1, (q-4)/3 - 1, 1).
constexpr int kAxes = 13;

__device__ __forceinline__ void axis_delta(int q, int& dx, int& dy, int& dz) {
  if (q == 0) {
    dx = 1;
    dy = 0;
    dz = 0;
  } else if (q < 4) {
    dx = q - 2;
    dy = 1;
    dz = 0;
  } else {
    dx = (q - 4) % 3 - 1;
    dy = (q - 4) / 3 - 1;
    dz = 1;
  }
}

// Projection onto the (unnormalised) axis q.
__device__ __forceinline__ float axis_proj(float x, float y, float z, int q) {
  int dx, dy, dz;
  axis_delta(q, dx, dy, dz);
  return fmaf((float)dx, x, fmaf((float)dy, y, (float)dz * z));
}

// Axis of the neighbour offset (dx, dy, dz) != 0 and its sense: +1 when the
// offset is delta_q, -1 when it is -delta_q.
__device__ __forceinline__ int axis_of(int dx, int dy, int dz, int& sense) {
  const bool pos = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
  sense = pos ? 1 : -1;
  const int x = pos ? dx : -dx, y = pos ? dy : -dy, z = pos ? dz : -dz;
  return z == 1 ? 4 + (y + 1) * 3 + (x + 1) : (y == 1 ? 1 + (x + 1) : 0);
}

// Kernels (Sec. 3.1) in the Dehnen & Aly (2012) form W = w(q)/H^3, q = r/H,
// H = gamma_K h, with h twice the kernel's standard deviation per dimension:
//   0 cubic spline   w = 16/pi [(1-q)^3 - 4 (1/2-q)_+^3],                 gamma_K = 1.825742
//   1 quartic spline w = 15625/(512 pi) [(1-q)^4 - 5 (3/5-q)_+^4 + 10 (1/5-q)_+^4],
//                                                                          gamma_K = 2.018932
//   2 Wendland C2    w = 21/(2 pi) (1-q)^4 (1 + 4q),                       gamma_K = 1.936492
// The loops are compiled once per kernel (template parameter K).
// The quartic spline's pieces (x)_+ and w'(q) = -4 c [a^3 - 5 b^3 + 10 d^3]
// with a = (1-q)_+, b = (3/5-q)_+, d = (1/5-q)_+.  Near q = 0 the bracket
// cancels, so w'(q)/q there comes from its expansion c (24 q^2 - 24/5).
__device__ __forceinline__ void quartic_parts(float q, float& a, float& b, float& d) {
  a = fmaxf(1.0f - q, 0.0f);
  b = fmaxf(0.6f - q, 0.0f);
  d = fmaxf(0.2f - q, 0.0f);
}

// w(q) and g(q) = w'(q)/q, branch-free; both vanish for q >= 1.  H_rinv =
// H / r is only used where q is bounded away from 0.
template <int K = kKernCubic>
__device__ __forceinline__ void kernel_w_g(float q, float H_rinv, float& w, float& g) {
  if constexpr (K == kKernCubic) {
    const float a = fmaxf(1.0f - q, 0.0f);
    const bool inner = q < 0.5f;
    const float w_in = kWNorm * fmaf(q * q, fmaf(6.0f, q, -6.0f), 1.0f);  // 8/pi (1 - 6q^2 + 6q^3)
    const float w_out = 2.0f * kWNorm * a * a * a;                        // 16/pi (1 - q)^3
    const float g_in = kWNorm * fmaf(18.0f, q, -12.0f);                   // 8/pi (18 q - 12)
    const float g_out = -6.0f * kWNorm * a * a * H_rinv;                  // -48/pi (1-q)^2 / q
    w = inner ? w_in : w_out;
    g = inner ? g_in : g_out;
  } else if constexpr (K == kKernQuartic) {
    constexpr float c = KernT<K>::c;
    float a, b, d;
    quartic_parts(q, a, b, d);
    const float a2 = a * a, b2 = b * b, d2 = d * d;
    w = c * fmaf(a2, a2, fmaf(-5.0f * b2, b2, 10.0f * d2 * d2));
    const float dwq = -4.0f * c * fmaf(a2, a, fmaf(-5.0f * b2, b, 10.0f * d2 * d));
    g = q < 0.2f ? c * fmaf(24.0f, q * q, -4.8f) : dwq * H_rinv;
  } else {
    constexpr float c = KernT<K>::c;
    const float a = fmaxf(1.0f - q, 0.0f);
    const float a3 = a * a * a;
    w = c * a3 * a * fmaf(4.0f, q, 1.0f);
    g = -20.0f * c * a3;
  }
}

// w(q) and 3 w(q) + q w'(q), the two sums of the Newton passes, without
// the gradient.  Cubic: on the inner piece 8/pi (1 - 6q^2 + 6q^3) and
// 8/pi (3 - 30 q^2 + 36 q^3), on the outer piece 16/pi (1-q)^3 and
// 48/pi (1-q)^2 (1 - 2q).  Wendland C2: 3w + q w' = c (1-q)^3 (3 + 9q - 32 q^2).
// All vanish for q >= 1.
template <int K = kKernCubic>
__device__ __forceinline__ void kernel_w_dw(float q, float& w, float& dw) {
  if constexpr (K == kKernCubic) {
    const float c = kWNorm;
    const float q2 = q * q;
    const float w_in = fmaf(q2, fmaf(6.0f * c, q, -6.0f * c), c);
    const float dw_in = fmaf(q2, fmaf(36.0f * c, q, -30.0f * c), 3.0f * c);
    const float a = fmaxf(1.0f - q, 0.0f);
    const float a2 = a * a;
    const float w_out = (2.0f * c) * a2 * a;
    const float dw_out = a2 * fmaf(-12.0f * c, q, 6.0f * c);
    const bool inner = q < 0.5f;
    w = inner ? w_in : w_out;
    dw = inner ? dw_in : dw_out;
  } else if constexpr (K == kKernQuartic) {
    constexpr float c = KernT<K>::c;
    float a, b, d;
    quartic_parts(q, a, b, d);
    const float a2 = a * a, b2 = b * b, d2 = d * d;
    w = c * fmaf(a2, a2, fmaf(-5.0f * b2, b2, 10.0f * d2 * d2));
    const float dwq = -4.0f * c * fmaf(a2, a, fmaf(-5.0f * b2, b, 10.0f * d2 * d));
    dw = fmaf(q, dwq, 3.0f * w);
  } else {
    constexpr float c = KernT<K>::c;
    const float a = fmaxf(1.0f - q, 0.0f);
    const float a3 = a * a * a;
    w = c * a3 * a * fmaf(4.0f, q, 1.0f);
    dw = c * a3 * fmaf(q, fmaf(-32.0f, q, 9.0f), 3.0f);
  }
}

// g(q) = w'(q)/q only.
template <int K = kKernCubic>
__device__ __forceinline__ float kernel_g(float q, float H_rinv) {
  if constexpr (K == kKernCubic) {
    const float a = fmaxf(1.0f - q, 0.0f);
    const float g_in = kWNorm * fmaf(18.0f, q, -12.0f);
    const float g_out = -6.0f * kWNorm * a * a * H_rinv;
    return q < 0.5f ? g_in : g_out;
  } else {
    float w, g;
    kernel_w_g<K>(q, H_rinv, w, g);
    return g;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sphk

// Host-side launchers implemented in the .cu files.
namespace sphh {
struct Bufs;  // defined in api.cu
}
