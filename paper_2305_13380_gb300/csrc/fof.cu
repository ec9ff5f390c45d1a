// fof.cu -- friends-of-friends groups (Sec. 7.1) on the uniform cell grid.
//
// Particles i and j are friends when their minimum-image distance is below
// the linking length b; groups are the connected components (union-find,
// Sec. 7.1).  The grid's cells are at least b wide, so friends lie in the
// same or adjacent cells; every pair is visited once: from the particle of
// the lower sorted slot inside a cell, and across the 13 axes delta_q (the
// other 13 neighbours see the pair from the opposite side).
//
// The decision is the FP64 one of the definition (d = x_i - x_j wrapped once
// into [-L/2, L/2], r2 = dx*dx + dy*dy + dz*dz, r2 < b*b, no contraction).
// An FP32 distance from cell-relative positions settles every pair whose r2
// is farther from b^2 than its rounding can reach; the rest take the FP64
// test, so the links are exactly those of the definition.
//
// Union-find on the caller's group array, lock-free: a set's root is its
// smallest index, a union hooks the larger root below the smaller one with
// one compare-and-swap (retried when the root changed meanwhile), and the
// link pass's finds halve their paths.  Every parent pointer only ever moves to an ancestor,
// so concurrent halving and hooking keep a valid forest, and the final roots
// are the groups' smallest indices whatever the order of the unions.  The
// parent loads bypass L1 (other SMs write them).  Loops are bounded; a
// bound that is hit sets SPH_ST_CAPACITY.
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

constexpr int kFofMaxSteps = 1 << 20;  // bound of one find or one union's retries

// kHalve: path halving (the link pass).  The label pass reads only: there
// every particle's entry is overwritten with its root while other threads
// walk through it, and a halving write arriving after that would replace a
// final root by a mere ancestor.
template <bool kHalve>
__device__ __forceinline__ int32_t fof_find(int32_t* parent, int32_t x, int32_t* status) {
  for (int it = 0; it < kFofMaxSteps; ++it) {
    const int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    const int32_t gp = __ldcg(parent + p);
    if (kHalve && gp != p) __stcg(parent + x, gp);  // gp is an ancestor of x
    x = gp;
  }
  atomicOr(status, SPH_ST_CAPACITY);
  return x;
}

__device__ __forceinline__ void fof_union(int32_t* parent, int32_t a, int32_t b, int32_t* status) {
  for (int it = 0; it < kFofMaxSteps; ++it) {
    a = fof_find<true>(parent, a, status);
    b = fof_find<true>(parent, b, status);
    if (a == b) return;
    if (a > b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + b, b, a) == b) return;  // b was still a root: hooked
  }
  atomicOr(status, SPH_ST_CAPACITY);
}

// FP64 friendship test of the definition (minimum image, no contraction).
__device__ __forceinline__ double fof_min_image(double d, double L) {
  if (d > 0.5 * L) return __dadd_rn(d, -L);
  if (d < -0.5 * L) return __dadd_rn(d, L);
  return d;
}

__device__ __forceinline__ bool fof_friends64(const double* x, const double* y, const double* z, int32_t i,
                                              int32_t j, double L, double b2) {
  const double dx = fof_min_image(__dadd_rn(x[i], -x[j]), L);
  const double dy = fof_min_image(__dadd_rn(y[i], -y[j]), L);
  const double dz = fof_min_image(__dadd_rn(z[i], -z[j]), L);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return r2 < b2;
}

// Sorted cell-relative positions (index in .w) and singleton sets.
__global__ void k_fof_prep(sphh::FofArgs a) {
  const GridDev G = a.grid[0];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = a.perm[s];
    const int32_t c = a.key[p] - G.cell_base;
    const int32_t kx = c % G.n_c, ky = (c / G.n_c) % G.n_c, kz = c / (G.n_c * G.n_c);
    a.rel[s] = make_float4((float)(a.x[p] - (double)kx * G.cell), (float)(a.y[p] - (double)ky * G.cell),
                           (float)(a.z[p] - (double)kz * G.cell), __int_as_float(p));
    a.group[p] = p;
  }
}

__global__ void k_fof_link(sphh::FofArgs a) {
  const GridDev G = a.grid[0];
  const int32_t nc = G.n_c;
  const double b2 = a.link * a.link;
  // FP32 distances of cell-relative coordinates (|x| below two cells) are
  // within ~1e-6 (2 cell)^2 of the true r2: a band of that width around b^2,
  // plus a margin, goes to the FP64 test
  const float cf = G.cell_f;
  const float band = 4e-6f * (2.0f * cf) * (2.0f * cf) + 1e-5f * (float)b2;
  const float lo = (float)b2 - band, hi = (float)b2 + band;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const float4 me = a.rel[s];
    const int32_t pi = __float_as_int(me.w);
    const int32_t c = a.key[pi] - G.cell_base;
    const int32_t kx = c % nc, ky = (c / nc) % nc, kz = c / (nc * nc);
    for (int o = 0; o <= kAxes; ++o) {
      int dx = 0, dy = 0, dz = 0;
      if (o > 0) axis_delta(o - 1, dx, dy, dz);
      int32_t cx = kx + dx, cy = ky + dy, cz = kz + dz;
      cx += cx < 0 ? nc : 0;
      cx -= cx >= nc ? nc : 0;
      cy += cy < 0 ? nc : 0;
      cy -= cy >= nc ? nc : 0;
      cz += cz < 0 ? nc : 0;
      cz -= cz >= nc ? nc : 0;
      const int32_t cn = G.cell_base + cx + nc * (cy + nc * cz);
      const int32_t t0 = o == 0 ? (int32_t)s + 1 : a.cell_start[cn];
      const int32_t t1 = a.cell_start[cn + 1];
      const float ox = (float)dx * cf, oy = (float)dy * cf, oz = (float)dz * cf;
      for (int32_t t = t0; t < t1; ++t) {
        const float4 q = a.rel[t];
        const float fx = me.x - (q.x + ox), fy = me.y - (q.y + oy), fz = me.z - (q.z + oz);
        const float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        if (r2 >= hi) continue;
        const int32_t pj = __float_as_int(q.w);
        if (r2 < lo || fof_friends64(a.x, a.y, a.z, pi, pj, G.L, b2)) fof_union(a.group, pi, pj, a.status);
      }
    }
  }
}

// Final labels: every particle's root, the smallest index of its group.
__global__ void k_fof_label(sphh::FofArgs a) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n_total;
       p += (int64_t)gridDim.x * blockDim.x)
    a.group[p] = fof_find<false>(a.group, (int32_t)p, a.status);
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

cudaError_t launch_fof(const FofArgs& a, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  int64_t b = (a.n_total + 255) / 256;
  if (b > 65535) b = 65535;
  k_fof_prep<<<(int)b, 256, 0, st>>>(a);
  k_fof_link<<<(int)b, 256, 0, st>>>(a);
  k_fof_label<<<(int)b, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sphh
