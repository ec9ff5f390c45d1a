// axis.cu -- per-cell orders along the axes linking neighbouring cells, for
// the sorted-interaction pruning of Sec. 2.2 (the pseudo-Verlet figure).
//
// The 26 neighbours of a cell lie along 13 axes delta_q (each with its
// opposite).  For every cell and every axis q the particles of the cell are
// ranked by their projection x . delta_q (cell-relative FP32 positions of the
// density copies; ties by index), and order[q * n + cell_start + rank] holds
// the index within the cell of the particle of that rank.  A target walking a
// neighbour cell along the axis towards it meets the cell's particles by
// increasing distance along the axis, and stops at the first one whose
// distance along the axis already exceeds its search radius (density.cu).
//
// One thread per particle ranks it against the other particles of its cell
// for all 13 axes at once (the cell's copies stay in L1).  Cells larger than
// a block's staging buffer get no order.
#include "blocks.cuh"
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__global__ void k_axis_sort(int64_t n_total, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ key, const int32_t* __restrict__ cell_start,
                            const float4* __restrict__ pos4, uint16_t* __restrict__ order) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = key[perm[s]];
    const int32_t cs = cell_start[c], ce = cell_start[c + 1];
    // a cell beyond one block's staging is only ever walked by the overflow
    // kernels, which do not use the orders
    if (ce - cs > kBlkStageCap) continue;
    const float4 me = pos4[s];
    float mine[kAxes];
#pragma unroll
    for (int q = 0; q < kAxes; ++q) mine[q] = axis_proj(me.x, me.y, me.z, q);
    int rank[kAxes];
#pragma unroll
    for (int q = 0; q < kAxes; ++q) rank[q] = 0;
    for (int32_t m = cs; m < ce; ++m) {
      const float4 o = pos4[m];
#pragma unroll
      for (int q = 0; q < kAxes; ++q) {
        const float p = axis_proj(o.x, o.y, o.z, q);
        rank[q] += (p < mine[q] || (p == mine[q] && m < s)) ? 1 : 0;
      }
    }
#pragma unroll
    for (int q = 0; q < kAxes; ++q) order[(int64_t)q * n_total + cs + rank[q]] = (uint16_t)(s - cs);
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

cudaError_t launch_axis_sort(const AxisSortArgs& a, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  int64_t b = (a.n_total + 255) / 256;
  if (b > 65535) b = 65535;
  k_axis_sort<<<(int)b, 256, 0, st>>>(a.n_total, a.perm, a.key, a.cell_start, a.pos4, a.order);
  return cudaGetLastError();
}

}  // namespace sphh
