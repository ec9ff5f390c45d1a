// pool.cu -- sph_pool_move: copies the particle fields of whole simulations
// between a pool whose simulations sit anywhere in its arrays ("spread", e.g.
// a store of resident simulations) and one whose simulations are packed back
// to back ("packed", e.g. the arena of a batch).  One launch moves every
// field of every range; no step of the SPH method happens here.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace {

constexpr int kF32 = 18;  // vx vy vz u m h ax ay az du_dt v_sig rho f div_v curl_v P c balsara

struct PoolFields {
  double* f64[3];
  float* f32[kF32];
};

PoolFields fields_of(const sph_pool& p) {
  PoolFields f;
  f.f64[0] = p.x;
  f.f64[1] = p.y;
  f.f64[2] = p.z;
  float* const v[kF32] = {p.vx, p.vy, p.vz, p.u, const_cast<float*>(p.m), p.h, p.ax, p.ay, p.az, p.du_dt,
                          p.v_sig, p.rho, p.f, p.div_v, p.curl_v, p.P, p.c, p.balsara};
  for (int k = 0; k < kF32; ++k) f.f32[k] = v[k];
  return f;
}

// Thread per packed particle: its range by binary search over the packed
// offsets, then every field copied between the two positions.
__global__ void k_pool_move(int64_t n_total, int32_t n_ranges, const int64_t* __restrict__ starts,
                            const int64_t* __restrict__ offsets, PoolFields spread, PoolFields packed,
                            int to_packed) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_ranges - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= k) lo = mid; else hi = mid - 1;
    }
    if (k >= offsets[lo + 1]) continue;  // beyond the last range
    const int64_t s = starts[lo] + (k - offsets[lo]);
    if (to_packed) {
#pragma unroll
      for (int f = 0; f < 3; ++f) packed.f64[f][k] = spread.f64[f][s];
#pragma unroll
      for (int f = 0; f < kF32; ++f) packed.f32[f][k] = spread.f32[f][s];
    } else {
#pragma unroll
      for (int f = 0; f < 3; ++f) spread.f64[f][s] = packed.f64[f][k];
#pragma unroll
      for (int f = 0; f < kF32; ++f) spread.f32[f][s] = packed.f32[f][k];
    }
  }
}

bool all_fields(const sph_pool& p) {
  return p.x && p.y && p.z && p.vx && p.vy && p.vz && p.u && p.m && p.h && p.ax && p.ay && p.az && p.du_dt &&
         p.v_sig && p.rho && p.f && p.div_v && p.curl_v && p.P && p.c && p.balsara;
}

}  // namespace

extern "C" int sph_pool_move(const sph_pool* spread, const sph_pool* packed, int32_t n_ranges,
                             const int64_t* starts, const int64_t* offsets, int32_t to_packed, void* stream) {
  if (!spread || !packed || n_ranges < 0 || (n_ranges > 0 && (!starts || !offsets))) return SPH_E_INVAL;
  if (packed->n_total < 0) return SPH_E_INVAL;
  if (n_ranges == 0 || packed->n_total == 0) return SPH_OK;
  if (!all_fields(*spread) || !all_fields(*packed)) return SPH_E_INVAL;
  const int64_t n = packed->n_total;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  k_pool_move<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(n, n_ranges, starts, offsets, fields_of(*spread),
                                                             fields_of(*packed), to_packed ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
