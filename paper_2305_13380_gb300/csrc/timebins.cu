// timebins.cu -- time bins of the power-of-two time-step hierarchy (Sec. 2.4,
// "Local time-step optimisations") and the records of the first time-step
// limiter, whose neighbour pass is the kFlLimit flavour of the force kernels.
//
// A particle's CFL step is dt_i = C_CFL gamma_K h_i / v_sig,i; its bin is the
// smallest b in [0, max_bin] with dt_max 2^-b <= dt_i (max_bin if none; 0
// where v_sig <= 0).  The bin is an integer decided by floating point: it is
// taken in FP32 with correctly rounded operations, c = fl(C_CFL gamma_K),
// dt_i = fl(fl(c h_i) / v_sig,i), against fl(dt_max) 2^-b (exact).
#include <math.h>

#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__global__ void k_time_bins(int64_t n, const float* __restrict__ h, const float* __restrict__ v_sig, float c,
                            float dt_max, int max_bin, int32_t* __restrict__ bins) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = v_sig[i];
    const float dt = v > 0.0f ? __fdiv_rn(__fmul_rn(c, h[i]), v) : INFINITY;
    int b = max_bin;
    for (int k = max_bin; k >= 0; --k)
      if (ldexpf(dt_max, -k) <= dt) b = k;
    bins[i] = b;
  }
}

// Sorted limiter records: E[s] = (bin of particle perm[s], 0, 0, 0).
__global__ void k_gather_bins(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ bins,
                              float4* __restrict__ fE) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    fE[s] = make_float4((float)bins[perm[s]], 0.0f, 0.0f, 0.0f);
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

static int grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_time_bins(int64_t n, const float* h, const float* v_sig, float c, float dt_max, int max_bin,
                             int32_t* bins, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_time_bins<<<grid_n(n), 256, 0, st>>>(n, h, v_sig, c, dt_max, max_bin, bins);
  return cudaGetLastError();
}

cudaError_t launch_gather_bins(int64_t n, const int32_t* perm, const int32_t* bins, float4* fE, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather_bins<<<grid_n(n), 256, 0, st>>>(n, perm, bins, fE);
  return cudaGetLastError();
}

}  // namespace sphh
