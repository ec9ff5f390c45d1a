// fp32_probe.cu -- a measurement kernel for the benchmark only, built into its
// own shared object (not the SPH library): independent FP32 fused multiply-add
// chains, timed by the caller to measure the FP32 pipe's peak rate on the
// device at hand (the denominator of the loops' roofline, which are bound by
// FP32 arithmetic).  Not part of the method.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp32_probe(int64_t iters, float a, float b, float* __restrict__ sink) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (float)(threadIdx.x + c);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains live
}

}  // namespace

// Launches `blocks` blocks of 256 threads, each running 8 chains of `iters`
// FMAs (16 flop per thread and iteration), on `stream`.  Returns 0, or -1 for
// bad arguments, -2 for a launch error.
extern "C" int fp32_probe(int32_t blocks, int64_t iters, float* sink, void* stream) {
  if (blocks < 1 || iters < 1 || !sink) return -1;
  k_fp32_probe<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 0.999999f, 1e-7f, sink);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
