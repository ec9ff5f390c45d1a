// radix.cu -- stable least-significant-digit radix sort of (key, value)
// pairs, used to order particles by cell id.  Values enter in ascending
// particle index, so equal keys keep ascending index: the result is exactly
// the stable counting sort of the cell grid (Sec. 2.1), for any cell size.
//
// Each pass sorts by one 8-bit digit:
//   k_radix_hist     per tile of 2048 items: digit histogram -> hist[d * T + t]
//   (scan)           exclusive scan of hist, digit-major, so that tiles of the
//                    same digit follow each other in index order
//   k_radix_scatter  per tile: stable rank of each item among equal digits
//                    (warp match + running per-warp counts, then a prefix over
//                    the warps of the tile), written to hist[d * T + t] + rank
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

template <class K>
__global__ void k_radix_hist(int64_t n, const K* __restrict__ keys, int shift, int n_tiles,
                             int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int i = threadIdx.x; i < kRadixTile; i += kRadixThreads) {
    const int64_t p = base + i;
    if (p < n) atomicAdd(&h[(int)((keys[p] >> shift) & 255)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Warp w of the tile handles items base + w * 256 + j * 32 + lane, j = 0..7,
// i.e. 8 consecutive groups of 32 consecutive items: processing j in order
// visits the warp's items in index order.
template <class K>
__global__ void k_radix_scatter(int64_t n, const K* __restrict__ keys_in,
                                const int32_t* __restrict__ vals_in, int shift, int n_tiles,
                                const int32_t* __restrict__ offsets, K* __restrict__ keys_out,
                                int32_t* __restrict__ vals_out) {
  __shared__ int32_t wcount[kRadixWarps][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < 256; d += 32) wcount[warp][d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile + warp * (32 * kRadixItems);
  K key[kRadixItems];
  int32_t val[kRadixItems], rank[kRadixItems];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const int64_t p = base + j * 32 + lane;
    const bool ok = p < n;
    key[j] = ok ? keys_in[p] : (K)0;
    val[j] = ok ? vals_in[p] : 0;
    const int d = ok ? (int)((key[j] >> shift) & 255) : 256 + lane;  // out-of-range items never match
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = __popc(peers & lt);
    int r = 0;
    if (ok) r = wcount[warp][d] + before;
    rank[j] = r;
    __syncwarp();
    // the highest lane of each group of equal digits advances the count
    if (ok && (peers >> lane) == 1u) wcount[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over the warps of the tile, per digit, in place
  for (int d = threadIdx.x; d < 256; d += kRadixThreads) {
    int32_t run = 0;
    for (int w = 0; w < kRadixWarps; ++w) {
      const int32_t c = wcount[w][d];
      wcount[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRadixItems; ++j) {
    const int64_t p = base + j * 32 + lane;
    if (p < n) {
      const int d = (int)((key[j] >> shift) & 255);
      const int64_t dst = (int64_t)offsets[(int64_t)d * n_tiles + blockIdx.x] + wcount[warp][d] + rank[j];
      keys_out[dst] = key[j];
      vals_out[dst] = val[j];
    }
  }
}

__global__ void k_iota(int64_t n, int32_t* __restrict__ v) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    v[p] = (int32_t)p;
}

// Exclusive scan of m (host-known) int32 in place: per-tile scans, a scan
// of the tile totals, and a final add.
constexpr int kScanTileH = kRadixThreads * 4;

__device__ __forceinline__ int32_t radix_block_scan(int32_t v, int32_t* total) {
  __shared__ int32_t ws[kRadixWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  int32_t wbase = 0, tot = 0;
  for (int k = 0; k < kRadixWarps; ++k) {
    wbase += k < w ? ws[k] : 0;
    tot += ws[k];
  }
  __syncthreads();
  *total = tot;
  return wbase + x - v;
}

__global__ void k_scanh_tiles(int32_t* __restrict__ a, int64_t m, int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTileH;
  int32_t v[4];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t k = base + threadIdx.x * 4 + i;
    v[i] = k < m ? a[k] : 0;
    s += v[i];
  }
  int32_t tot;
  int32_t run = radix_block_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t k = base + threadIdx.x * 4 + i;
    if (k < m) a[k] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scanh_sums(int32_t* __restrict__ sums, int64_t nt) {
  int32_t carry = 0;
  for (int64_t b0 = 0; b0 < nt; b0 += kRadixThreads) {
    const int64_t i = b0 + threadIdx.x;
    const int32_t v = i < nt ? sums[i] : 0;
    int32_t tot;
    const int32_t ex = radix_block_scan(v, &tot);
    if (i < nt) sums[i] = carry + ex;
    carry += tot;
  }
}

__global__ void k_scanh_add(int32_t* __restrict__ a, int64_t m, const int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTileH;
  const int32_t add = sums[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTileH; i += kRadixThreads) {
    const int64_t k = base + i;
    if (k < m) a[k] += add;
  }
}

}  // namespace sphk

namespace sphh {
using namespace sphk;

// histogram (256 per tile) followed by the scan's tile totals
int64_t radix_hist_words(int64_t n) {
  const int64_t h = 256 * ((n + kRadixTile - 1) / kRadixTile);
  return h + (h + kScanTileH - 1) / kScanTileH + 1;
}

// Sorts keys (bits significant bits) stably, values = 0..n-1, into vals_out.
// keys / keys_tmp / vals_tmp / vals_out hold n entries; hist holds
// radix_hist_words(n).  keys is clobbered.
template <class K>
static cudaError_t radix_sort_impl(int64_t n, int bits, K* keys, K* keys_tmp, int32_t* vals_out,
                                   int32_t* vals_tmp, int32_t* hist, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int n_tiles = (int)((n + kRadixTile - 1) / kRadixTile);
  const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
  int64_t ib = (n + 255) / 256;
  if (ib > 65535) ib = 65535;
  // values ping-pong so that the last pass lands in vals_out
  int32_t* v_in = (passes % 2 == 0) ? vals_out : vals_tmp;
  int32_t* v_out = (passes % 2 == 0) ? vals_tmp : vals_out;
  k_iota<<<(int)ib, 256, 0, st>>>(n, v_in);
  K* k_in = keys;
  K* k_out = keys_tmp;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    k_radix_hist<K><<<n_tiles, kRadixThreads, 0, st>>>(n, k_in, shift, n_tiles, hist);
    const int64_t m = (int64_t)256 * n_tiles;
    const int64_t nt = (m + kScanTileH - 1) / kScanTileH;
    k_scanh_tiles<<<(unsigned)nt, kRadixThreads, 0, st>>>(hist, m, hist + m);
    k_scanh_sums<<<1, kRadixThreads, 0, st>>>(hist + m, nt);
    k_scanh_add<<<(unsigned)nt, kRadixThreads, 0, st>>>(hist, m, hist + m);
    k_radix_scatter<K><<<n_tiles, kRadixThreads, 0, st>>>(n, k_in, v_in, shift, n_tiles, hist, k_out, v_out);
    K* t = k_in;
    k_in = k_out;
    k_out = t;
    int32_t* tv = v_in;
    v_in = v_out;
    v_out = tv;
  }
  return cudaGetLastError();
}

cudaError_t scan_exclusive_host_n(int32_t* a, int64_t m, int32_t* tmp, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t nt = (m + kScanTileH - 1) / kScanTileH;
  k_scanh_tiles<<<(unsigned)nt, kRadixThreads, 0, st>>>(a, m, tmp);
  k_scanh_sums<<<1, kRadixThreads, 0, st>>>(tmp, nt);
  k_scanh_add<<<(unsigned)nt, kRadixThreads, 0, st>>>(a, m, tmp);
  return cudaGetLastError();
}

cudaError_t radix_sort_index(int64_t n, int bits, int32_t* keys, int32_t* keys_tmp, int32_t* vals_out,
                             int32_t* vals_tmp, int32_t* hist, cudaStream_t st) {
  return radix_sort_impl<int32_t>(n, bits, keys, keys_tmp, vals_out, vals_tmp, hist, st);
}

cudaError_t radix_sort_index64(int64_t n, int bits, uint64_t* keys, uint64_t* keys_tmp,
                               int32_t* vals_out, int32_t* vals_tmp, int32_t* hist, cudaStream_t st) {
  return radix_sort_impl<uint64_t>(n, bits, keys, keys_tmp, vals_out, vals_tmp, hist, st);
}

}  // namespace sphh
