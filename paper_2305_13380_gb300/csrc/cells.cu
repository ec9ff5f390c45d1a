// cells.cu -- cell grid construction on the device (Sec. 2.1, the Verlet-list
// grid whose cells are at least the search radius wide).
//
// Pipeline (all sizes that depend on the data stay on the device, so a whole
// step can be captured in a CUDA graph):
//   k_grid_setup   per simulation: max h -> cells per side n_c
//   k_grid_base    prefix of n_c^3 over simulations -> global cell ids
//   k_key_count    FP64 cell coordinates, cell id, per-cell count
//   k_scan_*       exclusive scan of the counts -> cell_start
//   radix sort     stable sort of (cell id, particle index) -> perm, so the
//                  order inside a cell is ascending index for any cell size
//                  (radix.cu)
//   k_gather_*     sorted float copies relative to each particle's cell
#include "sph_internal.cuh"
#include "sph_launch.h"

namespace sphk {

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Cells-per-side bound of a simulation of n particles: n_c^3 <= k n + 216
// (k = 8 for the SPH loops; friends-of-friends asks for more).
__device__ __forceinline__ int32_t cap_cells_per_side(int64_t n, int k) {
  double lim = (double)k * (double)n + 216.0;
  int32_t c = (int32_t)cbrt(lim);
  while ((double)(c + 1) * (c + 1) * (c + 1) <= lim) ++c;
  while (c > 3 && (double)c * c * c > lim) --c;
  return c;
}

// max h per simulation.  Non-negative floats order like their bit patterns,
// so each thread keeps a running maximum for its simulation, lanes of one
// simulation combine with shuffles and one of them publishes with an integer
// atomicMax.  Non-positive and NaN values are ignored.
__global__ void k_grid_hmax(const int64_t* __restrict__ sim_offset, int n_sims, int64_t n_total,
                            const float* __restrict__ h, int32_t* __restrict__ hmax_bits) {
  const WarpRange wr = warp_range(n_total);
  SimCursor sc;
  int cur = -1;
  float m = 0.0f;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(sim_offset, n_sims, p);
    if (s != cur) {
      if (cur >= 0 && m > 0.0f) atomicMax(&hmax_bits[cur], __float_as_int(m));
      cur = s;
      m = 0.0f;
    }
    const float v = h[p];
    if (v > m) m = v;
  }
  const unsigned grp = __match_any_sync(0xffffffffu, cur);
  for (int o = 0; o < 32; ++o) {
    const float other = __shfl_sync(0xffffffffu, m, o);
    if ((grp >> o) & 1u) m = fmaxf(m, other);
  }
  if (cur >= 0 && m > 0.0f && (threadIdx.x & 31) == __ffs(grp) - 1)
    atomicMax(&hmax_bits[cur], __float_as_int(m));
}

// One thread per simulation: cells per side from max h.
// radius > 0: the search radius is given (friends-of-friends), not derived
// from the smoothing lengths.
__global__ void k_grid_setup(const int64_t* __restrict__ sim_offset, const double* __restrict__ box,
                             const int32_t* __restrict__ hmax_bits, int n_sims, double margin,
                             double radius, int cells_per_particle, double gamma_k,
                             GridDev* __restrict__ grid, int32_t* __restrict__ misc) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sims; s += gridDim.x * blockDim.x) {
    const int64_t a = sim_offset[s], b = sim_offset[s + 1];
    const float m = __int_as_float(hmax_bits[s]);
    const double L = box[s];
    const double Hmax = radius > 0.0 ? radius : gamma_k * (double)m * (1.0 + margin);
    const int32_t cap = cap_cells_per_side(b - a, cells_per_particle);
    int32_t nc = cap;
    if (Hmax > 0.0) {
      const double t = floor(L / Hmax);
      nc = t < (double)cap ? (int32_t)t : cap;
    }
    // Any n_c >= 1 gives exact sums while H <= min(cell, L/2): with fewer
    // than 3 cells per side the 27-cell stencil visits a cell's periodic
    // images twice, and the farther image lies at least L - H >= H away,
    // where the kernel is exactly zero.  Supports above L/2 would break the
    // minimum image.
    if (Hmax > 0.5 * L) atomicOr(&misc[kStatus], SPH_ST_BOX);
    if (nc < 1) nc = 1;
    GridDev g;
    g.L = L;
    g.n_c = nc;
    g.cell = L / (double)nc;
    g.cell_f = (float)g.cell;
    g.reach_f = g.cell_f;
    g.scale_f = (float)((double)nc / L);
    g.cell_base = 0;
    g.blk_base = 0;
    g.part_base = a;
    g.n = b - a;
    grid[s] = g;
  }
}

__global__ void k_grid_base(GridDev* __restrict__ grid, int n_sims, int32_t* __restrict__ misc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t base = 0, bbase = 0;
  for (int s = 0; s < n_sims; ++s) {
    grid[s].cell_base = (int32_t)base;
    grid[s].blk_base = (int32_t)bbase;
    const int64_t nc = grid[s].n_c;
    const int64_t nb = (nc + 1) / 2;
    base += nc * nc * nc;
    bbase += nb * nb * nb;
  }
  misc[kTotalCells] = (int32_t)base;
  misc[kTotalBlocks] = (int32_t)bbase;
}

__global__ void k_zero_counts(int32_t* __restrict__ count, const int32_t* __restrict__ misc) {
  const int32_t total = misc[kTotalCells];
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= total; c += gridDim.x * blockDim.x)
    count[c] = 0;
}

__global__ void k_key_count(int64_t n_total, const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ z, const int64_t* __restrict__ sim_offset,
                            int n_sims, const GridDev* __restrict__ grid, int32_t* __restrict__ key,
                            int32_t* __restrict__ sort_key, int32_t* __restrict__ count) {
  const WarpRange wr = warp_range(n_total);
  SimCursor sc;
  for (int64_t p = wr.lo + (threadIdx.x & 31); p < wr.hi; p += 32) {
    const int s = sc.at(sim_offset, n_sims, p);
    const GridDev G = grid[s];
    const int32_t kx = cell_coord_fast(x[p], G.L, G.n_c, G.scale_f);
    const int32_t ky = cell_coord_fast(y[p], G.L, G.n_c, G.scale_f);
    const int32_t kz = cell_coord_fast(z[p], G.L, G.n_c, G.scale_f);
    const int32_t k = G.cell_base + kx + G.n_c * (ky + G.n_c * kz);
    key[p] = k;
    sort_key[p] = k;
    // neighbours in index order often share a cell: one atomic per distinct
    // cell of the converged lanes
    const unsigned peers = __match_any_sync(__activemask(), k);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&count[k], __popc(peers));
  }
}

// ---- exclusive scan with a device-side length ------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total) {
  __shared__ int32_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < kScanThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < kScanThreads / 32) ws[lane] = s;
  }
  __syncthreads();
  const int32_t before = (w > 0 ? ws[w - 1] : 0) + x - v;
  *total = ws[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

// count[0 .. total) -> out (tile-local exclusive), tile sums -> sums
__device__ __forceinline__ void scan_tile(const int32_t* __restrict__ count, int32_t* __restrict__ out,
                                          int32_t* __restrict__ sums, int32_t total, int64_t tile) {
  const int64_t base = tile * kScanTile;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t c = base + threadIdx.x * kScanItems + i;
    v[i] = c < total ? count[c] : 0;
    s += v[i];
  }
  int32_t tot;
  int32_t run = block_exclusive_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t c = base + threadIdx.x * kScanItems + i;
    if (c < total) out[c] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) sums[tile] = tot;
}

// (tiles in a block-uniform grid-stride loop: the grid is sized for the
// capacity, the cell count is only known on the device)
__global__ void k_scan_tiles(const int32_t* __restrict__ count, int32_t* __restrict__ out,
                             int32_t* __restrict__ sums, const int32_t* __restrict__ misc) {
  const int32_t total = misc[kTotalCells];
  for (int64_t tile = blockIdx.x; tile * kScanTile < total; tile += gridDim.x)
    scan_tile(count, out, sums, total, tile);
}

// single block: exclusive scan of the tile sums; writes out[total] = grand total
__global__ void k_scan_sums(int32_t* __restrict__ sums, int32_t* __restrict__ out,
                            const int32_t* __restrict__ misc) {
  const int32_t total = misc[kTotalCells];
  const int32_t nt = (total + kScanTile - 1) / kScanTile;
  int32_t carry = 0;
  for (int32_t b0 = 0; b0 < nt; b0 += kScanThreads) {
    const int32_t i = b0 + threadIdx.x;
    const int32_t v = i < nt ? sums[i] : 0;
    int32_t tot;
    const int32_t ex = block_exclusive_scan(v, &tot);
    if (i < nt) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) out[total] = carry;
}

__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ sums,
                           const int32_t* __restrict__ misc) {
  const int32_t total = misc[kTotalCells];
  for (int64_t tile = blockIdx.x; tile * kScanTile < total; tile += gridDim.x) {
    const int64_t base = tile * kScanTile;
    const int32_t add = sums[tile];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
      const int64_t c = base + i;
      if (c < total) out[c] += add;
    }
  }
}

// Sorted copies for the density loop: position relative to the own cell's
// lower corner (computed in FP64, rounded once), mass, velocity, u, h.
__global__ void k_gather_density(int64_t n_total, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ key, const GridDev* __restrict__ grid,
                                 int n_sims, const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ z, const float* __restrict__ vx,
                                 const float* __restrict__ vy, const float* __restrict__ vz,
                                 const float* __restrict__ m, const float* __restrict__ u,
                                 const float* __restrict__ h, float4* __restrict__ pos4,
                                 float4* __restrict__ vel4, float* __restrict__ hs,
                                 const uint8_t* __restrict__ blk_need) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[s];
    const int32_t c = key[p];
    const GridDev G = grid[sim_of_cell(grid, n_sims, c)];
    if (blk_need != nullptr && !blk_need[block_of_cell(c, G)]) continue;
    const int32_t local = c - G.cell_base;
    const int32_t kx = local % G.n_c, ky = (local / G.n_c) % G.n_c, kz = local / (G.n_c * G.n_c);
    const float rx = (float)cell_offset(x[p], kx, G);
    const float ry = (float)cell_offset(y[p], ky, G);
    const float rz = (float)cell_offset(z[p], kz, G);
    pos4[s] = make_float4(rx, ry, rz, m[p]);
    vel4[s] = make_float4(vx[p], vy[p], vz[p], u[p]);
    hs[s] = h[p];
  }
}

// Sorted copies for the force loop: position relative to the own cell with
// the support H, velocity with the mass, (f P / rho^2, f, c, B), (rho, 1/H).
// kPos = false: fA.xyz already holds this build's positions (the density
// gather of the same step wrote them, or the nested-grid loops, which read
// positions elsewhere, do not use them); only H is written, and no FP64
// arithmetic is needed.
template <bool kPos>
__global__ void k_gather_force(int64_t n_total, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ key, const GridDev* __restrict__ grid,
                               int n_sims, const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, const float* __restrict__ vx,
                               const float* __restrict__ vy, const float* __restrict__ vz,
                               const float* __restrict__ m, const float* __restrict__ h,
                               const float* __restrict__ rho, const float* __restrict__ f,
                               const float* __restrict__ P, const float* __restrict__ c,
                               const float* __restrict__ B, float4* __restrict__ fA,
                               float4* __restrict__ fB, float4* __restrict__ fC,
                               float2* __restrict__ fD, const float4* __restrict__ trel,
                               const int4* __restrict__ tfine, float4* __restrict__ rec, float gamma_k,
                               const uint8_t* __restrict__ blk_need) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[s];
    if (blk_need != nullptr) {
      const int32_t cc = key[p];
      if (!blk_need[block_of_cell(cc, grid[sim_of_cell(grid, n_sims, cc)])]) continue;
    }
    const float H = gamma_k * h[p];
    if (rec != nullptr) {
      // nested grids: one record per source (the arrays below are not read)
      const float4 rl = trel[s];
      const int4 fn = tfine[s];
      const float r = rho[p];
      float4* o = rec + 4 * s;
      o[0] = make_float4(rl.x, rl.y, rl.z, H);
      o[1] = make_float4(__int_as_float(fn.x), __int_as_float(fn.y), __int_as_float(fn.z), r);
      o[2] = make_float4(vx[p], vy[p], vz[p], m[p]);
      o[3] = make_float4(f[p] * P[p] / (r * r), f[p], c[p], B[p]);
      continue;
    }
    if (kPos) {
      const int32_t cc = key[p];
      const GridDev G = grid[sim_of_cell(grid, n_sims, cc)];
      const int32_t local = cc - G.cell_base;
      const int32_t kx = local % G.n_c, ky = (local / G.n_c) % G.n_c, kz = local / (G.n_c * G.n_c);
      const float rx = (float)cell_offset(x[p], kx, G);
      const float ry = (float)cell_offset(y[p], ky, G);
      const float rz = (float)cell_offset(z[p], kz, G);
      fA[s] = make_float4(rx, ry, rz, H);
    } else {
      reinterpret_cast<float*>(fA)[4 * s + 3] = H;
    }
    fB[s] = make_float4(vx[p], vy[p], vz[p], m[p]);
    const float r = rho[p];
    fC[s] = make_float4(f[p] * P[p] / (r * r), f[p], c[p], B[p]);
    fD[s] = make_float2(r, 1.0f / H);
  }
}

// blk_need[b] = 1 where block b or one of its 26 periodic neighbours holds an
// active particle (simulation 0): the blocks whose cells the masked loops
// stage or walk.
__global__ void k_dilate_blocks(const GridDev* __restrict__ grid, const int32_t* __restrict__ total_blocks,
                                const uint8_t* __restrict__ blk_any, uint8_t* __restrict__ blk_need) {
  const GridDev G = grid[0];
  const int32_t nb = (G.n_c + 1) >> 1, nblk = *total_blocks;
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
    const int32_t l = b - G.blk_base;
    const int32_t bx = l % nb, by = (l / nb) % nb, bz = l / (nb * nb);
    uint8_t any = 0;
    for (int dz = -1; dz <= 1 && !any; ++dz)
      for (int dy = -1; dy <= 1 && !any; ++dy)
        for (int dx = -1; dx <= 1 && !any; ++dx) {
          const int32_t x = (bx + dx + nb) % nb, y = (by + dy + nb) % nb, z = (bz + dz + nb) % nb;
          any = blk_any[G.blk_base + x + nb * (y + nb * z)];
        }
    blk_need[b] = any;
  }
}

// Sorted copy of an active mask, act_s[s] = active[perm[s]], and the
// 2x2x2-cell blocks (of simulation 0) that hold an active particle.
__global__ void k_gather_mask(int64_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ key,
                              const GridDev* __restrict__ grid, const uint8_t* __restrict__ active,
                              uint8_t* __restrict__ act_s, uint8_t* __restrict__ blk_any) {
  const GridDev G = grid[0];
  const int32_t nc = G.n_c, nb = (nc + 1) >> 1;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[s];
    const uint8_t on = active[p];
    act_s[s] = on;
    if (on) {
      const int32_t c = key[p] - G.cell_base;
      const int32_t kx = c % nc, ky = (c / nc) % nc, kz = c / (nc * nc);
      blk_any[G.blk_base + (kx >> 1) + nb * ((ky >> 1) + nb * (kz >> 1))] = 1;
    }
  }
}

}  // namespace sphk

// ---- host launchers --------------------------------------------------------
namespace sphh {
using namespace sphk;

static int grid_for(int64_t n, int threads, int max_blocks) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

cudaError_t launch_build(const BuildArgs& a, cudaStream_t st) {
  if (cudaMemsetAsync(a.hmax_bits, 0, sizeof(int32_t) * a.n_sims, st) != cudaSuccess) return cudaGetLastError();
  if (a.n_total > 0 && !(a.radius > 0.0)) {
    int64_t hb = (a.n_total + 255) / 256;
    if (hb > (int64_t)a.num_sms * 8) hb = (int64_t)a.num_sms * 8;
    k_grid_hmax<<<(int)hb, 256, 0, st>>>(a.sim_offset, a.n_sims, a.n_total, a.h, a.hmax_bits);
  }
  k_grid_setup<<<(a.n_sims + 127) / 128, 128, 0, st>>>(a.sim_offset, a.box, a.hmax_bits, a.n_sims,
                                                       a.margin, a.radius, a.cells_per_particle, a.gamma_k,
                                                       a.grid, a.misc);
  k_grid_base<<<1, 32, 0, st>>>(a.grid, a.n_sims, a.misc);
  // grids sized for the capacity but capped: the kernels loop up to the
  // device-side cell count, and idle blocks would only cost launch time
  const int zb = grid_for(a.cap_cells + 1, 256, a.num_sms * 8);
  k_zero_counts<<<zb, 256, 0, st>>>(a.count, a.misc);
  const int pb = grid_for(a.n_total, 256, 65535);
  if (a.n_total > 0)
    k_key_count<<<pb, 256, 0, st>>>(a.n_total, a.x, a.y, a.z, a.sim_offset, a.n_sims, a.grid, a.key,
                                    a.slot, a.count);  // slot receives a copy of the keys to sort
  const int tb = grid_for(a.cap_cells, kScanTile, a.num_sms * 4);
  k_scan_tiles<<<tb, kScanThreads, 0, st>>>(a.count, a.cell_start, a.scan_sums, a.misc);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(a.scan_sums, a.cell_start, a.misc);
  k_scan_add<<<tb, kScanThreads, 0, st>>>(a.cell_start, a.scan_sums, a.misc);
  if (a.n_total > 0 && a.sort_cells) {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) <= a.cap_cells) ++bits;
    const cudaError_t e = radix_sort_index(a.n_total, bits, a.slot, a.rk, a.perm, a.rv, a.hist, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_density(const GatherDensityArgs& a, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  k_gather_density<<<grid_for(a.n_total, 256, 65535), 256, 0, st>>>(
      a.n_total, a.perm, a.key, a.grid, a.n_sims, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.m, a.u, a.h,
      a.pos4, a.vel4, a.hs, a.blk_need);
  return cudaGetLastError();
}

cudaError_t launch_gather_force(const GatherForceArgs& a, cudaStream_t st) {
  if (a.n_total <= 0) return cudaSuccess;
  auto kern = a.positions ? k_gather_force<true> : k_gather_force<false>;
  kern<<<grid_for(a.n_total, 256, 65535), 256, 0, st>>>(
      a.n_total, a.perm, a.key, a.grid, a.n_sims, a.x, a.y, a.z, a.vx, a.vy, a.vz, a.m, a.h, a.rho,
      a.f, a.P, a.c, a.B, a.fA, a.fB, a.fC, a.fD, a.rel, a.fine, a.rec, a.gamma_k, a.blk_need);
  return cudaGetLastError();
}

cudaError_t launch_dilate_blocks(const GridDev* grid, const int32_t* total_blocks, const uint8_t* blk_any,
                                 uint8_t* blk_need, int64_t blk_cap, cudaStream_t st) {
  k_dilate_blocks<<<grid_for(blk_cap, 256, 65535), 256, 0, st>>>(grid, total_blocks, blk_any, blk_need);
  return cudaGetLastError();
}

cudaError_t launch_gather_mask(int64_t n, const int32_t* perm, const int32_t* key, const GridDev* grid,
                               const uint8_t* active, uint8_t* act_s, uint8_t* blk_any, int64_t blk_cap,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(blk_any, 0, (size_t)blk_cap, st);
  if (e != cudaSuccess) return e;
  k_gather_mask<<<grid_for(n, 256, 65535), 256, 0, st>>>(n, perm, key, grid, active, act_s, blk_any);
  return cudaGetLastError();
}

}  // namespace sphh
