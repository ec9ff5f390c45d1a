// static_build.cu -- sph_build_cells_static: the cell build for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or arena, real-time loops whose allocator must not
// synchronise the device, or plugins that are only handed buffers by their
// host.  For them this entry point runs the same cell build as
// sph_build_cells, but every scratch array it needs (cell keys and their
// sort buffers, per-cell counts, scan partials, the grid record and status
// words) lives in one file-scope __device__ array of fixed size.  The caller passes
// the inputs and the outputs; nothing is allocated or freed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sph_internal.cuh"
#include "sph_launch.h"

namespace {

// Largest build served by the fixed scratch.
constexpr int64_t kStaticMaxN = 65536;
constexpr int64_t kStaticMaxCells = 8 * kStaticMaxN + 216;
constexpr int64_t kStaticScanSums = kStaticMaxCells / 1024 + 2;
constexpr int64_t kStaticHist = 256 * ((kStaticMaxN + 2047) / 2048) + 16;

// Layout of the scratch, in 4-byte words, each part 256-byte aligned.
constexpr int64_t align64(int64_t w) { return (w + 63) / 64 * 64; }
constexpr int64_t kOffGrid = 0;  // one GridDev
constexpr int64_t kOffOffset = kOffGrid + align64(sizeof(sphk::GridDev) / 4);  // int64[2]
constexpr int64_t kOffBox = kOffOffset + 64;                                     // double[1]
constexpr int64_t kOffMisc = kOffBox + 64;                                       // int32[8]
constexpr int64_t kOffHmax = kOffMisc + 64;                                      // int32[1]
constexpr int64_t kOffKey = kOffHmax + 64;
constexpr int64_t kOffSlot = kOffKey + align64(kStaticMaxN);
constexpr int64_t kOffCount = kOffSlot + align64(kStaticMaxN);
constexpr int64_t kOffSums = kOffCount + align64(kStaticMaxCells + 1);
constexpr int64_t kOffRk = kOffSums + align64(kStaticScanSums);
constexpr int64_t kOffRv = kOffRk + align64(kStaticMaxN);
constexpr int64_t kOffHist = kOffRv + align64(kStaticMaxN);
constexpr int64_t kWords = kOffHist + align64(kStaticHist);

// The scratch.  Every GPU that loads the library holds it (about 3.1 MB)
// until the process exits.
static __device__ __align__(256) int32_t g_scratch[kWords];

// Device address of g_scratch per device, resolved once per device and kept
// for the life of the process (a cudaDeviceReset would make it stale).
std::mutex g_mu;
int32_t* g_addr[64] = {nullptr};

__global__ void k_static_prepare(int64_t n, double box, int64_t* off, double* bx, int32_t* misc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    off[0] = 0;
    off[1] = n;
    bx[0] = box;
    for (int i = 0; i < sphk::kMiscWords; ++i) misc[i] = 0;
  }
}

__global__ void k_static_finish(const sphk::GridDev* grid, const int32_t* misc, int32_t* n_c_out,
                                int32_t* status_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (n_c_out) *n_c_out = grid[0].n_c;
    if (status_out) *status_out = misc[sphk::kStatus];
  }
}

}  // namespace

extern "C" int sph_build_cells_static(int64_t n, const double* x, const double* y, const double* z,
                                      const float* h, double box_size, double cell_margin,
                                      int32_t* cell_start, int64_t cell_start_cap, int32_t* perm,
                                      int32_t* n_c_out, int32_t* status_out, void* stream) {
  if (n < 0 || !(box_size > 0.0) || !(cell_margin >= 0.0) || !cell_start) return SPH_E_INVAL;
  if (n > 0 && (!x || !y || !z || !h || !perm)) return SPH_E_INVAL;
  if (n > kStaticMaxN) return SPH_E_CAPACITY;
  const int64_t cells = 8 * n + 216;
  if (cell_start_cap < cells + 1) return SPH_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPH_E_CUDA;
  int32_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // host code only holds a stand-in for g_scratch: resolve the device
      // address with this device current
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
        cudaGetLastError();
        return SPH_E_CUDA;
      }
      g_addr[dev] = static_cast<int32_t*>(p);
    }
    base = g_addr[dev];
  }
  int num_sms = 1;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPH_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  sphk::GridDev* grid = reinterpret_cast<sphk::GridDev*>(base + kOffGrid);
  int64_t* off = reinterpret_cast<int64_t*>(base + kOffOffset);
  double* bx = reinterpret_cast<double*>(base + kOffBox);
  int32_t* misc = base + kOffMisc;
  k_static_prepare<<<1, 32, 0, st>>>(n, box_size, off, bx, misc);
  sphh::BuildArgs b;
  b.n_sims = 1;
  b.n_total = n;
  b.cap_cells = cells;
  b.num_sms = num_sms;
  b.margin = cell_margin;
  b.sim_offset = off;
  b.box = bx;
  b.x = x;
  b.y = y;
  b.z = z;
  b.h = h;
  b.grid = grid;
  b.misc = misc;
  b.hmax_bits = base + kOffHmax;
  b.key = base + kOffKey;
  b.slot = base + kOffSlot;
  b.count = base + kOffCount;
  b.cell_start = cell_start;
  b.scan_sums = base + kOffSums;
  b.perm = perm;
  b.rk = base + kOffRk;
  b.rv = base + kOffRv;
  b.hist = base + kOffHist;
  if (sphh::launch_build(b, st) != cudaSuccess) return SPH_E_CUDA;
  k_static_finish<<<1, 32, 0, st>>>(grid, misc, n_c_out, status_out);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
