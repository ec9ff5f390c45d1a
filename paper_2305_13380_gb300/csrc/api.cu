// api.cu -- the C ABI declared in include/sph.h: context and scratch
// management, argument checks and the order of the kernel launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <cstddef>
#include <new>
#include <vector>

#include "blocks.cuh"
#include "sph_internal.cuh"
#include "sph_launch.h"
#include "tree.cuh"

using sphk::GridDev;
using sphk::PhysDev;

struct sph_ctx {
  sph_params p;
  cudaStream_t st = nullptr;
  int device = 0;
  int num_sms = 1;
  // capacities of the scratch below
  int64_t cap_n = 0;
  int64_t cap_cells = 0;
  int cap_sims = 0;
  // fixed buffers
  int32_t* misc = nullptr;
  unsigned long long* pairs = nullptr;
  int64_t* off1 = nullptr;  // single-simulation tables (device)
  double* box1 = nullptr;
  int64_t* h_off1 = nullptr;  // pinned mirrors
  double* h_box1 = nullptr;
  // grown buffers
  GridDev* grid = nullptr;
  int32_t *key = nullptr, *slot = nullptr, *count = nullptr, *cell_start = nullptr;
  int32_t *scan_sums = nullptr, *perm = nullptr, *overflow = nullptr;
  int32_t *rk = nullptr, *rv = nullptr, *rhist = nullptr;
  float4 *pos4 = nullptr, *vel4 = nullptr, *th4 = nullptr;
  float* hs = nullptr;
  float2* fD = nullptr;
  unsigned* dt_bits = nullptr;
  float* dt_f = nullptr;  // per simulation: 0.5 dt, dt / 3 (FP32)
  int32_t* hmax_bits = nullptr;
  uint16_t *lists = nullptr, *list_cnt = nullptr;
  bool lists_valid = false;  // lists belong to the current build
  uint16_t* axis = nullptr;  // per-cell axis orders (SPH_FLAG_AXIS_SORT), kAxes * cap_axis
  int64_t cap_axis = 0;
  float *vpx = nullptr, *vpy = nullptr, *vpz = nullptr, *up = nullptr;
  // nested-grid scratch (SPH_FLAG_TREE), grown separately
  int64_t cap_tree = 0;
  int64_t rev_cap = 0;
  uint64_t *key64 = nullptr, *key64_b = nullptr, *key64_c = nullptr, *skey = nullptr;
  int32_t *tgt = nullptr, *flag = nullptr, *leaf_of = nullptr, *n_leaves = nullptr;
  int8_t *level = nullptr, *fb_level = nullptr;
  int32_t* fb_list = nullptr;
  sphk::TreeLeaf* leaves = nullptr;
  sphk::TreeRange* ranges = nullptr;
  float *leaf_side = nullptr, *lrad = nullptr;
  int4* fine = nullptr;
  float4* rel = nullptr;
  float4* trec = nullptr;  // force records of the nested grids, 4 per particle
  uint8_t* act_s = nullptr;         // sorted active mask (masked loops)
  int32_t* act_pre = nullptr;       // nested grids: its exclusive prefix sums (n + 1)
  uint8_t* blk_any = nullptr;       // blocks holding an active particle
  uint8_t* blk_need = nullptr;      // those blocks and their neighbours (the gathers' set)
  int64_t cap_act = 0, cap_blk = 0;
  const uint8_t* lists_mask = nullptr;  // the mask the current lists were built with
  uint8_t* hact = nullptr;   // time-step hierarchy: active mask (input order)
  int32_t* hbin = nullptr;   // proposed bins
  int32_t* hwake = nullptr;  // wake-up bins
  int32_t* hcellmin = nullptr;  // per cell: the smallest bin of its inactive particles
  unsigned long long* htick = nullptr;
  int64_t cap_hier = 0;
  // cells kept across sub-steps (SPH_HIER_KEEP_CELLS): the build they come
  // from, its cell side, and the drift bound accumulated since
  int64_t build_epoch = 0, hier_epoch = -1, hier_n = -1;
  double hier_cell = 0.0, hier_drift = 0.0;
  float4* sx4 = nullptr;   // SPHENIX: sorted (u, alpha_V, P, alpha_c)
  float* dvp = nullptr;    // SPHENIX step: the divergence of the previous evaluation
  int64_t cap_sx = 0;
  uint32_t* tlists = nullptr;
  uint64_t* rev_raw = nullptr;
  uint32_t* rev = nullptr;
  unsigned long long* rev_count = nullptr;
  int32_t *rev_start = nullptr, *rev_fill = nullptr;
  bool built_tree = false;
  // symmetric force (SPH_FLAG_SYMMETRIC): the density's lists hold only the
  // later sources; records of the partners' sides and their grouping
  bool lists_upper = false;
  int64_t cap_sym = 0, cap_sym_rec = 0;
  float4* sym_a = nullptr;
  int2* sym_b = nullptr;
  int32_t *sym_recv = nullptr, *sym_order = nullptr, *sym_cnt = nullptr, *sym_off = nullptr;
  int32_t *sym_cursor = nullptr, *sym_tiles = nullptr, *sym_counter = nullptr;
  // CUDA-event timing of kernel groups (SPH_FLAG_TIMING)
  std::vector<cudaEvent_t> ev_start[SPH_T_COUNT], ev_stop[SPH_T_COUNT];
  int ev_used[SPH_T_COUNT] = {0, 0, 0, 0, 0};
  double t_ms[SPH_T_COUNT] = {0, 0, 0, 0, 0};
  int64_t t_calls[SPH_T_COUNT] = {0, 0, 0, 0, 0};
  // last build
  int built_sims = 0;
  int64_t built_n = -1;
  const int64_t* built_offset = nullptr;
};

namespace {

template <class T>
void dfree(T*& ptr) {
  if (ptr) cudaFree((void*)ptr);
  ptr = nullptr;
}

template <class T>
bool dalloc(T*& ptr, int64_t count) {
  void* v = nullptr;
  if (cudaMalloc(&v, (size_t)(count > 0 ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
    return false;
  }
  ptr = (T*)v;
  return true;
}

void free_grown(sph_ctx* c) {
  dfree(c->grid);
  dfree(c->key);
  dfree(c->slot);
  dfree(c->count);
  dfree(c->cell_start);
  dfree(c->scan_sums);
  dfree(c->perm);
  dfree(c->rk);
  dfree(c->rv);
  dfree(c->rhist);
  dfree(c->overflow);
  dfree(c->pos4);
  dfree(c->vel4);
  dfree(c->th4);
  dfree(c->hs);
  dfree(c->fD);
  dfree(c->dt_bits);
  dfree(c->dt_f);
  dfree(c->hmax_bits);
  dfree(c->lists);
  dfree(c->list_cnt);
  dfree(c->axis);
  c->cap_axis = 0;
  dfree(c->vpx);
  dfree(c->vpy);
  dfree(c->vpz);
  dfree(c->up);
  c->cap_n = c->cap_cells = 0;
  c->cap_sims = 0;
}

void free_tree(sph_ctx* c) {
  dfree(c->key64);
  dfree(c->key64_b);
  dfree(c->key64_c);
  dfree(c->skey);
  dfree(c->tgt);
  dfree(c->level);
  dfree(c->fb_level);
  dfree(c->fb_list);
  dfree(c->flag);
  dfree(c->leaf_of);
  dfree(c->n_leaves);
  dfree(c->leaves);
  dfree(c->ranges);
  dfree(c->leaf_side);
  dfree(c->lrad);
  dfree(c->fine);
  dfree(c->rel);
  dfree(c->trec);
  dfree(c->tlists);
  dfree(c->rev_raw);
  dfree(c->rev);
  dfree(c->rev_count);
  dfree(c->rev_start);
  dfree(c->rev_fill);
  c->cap_tree = 0;
  c->rev_cap = 0;
  c->built_tree = false;
}

// Nested-grid scratch for n particles (after ensure()): keys, the two
// orders, target groups with their 27 neighbour ranges, tree-order copies, lists and the
// reverse pairs.  Every reverse pair is one of its emitter's in-support
// density pairs, whose total is ~50 per particle at the converged h; room
// starts at 64 per particle, and SPH_ST_CAPACITY in a synchronous step
// grows it to the emitted count.
int ensure_tree(sph_ctx* c, int64_t n, int64_t rev_need) {
  if (c->cap_tree > 0 && n <= c->cap_tree && rev_need <= c->rev_cap) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  const int64_t rev_old = c->rev_cap;
  free_tree(c);
  const int64_t cn = c->cap_n;
  int64_t rc = 64 * cn + 65536;
  if (rc < rev_need) rc = rev_need;
  if (rc < rev_old) rc = rev_old;
  if (rc > INT32_MAX) rc = INT32_MAX;
  bool ok = dalloc(c->key64, cn) && dalloc(c->key64_b, cn) && dalloc(c->key64_c, cn) &&
            dalloc(c->skey, cn) && dalloc(c->tgt, cn) && dalloc(c->flag, cn) && dalloc(c->level, cn) &&
            dalloc(c->fb_level, cn) && dalloc(c->fb_list, cn) && dalloc(c->leaf_of, cn) && dalloc(c->n_leaves, 1) &&
            dalloc(c->leaves, cn + 1) && dalloc(c->ranges, 27 * cn) && dalloc(c->leaf_side, cn) &&
            dalloc(c->lrad, cn) && dalloc(c->fine, cn) && dalloc(c->rel, cn) && dalloc(c->trec, 4 * cn) &&
            dalloc(c->tlists, (int64_t)sphk::kTreeListRegion * sphk::kTreeTpp * cn) &&
            dalloc(c->rev_raw, rc) && dalloc(c->rev, rc) && dalloc(c->rev_count, 1) &&
            dalloc(c->rev_start, cn + 1) && dalloc(c->rev_fill, cn);
  if (!ok) {
    free_tree(c);
    return SPH_E_NOMEM;
  }
  c->cap_tree = cn;
  c->rev_cap = rc;
  c->built_n = -1;
  c->lists_valid = false;
  return SPH_OK;
}

// Scratch for n particles in n_sims simulations; every simulation may use
// up to k n_s + 216 cells (k = cells_per_particle: 8 for the SPH loops), so
// the total is bounded by k n + 216 n_sims.
int ensure(sph_ctx* c, int64_t n, int n_sims, int cells_per_particle = 8) {
  const int64_t need_cells = cells_per_particle * n + 216 * (int64_t)n_sims;
  if (n <= c->cap_n && n_sims <= c->cap_sims && need_cells <= c->cap_cells) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  free_grown(c);
  const int64_t rev_keep = c->rev_cap;
  free_tree(c);
  c->rev_cap = rev_keep;
  const int64_t cn = n + n / 4 + 64;
  const int cs = n_sims + n_sims / 4 + 1;
  const int64_t cc = (cells_per_particle > 8 ? cells_per_particle : 8) * cn + 216 * (int64_t)cs;
  bool ok = dalloc(c->grid, cs) && dalloc(c->key, cn) && dalloc(c->slot, cn) &&
            dalloc(c->count, cc + 1) && dalloc(c->cell_start, cc + 1) &&
            dalloc(c->scan_sums, cc / 1024 + 2) && dalloc(c->perm, cn) &&
            dalloc(c->rk, cn) && dalloc(c->rv, cn) && dalloc(c->rhist, sphh::radix_hist_words(cn)) &&
            dalloc(c->overflow, (8 * cn + 216 * (int64_t)cs) / 3 + 2) && dalloc(c->pos4, cn) &&
            dalloc(c->vel4, cn) && dalloc(c->th4, cn) && dalloc(c->hs, cn) && dalloc(c->fD, cn) &&
            dalloc(c->dt_bits, cs) && dalloc(c->dt_f, 2 * cs) && dalloc(c->hmax_bits, cs) &&
            dalloc(c->lists, (int64_t)sphk::kListRegion * 4 * cn) &&
            dalloc(c->list_cnt, (int64_t)(sphk::kTreeTpp > 4 ? sphk::kTreeTpp : 4) * cn) &&
            dalloc(c->vpx, cn) && dalloc(c->vpy, cn) && dalloc(c->vpz, cn) && dalloc(c->up, cn) &&
            (!(c->p.flags & SPH_FLAG_AXIS_SORT) || dalloc(c->axis, (int64_t)sphk::kAxes * cn));
  if (!ok) {
    free_grown(c);
    return SPH_E_NOMEM;
  }
  if (c->p.flags & SPH_FLAG_AXIS_SORT) c->cap_axis = cn;
  c->cap_n = cn;
  c->cap_sims = cs;
  c->cap_cells = cc;
  c->lists_valid = false;
  c->built_n = -1;
  return SPH_OK;
}

// Scratch of the time-step hierarchy's sub-steps for n particles.
int ensure_hier(sph_ctx* c, int64_t n) {
  if (n <= c->cap_hier) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  dfree(c->hact);
  dfree(c->hbin);
  dfree(c->hwake);
  dfree(c->hcellmin);
  dfree(c->htick);
  c->cap_hier = 0;
  const int64_t cn = n + n / 4 + 64;
  // cells of one simulation: at most 8 n + 216 (the build's cap), + 1
  if (!(dalloc(c->hact, cn) && dalloc(c->hbin, cn) && dalloc(c->hwake, cn) && dalloc(c->hcellmin, 8 * cn + 217) &&
        dalloc(c->htick, 1))) {
    dfree(c->hact);
    dfree(c->hbin);
    dfree(c->hwake);
    dfree(c->hcellmin);
    dfree(c->htick);
    return SPH_E_NOMEM;
  }
  c->cap_hier = cn;
  return SPH_OK;
}

// Sorted active mask of the masked loops, for n particles.
// The block flags are sized by the cell capacity (at least one cell per block).
int ensure_act(sph_ctx* c, int64_t n) {
  if (n <= c->cap_act && c->cap_cells <= c->cap_blk) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  dfree(c->act_s);
  dfree(c->act_pre);
  dfree(c->blk_any);
  dfree(c->blk_need);
  c->cap_act = c->cap_blk = 0;
  const int64_t cn = n + n / 4 + 64;
  if (!dalloc(c->act_s, cn) || !dalloc(c->act_pre, cn + 1) || !dalloc(c->blk_any, c->cap_cells + 1) ||
      !dalloc(c->blk_need, c->cap_cells + 1)) {
    dfree(c->act_s);
    dfree(c->act_pre);
    dfree(c->blk_any);
    dfree(c->blk_need);
    return SPH_E_NOMEM;
  }
  c->cap_act = cn;
  c->cap_blk = c->cap_cells;
  return SPH_OK;
}

void free_sym(sph_ctx* c) {
  dfree(c->sym_a);
  dfree(c->sym_b);
  dfree(c->sym_recv);
  dfree(c->sym_order);
  dfree(c->sym_cnt);
  dfree(c->sym_off);
  dfree(c->sym_cursor);
  dfree(c->sym_tiles);
  dfree(c->sym_counter);
  c->cap_sym = c->cap_sym_rec = 0;
}

// Scratch of the symmetric force for n particles: room for 64 records (pairs
// met from the earlier particle) per particle; a lattice with ~48 neighbours
// needs ~24, a strongly clustered box on the uniform grid ~60.  More pairs
// set SPH_ST_CAPACITY.
constexpr int64_t kSymRecPerParticle = 64;
int ensure_sym(sph_ctx* c, int64_t n) {
  if (n <= c->cap_sym) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  free_sym(c);
  const int64_t cn = n + n / 4 + 64;
  const int64_t cr = kSymRecPerParticle * cn;
  if (!(dalloc(c->sym_a, cr) && dalloc(c->sym_b, cr) && dalloc(c->sym_recv, cr) && dalloc(c->sym_order, cr) &&
        dalloc(c->sym_cnt, cn) && dalloc(c->sym_off, cn + 1) && dalloc(c->sym_cursor, cn) &&
        dalloc(c->sym_tiles, sphh::sym_tiles(cn) + 2) && dalloc(c->sym_counter, 1))) {
    free_sym(c);
    return SPH_E_NOMEM;
  }
  c->cap_sym = cn;
  c->cap_sym_rec = cr;
  return SPH_OK;
}

// The symmetric force serves the Minimal flavour with the cubic spline on the
// uniform grid, all particles active.
bool sym_applies(const sph_ctx* c, const uint8_t* active) {
  return (c->p.flags & SPH_FLAG_SYMMETRIC) && !(c->p.flags & SPH_FLAG_TREE) && !c->built_tree &&
         c->p.kernel == SPH_KERNEL_CUBIC && active == nullptr;
}

// SPHENIX scratch for n particles (kept apart from the loops' scratch).
int ensure_sphenix(sph_ctx* c, int64_t n) {
  if (n <= c->cap_sx) return SPH_OK;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  dfree(c->sx4);
  dfree(c->dvp);
  c->cap_sx = 0;
  const int64_t cn = n + n / 4 + 64;
  if (!(dalloc(c->sx4, cn) && dalloc(c->dvp, cn))) {
    dfree(c->sx4);
    dfree(c->dvp);
    return SPH_E_NOMEM;
  }
  c->cap_sx = cn;
  return SPH_OK;
}

// Folds the recorded event pairs of group k into t_ms (waits for them).
void t_collect(sph_ctx* c, int k) {
  for (int i = 0; i < c->ev_used[k]; ++i) {
    float ms = 0.f;
    cudaEventSynchronize(c->ev_stop[k][i]);
    if (cudaEventElapsedTime(&ms, c->ev_start[k][i], c->ev_stop[k][i]) == cudaSuccess) c->t_ms[k] += ms;
  }
  c->ev_used[k] = 0;
  cudaGetLastError();
}

void t_begin(sph_ctx* c, int k) {
  if (!(c->p.flags & SPH_FLAG_TIMING)) return;
  if (c->ev_used[k] >= 1024) t_collect(c, k);
  const int i = c->ev_used[k];
  if (i == (int)c->ev_start[k].size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    c->ev_start[k].push_back(a);
    c->ev_stop[k].push_back(b);
  }
  cudaEventRecord(c->ev_start[k][i], c->st);
}

void t_end(sph_ctx* c, int k) {
  if (!(c->p.flags & SPH_FLAG_TIMING)) return;
  const int i = c->ev_used[k];
  if (i >= (int)c->ev_stop[k].size()) return;
  cudaEventRecord(c->ev_stop[k][i], c->st);
  c->ev_used[k] = i + 1;
  c->t_calls[k] += 1;
}

PhysDev phys_of(const sph_params& p) {
  PhysDev ph;
  ph.gamma = (float)p.gamma;
  ph.eta3 = (float)(p.eta * p.eta * p.eta);
  ph.alpha_v = (float)p.alpha_v;
  ph.beta_v = (float)p.beta_v;
  ph.eps_balsara = (float)p.eps_balsara;
  ph.h_tol = p.h_tol;
  ph.max_h_iter = p.max_h_iter;
  ph.count_pairs = (p.flags & SPH_FLAG_COUNT_PAIRS) ? 1 : 0;
  ph.kernel = p.kernel;
  ph.lanes = p.lanes_per_target;
  return ph;
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? SPH_OK : SPH_E_CUDA; }

// Maps device status bits to the most severe return code.
int code_of_status(int32_t s) {
  if (s & SPH_ST_BOX) return SPH_E_BOX;
  if (s & SPH_ST_CAPACITY) return SPH_E_CAPACITY;
  if (s & SPH_ST_REBUILD) return SPH_E_REBUILD;
  if (s & SPH_ST_H_NOCONV) return SPH_E_H_NOCONV;
  return SPH_OK;
}

int read_status(sph_ctx* c, int32_t* out) {
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  int32_t s = 0;
  if (cudaMemcpy(&s, c->misc + sphk::kStatus, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SPH_E_CUDA;
  if (cudaMemsetAsync(c->misc + sphk::kStatus, 0, sizeof(int32_t), c->st) != cudaSuccess)
    return SPH_E_CUDA;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  *out = s;
  return SPH_OK;
}

int finish(sph_ctx* c) {
  if (cudaGetLastError() != cudaSuccess) return SPH_E_CUDA;
  if (!(c->p.flags & SPH_FLAG_SYNC)) return SPH_OK;
  int32_t s = 0;
  int rc = read_status(c, &s);
  return rc != SPH_OK ? rc : code_of_status(s);
}

bool params_ok(const sph_params& p) {
  return p.box_size > 0 && p.gamma > 1 && p.eta > 0 && p.alpha_v >= 0 && p.beta_v >= 0 &&
         p.eps_balsara > 0 && p.h_tol > 0 && p.cfl > 0 && p.cell_margin >= 0 && p.max_h_iter > 0 &&
         (!(p.flags & SPH_FLAG_TREE) || p.n_leaf >= 1) && p.kernel >= SPH_KERNEL_CUBIC &&
         p.kernel <= SPH_KERNEL_WENDLAND_C2 &&
         (p.lanes_per_target == 0 || p.lanes_per_target == 2 || p.lanes_per_target == 4);
}

int do_build(sph_ctx* c, int n_sims, int64_t n_total, const int64_t* off, const double* box,
             const double* x, const double* y, const double* z, const float* h, double radius = 0.0,
             int cells_per_particle = 8) {
  ++c->build_epoch;
  sphh::BuildArgs b;
  b.gamma_k = sphk::kernel_gamma(c->p.kernel);
  b.radius = radius;
  b.cells_per_particle = cells_per_particle;
  b.n_sims = n_sims;
  b.n_total = n_total;
  b.cap_cells = cells_per_particle * n_total + 216 * (int64_t)n_sims;
  b.num_sms = c->num_sms;
  b.margin = c->p.cell_margin;
  b.sim_offset = off;
  b.box = box;
  b.x = x;
  b.y = y;
  b.z = z;
  b.h = h;
  b.grid = c->grid;
  b.misc = c->misc;
  b.hmax_bits = c->hmax_bits;
  b.key = c->key;
  b.slot = c->slot;
  b.count = c->count;
  b.cell_start = c->cell_start;
  b.scan_sums = c->scan_sums;
  b.perm = c->perm;
  b.rk = c->rk;
  b.rv = c->rv;
  b.hist = c->rhist;
  // a given radius (friends-of-friends) always builds the uniform grid
  const bool tree = (c->p.flags & SPH_FLAG_TREE) != 0 && !(radius > 0.0);
  b.sort_cells = tree ? 0 : 1;
  if (tree) {
    const int rc = ensure_tree(c, n_total, 0);
    if (rc != SPH_OK) return rc;
  }
  t_begin(c, SPH_T_BUILD);
  if (sphh::launch_build(b, c->st) != cudaSuccess) return SPH_E_CUDA;
  if (tree) {
    sphh::TreeBuildArgs t;
    t.gamma_k = (float)sphk::kernel_gamma(c->p.kernel);
    t.n_sims = n_sims;
    t.n_total = n_total;
    t.cap_cells = b.cap_cells;
    t.n_leaf = c->p.n_leaf;
    t.margin = c->p.cell_margin;
    t.sim_offset = off;
    t.grid = c->grid;
    t.x = x;
    t.y = y;
    t.z = z;
    t.h = h;
    t.cell_key = c->key;
    t.cell_start = c->cell_start;
    t.key64 = c->key64;
    t.key64_b = c->key64_b;
    t.key64_c = c->key64_c;
    t.skey = c->skey;
    t.perm = c->perm;
    t.tgt = c->tgt;
    t.rv = c->rv;
    t.hist = c->rhist;
    t.flag = c->flag;
    t.leaf_of = c->leaf_of;
    t.scan_tmp = c->scan_sums;
    t.leaves = c->leaves;
    t.n_leaves = c->n_leaves;
    t.ranges = c->ranges;
    t.leaf_side = c->leaf_side;
    t.level = c->level;
    if (sphh::launch_tree_build(t, c->st) != cudaSuccess) return SPH_E_CUDA;
  }
  t_end(c, SPH_T_BUILD);
  c->built_sims = n_sims;
  c->built_n = n_total;
  c->built_offset = off;
  c->built_tree = tree;
  c->lists_valid = false;
  return SPH_OK;
}

int do_tree_density(sph_ctx* c, const double* x, const double* y, const double* z, const float* vx,
                    const float* vy, const float* vz, const float* m, const float* u, const float* h_in,
                    float* h, float* rho, float* f, float* div_v, float* curl_v, float* P, float* cs,
                    float* B, int32_t* n_iter, const uint8_t* active) {
  sphh::TreeGatherArgs g;
  g.gamma_k = (float)sphk::kernel_gamma(c->p.kernel);
  g.n_total = c->built_n;
  g.n_sims = c->built_sims;
  g.perm = c->perm;
  g.skey = c->skey;
  g.grid = c->grid;
  g.x = x;
  g.y = y;
  g.z = z;
  g.m = m;
  g.vx = vx;
  g.vy = vy;
  g.vz = vz;
  g.u = u;
  g.h = h_in;
  g.leaf_side = c->leaf_side;
  g.list_reach = sphk::kTreeListReach;
  g.fine = c->fine;
  g.rel = c->rel;
  g.vel4 = c->vel4;
  g.hs = c->hs;
  g.lrad = c->lrad;
  t_begin(c, SPH_T_GATHER);
  if (sphh::launch_tree_gather(g, c->st) != cudaSuccess) return SPH_E_CUDA;
  t_end(c, SPH_T_GATHER);
  if (c->p.flags & SPH_FLAG_COUNT_PAIRS) {
    if (cudaMemsetAsync(c->pairs, 0, sizeof(unsigned long long), c->st) != cudaSuccess ||
        cudaMemsetAsync(c->pairs + 2, 0, sizeof(unsigned long long), c->st) != cudaSuccess)
      return SPH_E_CUDA;
  }
  sphh::TreeDensityArgs d;
  d.n_sims = c->built_sims;
  d.num_sms = c->num_sms;
  d.n_total = c->built_n;
  d.grid = c->grid;
  d.tgt = c->tgt;
  d.leaves = c->leaves;
  d.n_leaves = c->n_leaves;
  d.ranges = c->ranges;
  d.fine = c->fine;
  d.rel = c->rel;
  d.vel4 = c->vel4;
  d.hs = c->hs;
  d.lrad = c->lrad;
  d.leaf_side = c->leaf_side;
  d.perm = c->perm;
  d.status = c->misc + sphk::kStatus;
  d.pairs = c->pairs;
  d.h = h;
  d.rho = rho;
  d.f = f;
  d.div_v = div_v;
  d.curl_v = curl_v;
  d.P = P;
  d.c = cs;
  d.B = B;
  d.n_iter = n_iter;
  d.lists = c->tlists;
  d.list_cnt = c->list_cnt;
  d.rev_raw = c->rev_raw;
  d.rev_count = c->rev_count;
  d.rev_start = c->rev_start;
  d.rev_fill = c->rev_fill;
  d.rev = c->rev;
  d.rev_cap = c->rev_cap;
  d.scan_tmp = c->scan_sums;
  d.work = c->misc + sphk::kTreeWork;
  d.skey = c->skey;
  d.cell_start = c->cell_start;
  d.level = c->level;
  d.fb_list = c->fb_list;
  d.fb_count = c->misc + sphk::kTreeFbCount;
  d.fb_level = c->fb_level;
  d.fb_work = c->misc + sphk::kTreeFbWork;
  d.list_free = c->pairs + 2;
  if (active) {
    // masked loops: the mask in tree order
    const int rc = ensure_act(c, c->built_n);
    if (rc != SPH_OK) return rc;
    if (sphh::launch_tree_mask(c->built_n, c->perm, active, c->act_s, c->act_pre, c->scan_sums, c->st) !=
        cudaSuccess)
      return SPH_E_CUDA;
    d.act = c->act_s;
    d.act_pre = c->act_pre;
  }
  t_begin(c, SPH_T_DENSITY);
  const cudaError_t e = sphh::launch_tree_density(d, phys_of(c->p), c->st);
  t_end(c, SPH_T_DENSITY);
  c->lists_valid = (e == cudaSuccess);
  c->lists_mask = active;
  return cuda_code(e);
}

int do_density(sph_ctx* c, const double* x, const double* y, const double* z, const float* vx,
               const float* vy, const float* vz, const float* m, const float* u, const float* h_in,
               float* h, float* rho, float* f, float* div_v, float* curl_v, float* P, float* cs,
               float* B, int32_t* n_iter, const uint8_t* active = nullptr) {
  if (c->built_tree)
    return do_tree_density(c, x, y, z, vx, vy, vz, m, u, h_in, h, rho, f, div_v, curl_v, P, cs, B, n_iter, active);
  sphh::GatherDensityArgs g;
  g.n_total = c->built_n;
  g.n_sims = c->built_sims;
  g.perm = c->perm;
  g.key = c->key;
  g.grid = c->grid;
  g.x = x;
  g.y = y;
  g.z = z;
  g.vx = vx;
  g.vy = vy;
  g.vz = vz;
  g.m = m;
  g.u = u;
  g.h = h_in;
  g.pos4 = c->pos4;
  g.vel4 = c->vel4;
  g.hs = c->hs;
  if (active) {
    // the masked loops read only the blocks around the active particles:
    // the mask first, then the gather of those blocks' particles
    const int rc = ensure_act(c, c->built_n);
    if (rc != SPH_OK) return rc;
    if (sphh::launch_gather_mask(c->built_n, c->perm, c->key, c->grid, active, c->act_s, c->blk_any, c->cap_blk,
                                 c->st) != cudaSuccess ||
        sphh::launch_dilate_blocks(c->grid, c->misc + sphk::kTotalBlocks, c->blk_any, c->blk_need, c->cap_blk,
                                   c->st) != cudaSuccess)
      return SPH_E_CUDA;
    g.blk_need = c->blk_need;
  }
  t_begin(c, SPH_T_GATHER);
  if (sphh::launch_gather_density(g, c->st) != cudaSuccess) return SPH_E_CUDA;
  const bool axis = (c->p.flags & SPH_FLAG_AXIS_SORT) != 0;
  if (axis) {
    // per-cell orders along the neighbour axes, from this gather's positions
    // (the buffer is sized with the other scratch, so nothing is allocated
    // here, e.g. during graph capture)
    if (c->cap_axis < c->built_n) return SPH_E_INVAL;
    sphh::AxisSortArgs x;
    x.n_total = c->built_n;
    x.perm = c->perm;
    x.key = c->key;
    x.cell_start = c->cell_start;
    x.pos4 = c->pos4;
    x.order = c->axis;
    if (sphh::launch_axis_sort(x, c->st) != cudaSuccess) return SPH_E_CUDA;
  }
  t_end(c, SPH_T_GATHER);
  if (c->p.flags & SPH_FLAG_COUNT_PAIRS)
    if (cudaMemsetAsync(c->pairs, 0, sizeof(unsigned long long), c->st) != cudaSuccess)
      return SPH_E_CUDA;
  sphh::DensityArgs d;
  if (active) {
    d.act = c->act_s;
    d.blk_any = c->blk_any;
  }
  d.n_sims = c->built_sims;
  d.num_sms = c->num_sms;
  d.grid = c->grid;
  d.misc_ro = c->misc;
  d.misc = c->misc;
  d.overflow = c->overflow;
  d.status = c->misc + sphk::kStatus;
  d.pairs = c->pairs;
  d.cell_start = c->cell_start;
  d.perm = c->perm;
  d.pos4 = c->pos4;
  d.vel4 = c->vel4;
  d.hs = c->hs;
  d.h = h;
  d.rho = rho;
  d.f = f;
  d.div_v = div_v;
  d.curl_v = curl_v;
  d.P = P;
  d.c = cs;
  d.B = B;
  d.n_iter = n_iter;
  d.lists = c->lists;
  d.list_cnt = c->list_cnt;
  d.axis_order = axis ? c->axis : nullptr;
  d.axis_stride = c->built_n;
  const bool upper = sym_applies(c, active);
  d.upper = upper ? 1 : 0;
  t_begin(c, SPH_T_DENSITY);
  const cudaError_t e = sphh::launch_density(d, phys_of(c->p), c->st);
  t_end(c, SPH_T_DENSITY);
  c->lists_valid = (e == cudaSuccess);
  c->lists_mask = active;
  c->lists_upper = upper;
  return cuda_code(e);
}

bool sphenix_params_ok(const sph_sphenix_params& x) {
  return std::isfinite(x.alpha_v_max) && x.alpha_v_max > 0.0 && std::isfinite(x.ell) && x.ell >= 0.0 &&
         std::isfinite(x.beta_c) && x.beta_c >= 0.0 && std::isfinite(x.alpha_c_min) && x.alpha_c_min >= 0.0 &&
         std::isfinite(x.alpha_c_max) && x.alpha_c_max >= x.alpha_c_min;
}

sphk::SphenixDev sphenix_dev(const sph_sphenix_params& x, double dt, const double* dt_dev) {
  sphk::SphenixDev d;
  d.av_max = (float)x.alpha_v_max;
  d.ell = (float)x.ell;
  d.beta_c = (float)x.beta_c;
  d.ac_min = (float)x.alpha_c_min;
  d.ac_max = (float)x.alpha_c_max;
  d.dt = dt;
  d.dt_dev = dt_dev;
  return d;
}

// A pass of do_force with a fifth staged record E per source: the SPHENIX
// gradient pass (gradient = true: writes alpha_c_out and, if given, lap_u),
// the SPHENIX force (E gathered from u, alpha_v, P and alpha_c), or the
// time-step limiter (limit = true: E.x = the bins bins_in, result in
// bins_out).  skip_gather reuses the A..D records of the previous pass on the
// same build and inputs.
struct LoopPass {
  bool gradient = false;
  bool skip_gather = false;
  // the time-step limiter pass instead (bins_in gathered as the E records)
  bool limit = false;
  const int32_t* bins_in = nullptr;
  int32_t* bins_out = nullptr;
  const float *u = nullptr, *alpha_v = nullptr, *alpha_c = nullptr;
  float *alpha_c_out = nullptr, *lap_u = nullptr;
  sphk::SphenixDev x;
};

// The nested grids' force-pass arguments of the current build (lists,
// reverse pairs, records, fallback queue); outputs and flavour fields unset.
sphh::TreeForceArgs tree_force_args(sph_ctx* c) {
  sphh::TreeForceArgs a;
  a.n_sims = c->built_sims;
  a.num_sms = c->num_sms;
  a.grid = c->grid;
  a.tgt = c->tgt;
  a.leaves = c->leaves;
  a.n_leaves = c->n_leaves;
  a.ranges = c->ranges;
  a.fine = c->fine;
  a.rel = c->rel;
  a.lrad = c->lrad;
  a.leaf_side = c->leaf_side;
  a.perm = c->perm;
  a.rec = c->trec;
  a.lists = c->tlists;
  a.list_cnt = c->list_cnt;
  a.rev_start = c->rev_start;
  a.rev = c->rev;
  a.pairs = c->pairs + 1;
  a.work = c->misc + sphk::kTreeWork;
  a.n_total = c->built_n;
  a.skey = c->skey;
  a.cell_start = c->cell_start;
  a.fb_list = c->fb_list;
  a.fb_count = c->misc + sphk::kTreeFbCount;
  a.fb_level = c->fb_level;
  a.fb_work = c->misc + sphk::kTreeFbWork;
  return a;
}

int do_force(sph_ctx* c, const double* x, const double* y, const double* z, const float* vx,
             const float* vy, const float* vz, const float* m, const float* h, const float* rho,
             const float* f, const float* P, const float* cs, const float* B, float* ax, float* ay,
             float* az, float* du_dt, float* v_sig, bool pos_ready = false, const LoopPass* sx = nullptr,
             const uint8_t* active = nullptr) {
  sphh::GatherForceArgs g;
  g.gamma_k = (float)sphk::kernel_gamma(c->p.kernel);
  // the nested-grid force reads positions from its own copies (fA.w only)
  g.positions = (pos_ready || c->built_tree) ? 0 : 1;
  g.n_total = c->built_n;
  g.n_sims = c->built_sims;
  g.perm = c->perm;
  g.key = c->key;
  g.grid = c->grid;
  g.x = x;
  g.y = y;
  g.z = z;
  g.vx = vx;
  g.vy = vy;
  g.vz = vz;
  g.m = m;
  g.h = h;
  g.rho = rho;
  g.f = f;
  g.P = P;
  g.c = cs;
  g.B = B;
  g.fA = c->pos4;
  g.fB = c->vel4;
  g.fC = c->th4;
  g.fD = c->fD;
  if (c->built_tree) {
    g.rel = c->rel;
    g.fine = c->fine;
    g.rec = c->trec;
  }
  if (active && !c->built_tree) {
    // as in the density: the mask, and the gather of the blocks around it
    const int rc = ensure_act(c, c->built_n);
    if (rc != SPH_OK) return rc;
    if (sphh::launch_gather_mask(c->built_n, c->perm, c->key, c->grid, active, c->act_s, c->blk_any, c->cap_blk,
                                 c->st) != cudaSuccess ||
        sphh::launch_dilate_blocks(c->grid, c->misc + sphk::kTotalBlocks, c->blk_any, c->blk_need, c->cap_blk,
                                   c->st) != cudaSuccess)
      return SPH_E_CUDA;
    g.blk_need = c->blk_need;
  }
  t_begin(c, SPH_T_GATHER);
  if (!(sx && sx->skip_gather) && sphh::launch_gather_force(g, c->st) != cudaSuccess) return SPH_E_CUDA;
  if (sx && !sx->limit &&
      sphh::launch_gather_sphenix(c->built_n, c->perm, sx->u, sx->alpha_v, P, sx->alpha_c, c->sx4, c->st) !=
          cudaSuccess)
    return SPH_E_CUDA;
  if (sx && sx->limit && sphh::launch_gather_bins(c->built_n, c->perm, sx->bins_in, c->sx4, c->st) != cudaSuccess)
    return SPH_E_CUDA;
  t_end(c, SPH_T_GATHER);
  if (c->p.flags & SPH_FLAG_COUNT_PAIRS && !(sx && sx->gradient))
    if (cudaMemsetAsync(c->pairs + 1, 0, sizeof(unsigned long long), c->st) != cudaSuccess)
      return SPH_E_CUDA;
  if (c->built_tree) {
    // the tree force needs the lists and reverse pairs of this build's
    // density, taken over every target or under the same mask
    if (!c->lists_valid || (c->lists_mask != nullptr && c->lists_mask != active)) return SPH_E_INVAL;
    sphh::TreeForceArgs a = tree_force_args(c);
    a.ax = ax;
    a.ay = ay;
    a.az = az;
    a.du_dt = du_dt;
    a.v_sig = v_sig;
    if (active) {
      const int rc = ensure_act(c, c->built_n);
      if (rc != SPH_OK) return rc;
      if (sphh::launch_tree_mask(c->built_n, c->perm, active, c->act_s, nullptr, nullptr, c->st) != cudaSuccess)
        return SPH_E_CUDA;
      a.act = c->act_s;
    }
    t_begin(c, SPH_T_FORCE);
    cudaError_t e;
    if (sx && sx->limit) {
      // the time-step limiter over the same pairs (bins in tree order)
      a.fE = c->sx4;
      a.pairs = nullptr;
      a.bins_out = sx->bins_out;
      e = sphh::launch_tree_limit(a, phys_of(c->p), c->st);
    } else if (sx) {
      // SPHENIX on the nested grids: the same lists and reverse pairs, the
      // fifth record in tree order
      a.fE = c->sx4;
      if (sx->gradient) {
        a.pairs = nullptr;
        a.alpha_c_out = sx->alpha_c_out;
        a.lap_u = sx->lap_u;
        e = sphh::launch_tree_sphenix_gradient(a, phys_of(c->p), sx->x, c->st);
      } else {
        e = sphh::launch_tree_sphenix_force(a, phys_of(c->p), sx->x, c->st);
      }
    } else {
      e = sphh::launch_tree_force(a, phys_of(c->p), c->st);
    }
    t_end(c, SPH_T_FORCE);
    return cuda_code(e);
  }
  sphh::ForceArgs a;
  a.n_sims = c->built_sims;
  a.num_sms = c->num_sms;
  a.grid = c->grid;
  a.misc_ro = c->misc;
  a.misc = c->misc;
  a.overflow = c->overflow;
  a.pairs = c->pairs + 1;
  a.cell_start = c->cell_start;
  a.perm = c->perm;
  a.fA = c->pos4;
  a.fB = c->vel4;
  a.fC = c->th4;
  a.fD = c->fD;
  a.ax = ax;
  a.ay = ay;
  a.az = az;
  a.du_dt = du_dt;
  a.v_sig = v_sig;
  // the density's lists are dealt by the same rounds only under the same
  // mask; lists of later sources only (symmetric mode) serve the symmetric
  // force alone (the other forces then filter the cells themselves)
  const bool sym = sx == nullptr && sym_applies(c, active);
  a.lists = (c->lists_valid && c->lists_mask == active && c->lists_upper == sym) ? c->lists : nullptr;
  a.list_cnt = c->list_cnt;
  if (sym) {
    // the density published full lists (or none): with the later sources only
    // the symmetric force would need them too, so walk the cells instead
    if (!c->lists_upper) a.lists = nullptr;
    const int rc = ensure_sym(c, c->built_n);
    if (rc != SPH_OK) return rc;
    sphh::SymArgs y;
    y.rec_a = c->sym_a;
    y.rec_b = c->sym_b;
    y.recv = c->sym_recv;
    y.order = c->sym_order;
    y.cnt = c->sym_cnt;
    y.off = c->sym_off;
    y.cursor = c->sym_cursor;
    y.tile_sum = c->sym_tiles;
    y.counter = c->sym_counter;
    y.cap = c->cap_sym_rec;
    y.status = c->misc + sphk::kStatus;
    t_begin(c, SPH_T_FORCE);
    const cudaError_t e = sphh::launch_force_sym(a, y, phys_of(c->p), c->built_n, c->st);
    t_end(c, SPH_T_FORCE);
    return cuda_code(e);
  }
  if (active) {
    a.act = c->act_s;
    a.blk_any = c->blk_any;
  }
  t_begin(c, SPH_T_FORCE);
  cudaError_t e;
  if (sx && sx->limit) {
    a.fE = c->sx4;
    a.pairs = nullptr;
    a.bins_out = sx->bins_out;
    e = sphh::launch_limit_bins(a, phys_of(c->p), c->st);
  } else if (sx) {
    a.fE = c->sx4;
    if (sx->gradient) {
      a.pairs = nullptr;
      a.alpha_c_out = sx->alpha_c_out;
      a.lap_u = sx->lap_u;
      e = sphh::launch_sphenix_gradient(a, phys_of(c->p), sx->x, c->st);
    } else {
      e = sphh::launch_sphenix_force(a, phys_of(c->p), sx->x, c->st);
    }
  } else {
    e = sphh::launch_force(a, phys_of(c->p), c->st);
  }
  t_end(c, SPH_T_FORCE);
  return cuda_code(e);
}

}  // namespace

extern "C" {

void sph_default_params(sph_params* p) {
  if (!p) return;
  p->box_size = 1.0;
  p->gamma = 5.0 / 3.0;
  p->eta = 1.2348;
  p->alpha_v = 0.8;
  p->beta_v = 3.0;
  p->eps_balsara = 1e-4;
  p->h_tol = 1e-4;
  p->cfl = 0.1;
  p->cell_margin = 0.05;
  p->max_h_iter = 30;
  p->flags = 0;
  p->n_leaf = 16;
  p->kernel = SPH_KERNEL_CUBIC;
  p->lanes_per_target = 0;
}

int sph_create(sph_ctx** out, const sph_params* p, void* stream) {
  if (!out || !p) return SPH_E_INVAL;
  *out = nullptr;
  if (!params_ok(*p)) return SPH_E_INVAL;
  sph_ctx* c = new (std::nothrow) sph_ctx();
  if (!c) return SPH_E_NOMEM;
  c->p = *p;
  c->st = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return SPH_E_CUDA;
  }
  bool ok = dalloc(c->misc, sphk::kMiscWords) && dalloc(c->pairs, 4) && dalloc(c->off1, 2) &&
            dalloc(c->box1, 1);
  if (ok) ok = cudaMallocHost((void**)&c->h_off1, 2 * sizeof(int64_t)) == cudaSuccess &&
               cudaMallocHost((void**)&c->h_box1, sizeof(double)) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(c->misc, 0, sphk::kMiscWords * sizeof(int32_t), c->st) == cudaSuccess &&
               cudaMemsetAsync(c->pairs, 0, 4 * sizeof(unsigned long long), c->st) == cudaSuccess;
  if (!ok) {
    sph_destroy(c);
    return SPH_E_NOMEM;
  }
  c->h_off1[0] = 0;
  c->h_off1[1] = -1;
  c->h_box1[0] = -1.0;
  *out = c;
  return SPH_OK;
}

void sph_destroy(sph_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  for (int k = 0; k < SPH_T_COUNT; ++k) {
    for (cudaEvent_t e : c->ev_start[k]) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_stop[k]) cudaEventDestroy(e);
  }
  free_grown(c);
  free_tree(c);
  free_sym(c);
  dfree(c->sx4);
  dfree(c->dvp);
  dfree(c->act_s);
  dfree(c->act_pre);
  dfree(c->blk_any);
  dfree(c->blk_need);
  dfree(c->hact);
  dfree(c->hbin);
  dfree(c->hwake);
  dfree(c->hcellmin);
  dfree(c->htick);
  dfree(c->misc);
  dfree(c->pairs);
  dfree(c->off1);
  dfree(c->box1);
  if (c->h_off1) cudaFreeHost(c->h_off1);
  if (c->h_box1) cudaFreeHost(c->h_box1);
  cudaGetLastError();
  delete c;
}

const char* sph_error_string(int code) {
  switch (code) {
    case SPH_OK: return "ok";
    case SPH_E_INVAL: return "invalid argument";
    case SPH_E_NOMEM: return "device allocation failed";
    case SPH_E_H_NOCONV: return "smoothing length did not converge";
    case SPH_E_REBUILD: return "kernel support larger than the cell: rebuild the cells";
    case SPH_E_BOX: return "largest support exceeds half the box";
    case SPH_E_TIMEOUT: return "bounded device wait expired";
    case SPH_E_CUDA: return "CUDA runtime error";
    case SPH_E_CAPACITY: return "fixed-size library limit exceeded";
    default: return "unknown error";
  }
}

int sph_status(sph_ctx* c, int32_t* status_out) {
  if (!c || !status_out) return SPH_E_INVAL;
  return read_status(c, status_out);
}

int sph_build_cells(sph_ctx* c, int64_t n, const double* x, const double* y, const double* z,
                    const float* h, sph_cells* out) {
  if (!c || !out || n < 0 || n > INT32_MAX / 16) return SPH_E_INVAL;
  if (n > 0 && (!x || !y || !z || !h)) return SPH_E_INVAL;
  int rc = ensure(c, n, 1);
  if (rc != SPH_OK) return rc;
  if (c->h_off1[1] != n || c->h_box1[0] != c->p.box_size) {
    // the pinned mirrors may still feed an earlier copy: wait before rewriting
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
    c->h_off1[0] = 0;
    c->h_off1[1] = n;
    c->h_box1[0] = c->p.box_size;
    if (cudaMemcpyAsync(c->off1, c->h_off1, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->box1, c->h_box1, sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return SPH_E_CUDA;
  }
  rc = do_build(c, 1, n, c->off1, c->box1, x, y, z, h);
  if (rc != SPH_OK) return rc;
  out->n = n;
  out->n_c = -1;
  out->n_c_dev = &c->grid[0].n_c;
  out->cell_start = c->cell_start;
  out->perm = c->perm;
  rc = finish(c);
  if (rc == SPH_OK && (c->p.flags & SPH_FLAG_SYNC)) return sph_cells_sync(c, out);
  return rc;
}

int sph_reserve(sph_ctx* c, int64_t n_total, int32_t n_sims) {
  if (!c || n_total < 0 || n_total > INT32_MAX / 16 || n_sims < 1) return SPH_E_INVAL;
  int rc = ensure(c, n_total, n_sims);
  if (rc == SPH_OK && (c->p.flags & SPH_FLAG_TREE)) rc = ensure_tree(c, n_total, 0);
  if (rc == SPH_OK && (c->p.flags & SPH_FLAG_SYMMETRIC)) rc = ensure_sym(c, n_total);
  return rc;
}

int sph_cells_sync(sph_ctx* c, sph_cells* cells) {
  if (!c || !cells || !cells->n_c_dev) return SPH_E_INVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  int32_t nc = -1;
  if (cudaMemcpy(&nc, cells->n_c_dev, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SPH_E_CUDA;
  cells->n_c = nc;
  return SPH_OK;
}

int sph_cells_copy(sph_ctx* c, sph_cells* cells, int32_t* cell_start_dst, int32_t* perm_dst) {
  if (!c || !cells || !cell_start_dst || (!perm_dst && cells->n > 0)) return SPH_E_INVAL;
  int rc = sph_cells_sync(c, cells);
  if (rc != SPH_OK) return rc;
  const int64_t nc = cells->n_c;
  if (nc < 1) return SPH_E_INVAL;
  if (cudaMemcpy(cell_start_dst, cells->cell_start, (size_t)(nc * nc * nc + 1) * sizeof(int32_t),
                 cudaMemcpyDefault) != cudaSuccess)
    return SPH_E_CUDA;
  if (cells->n > 0 &&
      cudaMemcpy(perm_dst, cells->perm, (size_t)cells->n * sizeof(int32_t), cudaMemcpyDefault) !=
          cudaSuccess)
    return SPH_E_CUDA;
  return SPH_OK;
}

int sph_density(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const float* h_in,
                sph_density_out* out) {
  if (!c || !cells || !in || !out) return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !in->u || !h_in ||
      !out->h || !out->rho || !out->f || !out->div_v || !out->curl_v || !out->P || !out->c ||
      !out->balsara)
    return SPH_E_INVAL;
  int rc = do_density(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, in->u, h_in, out->h,
                      out->rho, out->f, out->div_v, out->curl_v, out->P, out->c, out->balsara,
                      out->n_iter);
  return rc != SPH_OK ? rc : finish(c);
}

int sph_force(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
              sph_force_out* out) {
  if (!c || !cells || !in || !d || !out) return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !d->h || !d->rho ||
      !d->f || !d->P || !d->c || !d->balsara || !out->ax || !out->ay || !out->az || !out->du_dt ||
      !out->v_sig)
    return SPH_E_INVAL;
  int rc = do_force(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, d->h, d->rho, d->f, d->P,
                    d->c, d->balsara, out->ax, out->ay, out->az, out->du_dt, out->v_sig);
  return rc != SPH_OK ? rc : finish(c);
}

// One KDK step; with X, the SPHENIX flavour with its parameters alpha_v and
// alpha_c (in/out, pool order).
int step_impl(sph_ctx* c, const sph_pool* pl, const sph_sphenix_params* X, float* alpha_v, float* alpha_c) {
  if (!c || !pl || pl->n_sims < 1 || pl->n_total < 0 || pl->n_total > INT32_MAX / 16) return SPH_E_INVAL;
  if (!pl->sim_offset || !pl->box_size || !pl->dt) return SPH_E_INVAL;
  if (pl->n_total > 0 &&
      (!pl->x || !pl->y || !pl->z || !pl->vx || !pl->vy || !pl->vz || !pl->u || !pl->m || !pl->h ||
       !pl->ax || !pl->ay || !pl->az || !pl->du_dt || !pl->v_sig || !pl->rho || !pl->f ||
       !pl->div_v || !pl->curl_v || !pl->P || !pl->c || !pl->balsara))
    return SPH_E_INVAL;
  if (X && pl->n_total > 0 && (!alpha_v || !alpha_c)) return SPH_E_INVAL;
  int rc = ensure(c, pl->n_total, pl->n_sims);
  if (rc != SPH_OK) return rc;
  if (X) {
    rc = ensure_sphenix(c, pl->n_total);
    if (rc != SPH_OK) return rc;
  }
  sphh::StepArgs s;
  s.gamma_k = sphk::kernel_gamma(c->p.kernel);
  s.n_sims = pl->n_sims;
  s.n_total = pl->n_total;
  s.num_sms = c->num_sms;
  s.sim_offset = pl->sim_offset;
  s.box = pl->box_size;
  s.cfl = c->p.cfl;
  s.x = pl->x;
  s.y = pl->y;
  s.z = pl->z;
  s.vx = pl->vx;
  s.vy = pl->vy;
  s.vz = pl->vz;
  s.u = pl->u;
  s.m = pl->m;
  s.h = pl->h;
  s.ax = pl->ax;
  s.ay = pl->ay;
  s.az = pl->az;
  s.du_dt = pl->du_dt;
  s.v_sig = pl->v_sig;
  s.vpx = c->vpx;
  s.vpy = c->vpy;
  s.vpz = c->vpz;
  s.up = c->up;
  s.dt = pl->dt;
  s.dt_bits = c->dt_bits;
  s.dt_f = c->dt_f;
  s.status = c->misc + sphk::kStatus;
  s.h_guess = pl->h;
  s.div_v = pl->div_v;
  t_begin(c, SPH_T_INTEGRATE);
  if (sphh::launch_dt(s, c->st) != cudaSuccess) return SPH_E_CUDA;
  if (sphh::launch_kick_drift(s, c->st) != cudaSuccess) return SPH_E_CUDA;
  t_end(c, SPH_T_INTEGRATE);
  // SPHENIX: the divergence of the previous evaluation, before the density
  // loop replaces it
  if (X && pl->n_total > 0 &&
      cudaMemcpyAsync(c->dvp, pl->div_v, sizeof(float) * (size_t)pl->n_total, cudaMemcpyDeviceToDevice, c->st) !=
          cudaSuccess)
    return SPH_E_CUDA;
  const bool sync = (c->p.flags & SPH_FLAG_SYNC) != 0;
  for (int attempt = 0;; ++attempt) {
    rc = do_build(c, pl->n_sims, pl->n_total, pl->sim_offset, pl->box_size, pl->x, pl->y, pl->z, pl->h);
    if (rc != SPH_OK) return rc;
    rc = do_density(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, c->up, pl->h, pl->h,
                    pl->rho, pl->f, pl->div_v, pl->curl_v, pl->P, pl->c, pl->balsara, pl->n_iter);
    if (rc != SPH_OK) return rc;
    if (!sync) break;
    int32_t st = 0;
    rc = read_status(c, &st);
    if (rc != SPH_OK) return rc;
    if (c->built_tree && (st & SPH_ST_CAPACITY) && attempt < 8) {
      // more reverse pairs than room: grow to the emitted count and repeat
      unsigned long long emitted = 0;
      if (cudaMemcpy(&emitted, c->rev_count, sizeof(emitted), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SPH_E_CUDA;
      rc = ensure_tree(c, pl->n_total, (int64_t)(emitted + emitted / 4 + 65536));
      if (rc != SPH_OK) return rc;
      continue;
    }
    if (!(st & SPH_ST_REBUILD) || attempt >= 8) {
      const int code = code_of_status(st);
      if (code != SPH_OK) return code;
      break;
    }
    // h now holds the capped values; the next build sizes the cells from
    // them with the margin, which makes every cell larger.
  }
  // same build and positions as the density just run: its gather already
  // wrote the cell-relative positions into the buffer the force reads
  if (X) {
    const sphk::SphenixDev xd = sphenix_dev(*X, 0.0, pl->dt);
    sphh::SphenixAlphaArgs aa{pl->n_total, pl->n_sims, pl->sim_offset, pl->h, pl->c, pl->div_v, pl->v_sig,
                              c->dvp, alpha_v, (float)sphk::kernel_gamma(c->p.kernel)};
    t_begin(c, SPH_T_INTEGRATE);
    if (sphh::launch_sphenix_alpha_v(aa, xd, c->st) != cudaSuccess) return SPH_E_CUDA;
    t_end(c, SPH_T_INTEGRATE);
    LoopPass g;
    g.gradient = true;
    g.u = c->up;
    g.alpha_v = alpha_v;
    g.alpha_c = alpha_c;
    g.alpha_c_out = alpha_c;
    g.x = xd;
    rc = do_force(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, pl->h, pl->rho, pl->f, pl->P, pl->c,
                  pl->balsara, pl->ax, pl->ay, pl->az, pl->du_dt, pl->v_sig, true, &g);
    if (rc != SPH_OK) return rc;
    LoopPass f = g;
    f.gradient = false;
    f.skip_gather = true;
    rc = do_force(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, pl->h, pl->rho, pl->f, pl->P, pl->c,
                  pl->balsara, pl->ax, pl->ay, pl->az, pl->du_dt, pl->v_sig, true, &f);
  } else {
    rc = do_force(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, pl->h, pl->rho, pl->f, pl->P,
                  pl->c, pl->balsara, pl->ax, pl->ay, pl->az, pl->du_dt, pl->v_sig, true);
  }
  if (rc != SPH_OK) return rc;
  t_begin(c, SPH_T_INTEGRATE);
  if (sphh::launch_kick(s, c->st) != cudaSuccess) return SPH_E_CUDA;
  t_end(c, SPH_T_INTEGRATE);
  return finish(c);
}

int sph_step(sph_ctx* c, const sph_pool* pl) { return step_impl(c, pl, nullptr, nullptr, nullptr); }

int sph_time_bins(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
                  const float* v_sig, double cfl, double dt_max, int32_t max_bin, int32_t* bins) {
  if (!c || !cells || !in || !d || !v_sig || !bins) return SPH_E_INVAL;
  if (!(cfl > 0.0) || !std::isfinite(cfl) || !(dt_max > 0.0) || !std::isfinite(dt_max) || max_bin < 0 ||
      max_bin > 62)
    return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !d->h || !d->rho || !d->f ||
      !d->P || !d->c || !d->balsara)
    return SPH_E_INVAL;
  int rc = ensure_sphenix(c, in->n);
  if (rc != SPH_OK) return rc;
  const float cf = (float)(cfl * sphk::kernel_gamma(c->p.kernel));
  if (sphh::launch_time_bins(in->n, d->h, v_sig, cf, (float)dt_max, max_bin, bins, c->st) != cudaSuccess)
    return SPH_E_CUDA;
  LoopPass L;
  L.limit = true;
  L.bins_in = bins;
  L.bins_out = bins;
  rc = do_force(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, d->h, d->rho, d->f, d->P, d->c,
                d->balsara, nullptr, nullptr, nullptr, nullptr, nullptr, false, &L);
  return rc != SPH_OK ? rc : finish(c);
}

}  // extern "C"

namespace {

// One sub-step (the two entry points below): with tick_dev the current tick is
// read from and the next written to device memory, and nothing waits for the
// stream (a CUDA graph can capture the call); else t_now comes from the host
// and the next tick is read back into *t_next_out.
int hier_substep(sph_ctx* c, const sph_pool* pl, int32_t* bins, int64_t* tbeg, double dt_max, int32_t max_bin,
                 int64_t t_now, int64_t* tick_dev, int32_t options, uint8_t* sync_flags, int64_t* t_next_out) {
  if (!c || !pl || !bins || !tbeg || (!t_next_out && !tick_dev) || pl->n_sims != 1 || pl->n_total < 1 ||
      pl->n_total > INT32_MAX / 16 || !(dt_max > 0.0) || !std::isfinite(dt_max) || max_bin < 0 || max_bin > 40 ||
      t_now < 0 || (options & ~(SPH_HIER_ADAPT | SPH_HIER_WAKEUP | SPH_HIER_PREDICT | SPH_HIER_KEEP_CELLS)) != 0)
    return SPH_E_INVAL;
  // the device-tick form waits for nothing: no kept cells (a host decision),
  // no synchronous context, no kernel timing
  if (tick_dev && ((options & SPH_HIER_KEEP_CELLS) || (c->p.flags & (SPH_FLAG_SYNC | SPH_FLAG_TIMING))))
    return SPH_E_INVAL;
  const bool adapt = (options & SPH_HIER_ADAPT) != 0, wakeup = (options & SPH_HIER_WAKEUP) != 0;
  if (!pl->sim_offset || !pl->box_size || !pl->x || !pl->y || !pl->z || !pl->vx || !pl->vy || !pl->vz ||
      !pl->u || !pl->m || !pl->h || !pl->ax || !pl->ay || !pl->az || !pl->du_dt || !pl->v_sig || !pl->rho ||
      !pl->f || !pl->div_v || !pl->curl_v || !pl->P || !pl->c || !pl->balsara)
    return SPH_E_INVAL;
  // kept cells are uniform-grid cells
  const bool tree = (c->p.flags & SPH_FLAG_TREE) != 0;
  if (tree && (options & SPH_HIER_KEEP_CELLS)) return SPH_E_INVAL;
  const int64_t n = pl->n_total;
  int rc = ensure(c, n, 1);
  if (rc == SPH_OK) rc = ensure_hier(c, n);
  if (rc == SPH_OK && (adapt || (tree && wakeup))) rc = ensure_sphenix(c, n);
  if (rc != SPH_OK) return rc;
  sphh::HierArgs h;
  h.n = n;
  h.max_bin = max_bin;
  h.t_now = t_now;
  h.t_now_dev = tick_dev;
  h.tau = std::ldexp(dt_max, -max_bin);
  h.box = pl->box_size;
  h.x = pl->x;
  h.y = pl->y;
  h.z = pl->z;
  h.vx = pl->vx;
  h.vy = pl->vy;
  h.vz = pl->vz;
  h.u = pl->u;
  h.ax = pl->ax;
  h.ay = pl->ay;
  h.az = pl->az;
  h.du_dt = pl->du_dt;
  h.vpx = c->vpx;
  h.vpy = c->vpy;
  h.vpz = c->vpz;
  h.up = c->up;
  h.bin = bins;
  h.t_begin = tbeg;
  h.bin_new = nullptr;
  h.act = c->hact;
  h.sync = sync_flags;
  h.wake = nullptr;
  h.predict = (options & SPH_HIER_PREDICT) != 0;
  h.gamma = (float)c->p.gamma;
  h.h = pl->h;
  h.rho = pl->rho;
  h.P = pl->P;
  h.c = pl->c;
  h.div_v = pl->div_v;
  const bool keep = (options & SPH_HIER_KEEP_CELLS) != 0;
  h.vmax2_bits = keep ? reinterpret_cast<unsigned*>(c->misc + sphk::kHierVmax) : nullptr;
  h.hmax_bits = keep ? reinterpret_cast<unsigned*>(c->misc + sphk::kHierHmax) : nullptr;
  h.t_next = c->htick;
  h.status = c->misc + sphk::kStatus;
  t_begin(c, SPH_T_INTEGRATE);
  if (keep && cudaMemsetAsync(c->misc + sphk::kHierVmax, 0, 2 * sizeof(int32_t), c->st) != cudaSuccess)
    return SPH_E_CUDA;
  if (sphh::launch_hier_next(h, c->st) != cudaSuccess || sphh::launch_hier_drift(h, c->st) != cudaSuccess)
    return SPH_E_CUDA;
  t_end(c, SPH_T_INTEGRATE);
  // SPH_HIER_KEEP_CELLS: the cells of the last build still hold every pair
  // within the supports while the largest support plus twice the drift bound
  // since that build (the largest |v| times dt, summed over the sub-steps)
  // fits a cell; the loops then cap the supports at that reach
  bool kept = false;
  double drift = 0.0;
  if (keep) {
    unsigned long long tn = 0;
    uint32_t bits[2] = {0u, 0u};
    if (cudaMemcpyAsync(&tn, c->htick, sizeof(tn), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaMemcpyAsync(bits, c->misc + sphk::kHierVmax, sizeof(bits), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
      return SPH_E_CUDA;
    float v2 = 0.0f, hm = 0.0f;
    memcpy(&v2, &bits[0], sizeof(float));
    memcpy(&hm, &bits[1], sizeof(float));
    drift = c->hier_drift + std::sqrt((double)v2) * (double)(tn - (unsigned long long)t_now) * h.tau;
    const double Hmax = sphk::kernel_gamma(c->p.kernel) * (double)hm;
    // room for the active supports to grow in this sub-step's solve (2 %):
    // a support that reaches the reach anyway costs a rebuild and a second
    // density
    kept = c->hier_epoch == c->build_epoch && c->hier_n == n && c->hier_cell > 0.0 && std::isfinite(drift) &&
           Hmax * 1.02 + 2.0 * drift * (1.0 + 1e-6) < c->hier_cell * (1.0 - 1e-5);
  }
  const bool sync = (c->p.flags & SPH_FLAG_SYNC) != 0;
  for (int attempt = 0;; ++attempt) {
    if (kept) {
      // the supports' cap: the cell less twice the drift (rounded down)
      const float reach = (float)((c->hier_cell - 2.0 * drift * (1.0 + 1e-6)) * (1.0 - 1e-6));
      if (cudaMemcpyAsync(reinterpret_cast<char*>(c->grid) + offsetof(GridDev, reach_f), &reach, sizeof(float),
                          cudaMemcpyHostToDevice, c->st) != cudaSuccess)
        return SPH_E_CUDA;
      c->hier_drift = drift;
    } else {
      rc = do_build(c, 1, n, pl->sim_offset, pl->box_size, pl->x, pl->y, pl->z, pl->h);
      if (rc != SPH_OK) return rc;
      if (keep) {
        double cell = 0.0;
        if (cudaMemcpyAsync(&cell, reinterpret_cast<char*>(c->grid) + offsetof(GridDev, cell), sizeof(double),
                            cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
            cudaStreamSynchronize(c->st) != cudaSuccess)
          return SPH_E_CUDA;
        c->hier_epoch = c->build_epoch;
        c->hier_n = n;
        c->hier_cell = cell;
        c->hier_drift = 0.0;
      }
    }
    rc = do_density(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, c->up, pl->h, pl->h, pl->rho, pl->f,
                    pl->div_v, pl->curl_v, pl->P, pl->c, pl->balsara, pl->n_iter, c->hact);
    if (rc != SPH_OK) return rc;
    if (!sync && !kept) break;
    int32_t st = 0;
    rc = read_status(c, &st);
    if (rc != SPH_OK) return rc;
    if (kept && (st & SPH_ST_REBUILD)) {
      // a support reached the kept cells' reach: build afresh and repeat
      kept = false;
      continue;
    }
    if (!(st & SPH_ST_REBUILD) || attempt >= 8) {
      const int code = code_of_status(st);
      if (code != SPH_OK) return code;
      break;
    }
  }
  rc = do_force(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, pl->h, pl->rho, pl->f, pl->P, pl->c,
                pl->balsara, pl->ax, pl->ay, pl->az, pl->du_dt, pl->v_sig, true, nullptr, c->hact);
  if (rc != SPH_OK) return rc;
  if (adapt) {
    // proposed bins of the active particles: CFL bins, then the limiter over
    // the force pairs (the masked pass reuses the density's lists) against
    // the active neighbours' proposals and the bins the inactive ones hold
    const float cf = (float)(c->p.cfl * sphk::kernel_gamma(c->p.kernel));
    if (sphh::launch_time_bins(n, pl->h, pl->v_sig, cf, (float)dt_max, max_bin, c->hbin, c->st) != cudaSuccess ||
        sphh::launch_hier_held_bins(h, c->hbin, c->st) != cudaSuccess)
      return SPH_E_CUDA;
    LoopPass L;
    L.limit = true;
    L.skip_gather = true;
    L.bins_in = c->hbin;
    L.bins_out = c->hbin;
    rc = do_force(c, pl->x, pl->y, pl->z, c->vpx, c->vpy, c->vpz, pl->m, pl->h, pl->rho, pl->f, pl->P, pl->c,
                  pl->balsara, nullptr, nullptr, nullptr, nullptr, nullptr, true, &L, c->hact);
    if (rc != SPH_OK) return rc;
    h.bin_new = c->hbin;
  }
  t_begin(c, SPH_T_INTEGRATE);
  if (sphh::launch_hier_kick(h, c->st) != cudaSuccess) return SPH_E_CUDA;
  if (wakeup && tree) {
    // the wake-up pass over the nested grids' force pairs of this sub-step
    // (every pair within either support), with the bins after the kick
    sphh::TreeForceArgs a = tree_force_args(c);
    a.pairs = nullptr;
    a.fE = c->sx4;
    a.act = c->act_s;
    a.wake = c->hwake;
    if (cudaMemsetAsync(c->hwake, 0xff, (size_t)n * sizeof(int32_t), c->st) != cudaSuccess ||
        sphh::launch_gather_bins(n, c->perm, bins, c->sx4, c->st) != cudaSuccess ||
        sphh::launch_tree_mask(n, c->perm, c->hact, c->act_s, nullptr, nullptr, c->st) != cudaSuccess ||
        sphh::launch_tree_wake(a, phys_of(c->p), c->st) != cudaSuccess)
      return SPH_E_CUDA;
    h.wake = c->hwake;
  } else if (wakeup) {
    // the wake-up pass over the cells of this sub-step's build (the density
    // made them wide enough for every new H)
    sphh::WakeArgs w;
    w.n = n;
    w.grid = c->grid;
    w.cell_start = c->cell_start;
    w.perm = c->perm;
    w.key = c->key;
    w.x = pl->x;
    w.y = pl->y;
    w.z = pl->z;
    w.h = pl->h;
    w.gamma = sphk::kernel_gamma(c->p.kernel);
    w.act = c->hact;
    w.bin = bins;
    w.wake = c->hwake;
    w.act_s = c->act_s;
    w.pos4 = c->pos4;
    w.cellmin = c->hcellmin;
    w.total_cells = c->misc + sphk::kTotalCells;
    if (sphh::launch_hier_wake(w, c->st) != cudaSuccess) return SPH_E_CUDA;
    h.wake = c->hwake;
  }
  if ((wakeup || sync_flags != nullptr) && sphh::launch_hier_interrupt(h, c->st) != cudaSuccess) return SPH_E_CUDA;
  t_end(c, SPH_T_INTEGRATE);
  if (tick_dev) {
    // the next tick replaces the current one on the device
    if (cudaMemcpyAsync(tick_dev, c->htick, sizeof(int64_t), cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      return SPH_E_CUDA;
    return SPH_OK;
  }
  unsigned long long tn = 0;
  if (cudaMemcpyAsync(&tn, c->htick, sizeof(tn), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return SPH_E_CUDA;
  *t_next_out = (int64_t)tn;
  return finish(c);
}

}  // namespace

extern "C" {

int sph_hier_substep(sph_ctx* c, const sph_pool* pl, int32_t* bins, int64_t* tbeg, double dt_max,
                     int32_t max_bin, int64_t t_now, int32_t options, uint8_t* sync_flags, int64_t* t_next_out) {
  if (!t_next_out) return SPH_E_INVAL;
  return hier_substep(c, pl, bins, tbeg, dt_max, max_bin, t_now, nullptr, options, sync_flags, t_next_out);
}

int sph_hier_substep_dev(sph_ctx* c, const sph_pool* pl, int32_t* bins, int64_t* tbeg, double dt_max,
                         int32_t max_bin, int64_t* tick, int32_t options, uint8_t* sync_flags) {
  if (!tick) return SPH_E_INVAL;
  return hier_substep(c, pl, bins, tbeg, dt_max, max_bin, 0, tick, options, sync_flags, nullptr);
}

int sph_density_active(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const float* h_in,
                       const uint8_t* active, sph_density_out* out) {
  if (!c || !cells || !in || !out || !active) return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !in->u || !h_in ||
      !out->h || !out->rho || !out->f || !out->div_v || !out->curl_v || !out->P || !out->c ||
      !out->balsara)
    return SPH_E_INVAL;
  int rc = do_density(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, in->u, h_in, out->h, out->rho,
                      out->f, out->div_v, out->curl_v, out->P, out->c, out->balsara, out->n_iter, active);
  return rc != SPH_OK ? rc : finish(c);
}

int sph_force_active(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
                     const uint8_t* active, sph_force_out* out) {
  if (!c || !cells || !in || !d || !out || !active) return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !d->h || !d->rho ||
      !d->f || !d->P || !d->c || !d->balsara || !out->ax || !out->ay || !out->az || !out->du_dt ||
      !out->v_sig)
    return SPH_E_INVAL;
  int rc = do_force(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, d->h, d->rho, d->f, d->P, d->c,
                    d->balsara, out->ax, out->ay, out->az, out->du_dt, out->v_sig, false, nullptr, active);
  return rc != SPH_OK ? rc : finish(c);
}

void sph_sphenix_default_params(sph_sphenix_params* x) {
  if (!x) return;
  x->alpha_v_max = 2.0;
  x->ell = 0.05;
  x->beta_c = 1.0;
  x->alpha_c_min = 0.0;
  x->alpha_c_max = 1.0;
}

int sph_sphenix_gradient(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
                         const sph_sphenix_params* X, double dt, sph_sphenix_state* st) {
  if (!c || !cells || !in || !d || !X || !st || !sphenix_params_ok(*X) || !(dt >= 0.0) || !std::isfinite(dt))
    return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !in->u || !d->h || !d->rho ||
      !d->f || !d->div_v || !d->P || !d->c || !d->balsara || !st->alpha_v || !st->alpha_c || !st->div_v_prev ||
      !st->v_sig)
    return SPH_E_INVAL;
  int rc = ensure_sphenix(c, in->n);
  if (rc != SPH_OK) return rc;
  const sphk::SphenixDev xd = sphenix_dev(*X, dt, nullptr);
  sphh::SphenixAlphaArgs aa{in->n,      1,          nullptr,         d->h,
                            d->c,       d->div_v,   st->v_sig,       st->div_v_prev,
                            st->alpha_v, (float)sphk::kernel_gamma(c->p.kernel)};
  if (sphh::launch_sphenix_alpha_v(aa, xd, c->st) != cudaSuccess) return SPH_E_CUDA;
  LoopPass g;
  g.gradient = true;
  g.u = in->u;
  g.alpha_v = st->alpha_v;
  g.alpha_c = st->alpha_c;
  g.alpha_c_out = st->alpha_c;
  g.lap_u = st->lap_u;
  g.x = xd;
  rc = do_force(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, d->h, d->rho, d->f, d->P, d->c,
                d->balsara, nullptr, nullptr, nullptr, nullptr, nullptr, false, &g);
  return rc != SPH_OK ? rc : finish(c);
}

int sph_force_sphenix(sph_ctx* c, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
                      const float* alpha_v, const float* alpha_c, sph_force_out* out) {
  if (!c || !cells || !in || !d || !out) return SPH_E_INVAL;
  if (in->n != cells->n || cells->n != c->built_n || c->built_sims != 1) return SPH_E_INVAL;
  if (in->n == 0) return SPH_OK;
  if (!in->x || !in->y || !in->z || !in->vx || !in->vy || !in->vz || !in->m || !in->u || !d->h || !d->rho ||
      !d->f || !d->P || !d->c || !d->balsara || !alpha_v || !alpha_c || !out->ax || !out->ay || !out->az ||
      !out->du_dt || !out->v_sig)
    return SPH_E_INVAL;
  int rc = ensure_sphenix(c, in->n);
  if (rc != SPH_OK) return rc;
  LoopPass f;
  f.u = in->u;
  f.alpha_v = alpha_v;
  f.alpha_c = alpha_c;
  rc = do_force(c, in->x, in->y, in->z, in->vx, in->vy, in->vz, in->m, d->h, d->rho, d->f, d->P, d->c,
                d->balsara, out->ax, out->ay, out->az, out->du_dt, out->v_sig, false, &f);
  return rc != SPH_OK ? rc : finish(c);
}

int sph_step_sphenix(sph_ctx* c, const sph_pool* pool, const sph_sphenix_params* X, float* alpha_v,
                     float* alpha_c) {
  if (!X || !sphenix_params_ok(*X)) return SPH_E_INVAL;
  return step_impl(c, pool, X, alpha_v, alpha_c);
}

int sph_conservation(sph_ctx* c, const sph_pool* pl, double* out) {
  if (!c || !pl || !out || pl->n_sims < 1 || !pl->sim_offset) return SPH_E_INVAL;
  if (pl->n_total > 0 && (!pl->m || !pl->vx || !pl->vy || !pl->vz || !pl->ax || !pl->ay || !pl->az ||
                          !pl->du_dt))
    return SPH_E_INVAL;
  if (sphh::launch_conservation(pl->n_sims, pl->sim_offset, pl->m, pl->vx, pl->vy, pl->vz, pl->ax,
                                pl->ay, pl->az, pl->du_dt, out, c->st) != cudaSuccess)
    return SPH_E_CUDA;
  return finish(c);
}

// Friends-of-friends grids allow 160 cells per particle (8 for the SPH
// loops): at the usual linking length of 0.2 mean spacings, cells of b itself
// need 125 per particle, and cells capped wider multiply the pairs to test by
// the cube of the widening (2.5^3 = 16 at the SPH cap).  Their counts and
// offsets take 1.3 KB per particle.
constexpr int kFofCellsPerParticle = 160;

int sph_fof(sph_ctx* c, int64_t n, const double* x, const double* y, const double* z, double link_len,
            int32_t* group) {
  if (!c || n < 0 || n > INT32_MAX / 16 || !(link_len > 0.0)) return SPH_E_INVAL;
  if (n > 0 && (!x || !y || !z || !group)) return SPH_E_INVAL;
  if (link_len > c->p.box_size / 3.0) return SPH_E_BOX;
  if (n == 0) return SPH_OK;
  int rc = ensure(c, n, 1, kFofCellsPerParticle);
  if (rc != SPH_OK) return rc;
  if (c->h_off1[1] != n || c->h_box1[0] != c->p.box_size) {
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
    c->h_off1[0] = 0;
    c->h_off1[1] = n;
    c->h_box1[0] = c->p.box_size;
    if (cudaMemcpyAsync(c->off1, c->h_off1, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(c->box1, c->h_box1, sizeof(double), cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return SPH_E_CUDA;
  }
  // cells at least b wide: friends lie in the same or adjacent cells
  rc = do_build(c, 1, n, c->off1, c->box1, x, y, z, nullptr, link_len, kFofCellsPerParticle);
  if (rc != SPH_OK) return rc;
  sphh::FofArgs f;
  f.n_total = n;
  f.grid = c->grid;
  f.perm = c->perm;
  f.key = c->key;
  f.cell_start = c->cell_start;
  f.x = x;
  f.y = y;
  f.z = z;
  f.link = link_len;
  f.rel = c->pos4;  // the sorted density copies' buffer, free between loops
  f.group = group;
  f.status = c->misc + sphk::kStatus;
  c->lists_valid = false;
  t_begin(c, SPH_T_DENSITY);
  const cudaError_t e = sphh::launch_fof(f, c->st);
  t_end(c, SPH_T_DENSITY);
  if (e != cudaSuccess) return SPH_E_CUDA;
  return finish(c);
}

int sph_kernel_times(sph_ctx* c, double* ms_out, int64_t* calls_out) {
  if (!c || !ms_out) return SPH_E_INVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  for (int k = 0; k < SPH_T_COUNT; ++k) {
    t_collect(c, k);
    ms_out[k] = c->t_ms[k];
    if (calls_out) calls_out[k] = c->t_calls[k];
    c->t_ms[k] = 0.0;
    c->t_calls[k] = 0;
  }
  return SPH_OK;
}

int sph_tree_counts(sph_ctx* c, int64_t* out) {
  if (!c || !out) return SPH_E_INVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  for (int k = 0; k < 4; ++k) out[k] = 0;
  if (!c->built_tree) return SPH_OK;
  int32_t groups = 0, fb = 0;
  unsigned long long rev = 0, free_t = 0;
  if (cudaMemcpy(&groups, c->n_leaves, sizeof(groups), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&fb, c->misc + sphk::kTreeFbCount, sizeof(fb), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&rev, c->rev_count, sizeof(rev), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&free_t, c->pairs + 2, sizeof(free_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SPH_E_CUDA;
  out[0] = groups;
  out[1] = (int64_t)free_t;
  out[2] = (int64_t)rev;
  out[3] = fb;
  return SPH_OK;
}

int sph_pair_counts(sph_ctx* c, int64_t* out) {
  if (!c || !out) return SPH_E_INVAL;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return SPH_E_CUDA;
  unsigned long long v[2];
  if (cudaMemcpy(v, c->pairs, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return SPH_E_CUDA;
  out[0] = (int64_t)v[0];
  out[1] = (int64_t)v[1];
  return SPH_OK;
}

}  // extern "C"
