// sph_launch.h -- host-side argument records and launchers of the kernels
// (implemented in cells.cu, radix.cu, density.cu, force.cu, tree.cu,
// tree_loops.cu, step.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sphk {
struct GridDev;
struct PhysDev;
struct TreeLeaf;
struct TreeRange;
}  // namespace sphk

namespace sphh {

struct BuildArgs {
  int n_sims;
  int64_t n_total;
  int64_t cap_cells;  // upper bound of total cells (sizes count / cell_start)
  int num_sms;
  double margin;
  const int64_t* sim_offset;
  const double* box;
  const double *x, *y, *z;
  const float* h;
  sphk::GridDev* grid;
  int32_t* misc;
  int32_t* hmax_bits;  // per simulation scratch
  int32_t *key, *slot, *count, *cell_start, *scan_sums, *perm;
  int32_t *rk, *rv, *hist;  // radix-sort scratch: n, n, radix_hist_words(n)
  int sort_cells = 1;       // 0: counts and cell_start only (the tree build orders)
  double radius = 0.0;      // > 0: cells at least this wide, h unused (friends-of-friends)
  int cells_per_particle = 8;  // n_c^3 <= cells_per_particle n + 216 per simulation
  double gamma_k = sphk::kGammaKd;  // H / h of the kernel
};
cudaError_t launch_build(const BuildArgs& a, cudaStream_t st);

// Friends-of-friends groups (fof.cu) on a uniform build whose cells are at
// least the linking length wide: group[p] = smallest index of p's group.
struct FofArgs {
  int64_t n_total;
  const sphk::GridDev* grid;     // one simulation
  const int32_t *perm, *key, *cell_start;
  const double *x, *y, *z;
  double link;                   // linking length b
  float4* rel;                   // n scratch: sorted cell-relative positions
  int32_t* group;                // n: union-find parents, then the labels
  int32_t* status;
};
cudaError_t launch_fof(const FofArgs& a, cudaStream_t st);

// Stable radix sort of keys (bits significant bits) with values 0..n-1
// (radix.cu); keys is clobbered, the sorted values land in vals_out.
int64_t radix_hist_words(int64_t n);
cudaError_t radix_sort_index(int64_t n, int bits, int32_t* keys, int32_t* keys_tmp, int32_t* vals_out,
                             int32_t* vals_tmp, int32_t* hist, cudaStream_t st);
cudaError_t radix_sort_index64(int64_t n, int bits, uint64_t* keys, uint64_t* keys_tmp,
                               int32_t* vals_out, int32_t* vals_tmp, int32_t* hist, cudaStream_t st);

struct GatherDensityArgs {
  int64_t n_total;
  int n_sims;
  const int32_t *perm, *key;
  const sphk::GridDev* grid;
  const double *x, *y, *z;
  const float *vx, *vy, *vz, *m, *u, *h;
  float4 *pos4, *vel4;
  float* hs;
  // masked loops (one simulation): only the particles of the blocks flagged
  // here are gathered (nullptr: every particle)
  const uint8_t* blk_need = nullptr;
};
cudaError_t launch_gather_density(const GatherDensityArgs& a, cudaStream_t st);

// Force-loop copies: fA = (x, y, z, H), fB = (vx, vy, vz, m),
// fC = (f P / rho^2, f, c, B), fD = (rho, 1/H); positions relative to the cell.
struct GatherForceArgs {
  int64_t n_total;
  int n_sims;
  const int32_t *perm, *key;
  const sphk::GridDev* grid;
  const double *x, *y, *z;
  const float *vx, *vy, *vz, *m, *h, *rho, *f, *P, *c, *B;
  float4 *fA, *fB, *fC;
  float2* fD;
  // 1: compute fA.xyz from x, y, z; 0: fA.xyz already holds them (or is not
  // read), write H only
  int positions = 1;
  // nested grids: 64-byte records (rel, H), (fine, rho), (v, m), (fP, f, c, B)
  // per source instead of fA..fD; rel and fine are the tree gather's copies
  const float4* rel = nullptr;
  const int4* fine = nullptr;
  float4* rec = nullptr;
  float gamma_k = sphk::kGammaK;  // H / h of the kernel
  const uint8_t* blk_need = nullptr;  // as for the density gather
};
cudaError_t launch_gather_force(const GatherForceArgs& a, cudaStream_t st);
// Blocks within one block of a block holding an active particle (the blocks
// whose staged cells the masked loops read), one simulation, periodic.
cudaError_t launch_dilate_blocks(const sphk::GridDev* grid, const int32_t* total_blocks, const uint8_t* blk_any,
                                 uint8_t* blk_need, int64_t blk_cap, cudaStream_t st);
// Sorted copy of an active mask (act_s[s] = active[perm[s]]) and the flags
// of the blocks holding an active particle (blk_any, blk_cap bytes cleared
// first; one simulation).
cudaError_t launch_gather_mask(int64_t n, const int32_t* perm, const int32_t* key, const sphk::GridDev* grid,
                               const uint8_t* active, uint8_t* act_s, uint8_t* blk_any, int64_t blk_cap,
                               cudaStream_t st);

// Per-cell orders along the 13 neighbour axes (axis.cu): order[q n + s]
// for sorted slot s (the density copies pos4 must be current).
struct AxisSortArgs {
  int64_t n_total;
  const int32_t *perm, *key, *cell_start;
  const float4* pos4;
  uint16_t* order;  // kAxes * n_total
};
cudaError_t launch_axis_sort(const AxisSortArgs& a, cudaStream_t st);

// Outputs of the loops are written in pool order through perm.
struct DensityArgs {
  int n_sims;
  int num_sms;
  const sphk::GridDev* grid;
  const int32_t* misc_ro;  // total cells / blocks, overflow count
  int32_t* misc;           // same words, written by the loop kernels
  int32_t* overflow;       // blocks queued for the overflow kernel
  int32_t* status;
  unsigned long long* pairs;
  const int32_t *cell_start, *perm;
  const float4 *pos4, *vel4;
  const float* hs;
  float *h, *rho, *f, *div_v, *curl_v, *P, *c, *B;
  int32_t* n_iter;
  // optional neighbour lists for the force loop of the same build: the
  // entries of (sorted target ti, lane s) in lists[(4 ti + s) * kListRegion ...]
  uint16_t* lists;
  uint16_t* list_cnt;  // per (4 ti + s); 0xffff = overflow (not stored)
  // optional per-cell axis orders (axis.cu): the filter walks each neighbour
  // cell along the axis towards it and stops at the search radius
  const uint16_t* axis_order;
  int64_t axis_stride;  // n_total of the orders (one axis after the other)
  // optional active mask (sorted order): only targets with act != 0 are
  // computed and written; every particle is a source.  blk_any flags the
  // blocks with an active target (the others are skipped at once)
  const uint8_t* act = nullptr;
  const uint8_t* blk_any = nullptr;
  // publish only the list entries later in sorted order than the target
  // (the symmetric force, sym.cu)
  int32_t upper = 0;
};
cudaError_t launch_density(const DensityArgs& a, const sphk::PhysDev& ph, cudaStream_t st);

struct ForceArgs {
  int n_sims;
  int num_sms;
  const sphk::GridDev* grid;
  const int32_t* misc_ro;
  int32_t* misc;
  int32_t* overflow;
  unsigned long long* pairs;
  const int32_t *cell_start, *perm;
  const float4 *fA, *fB, *fC;
  const float2* fD;
  float *ax, *ay, *az, *du_dt, *v_sig;
  const uint16_t* lists;  // the density loop's lists, or nullptr
  const uint16_t* list_cnt;
  // SPHENIX: sorted (u, alpha_V, P, alpha_c) per source; the gradient pass
  // writes alpha_c (input order) and, if given, lap u
  const float4* fE = nullptr;
  float* alpha_c_out = nullptr;
  float* lap_u = nullptr;
  // optional active mask (sorted order) and block flags, as for the density loop
  const uint8_t* act = nullptr;
  const uint8_t* blk_any = nullptr;
  // time-step limiter pass: bins_out[p] = max(own bin, largest neighbour bin - 2)
  // (the bins come sorted in fE.x)
  int32_t* bins_out = nullptr;
};
cudaError_t launch_force(const ForceArgs& a, const sphk::PhysDev& ph, cudaStream_t st);
cudaError_t launch_sphenix_force(const ForceArgs& a, const sphk::PhysDev& ph, const sphk::SphenixDev& x,
                                 cudaStream_t st);
cudaError_t launch_sphenix_gradient(const ForceArgs& a, const sphk::PhysDev& ph, const sphk::SphenixDev& x,
                                    cudaStream_t st);
cudaError_t launch_limit_bins(const ForceArgs& a, const sphk::PhysDev& ph, cudaStream_t st);

// The symmetric force (sym.cu): records of the partners' sides, grouped by
// receiver.  Sizes: rec_a, rec_b, recv, order: cap; cnt, cursor: n;
// off: n + 1; tile_sum: sym_tiles(n) + 1.
struct SymArgs {
  float4* rec_a;   // (a_x, a_y, a_z, du/dt) of the receiver
  int2* rec_b;     // (v_sig bits, source sorted index)
  int32_t* recv;   // receiver sorted index
  int32_t* order;  // records by receiver
  int32_t *cnt, *off, *cursor, *tile_sum;
  int32_t* counter;
  int64_t cap;
  int32_t* status;
};
int64_t sym_tiles(int64_t n);
cudaError_t launch_force_sym(const ForceArgs& a, const SymArgs& y, const sphk::PhysDev& ph, int64_t n,
                             cudaStream_t st);

// Sub-steps of the time-step hierarchy (hier.cu), one simulation of side box.
struct HierArgs {
  int64_t n;
  int max_bin;
  int64_t t_now;
  const int64_t* t_now_dev;  // when set, the current tick is read from here
  double tau;  // dt_max / 2^max_bin
  const double* box;  // the pool's box side (device)
  double *x, *y, *z;
  float *vx, *vy, *vz, *u;            // half-kicked for the current step
  const float *ax, *ay, *az, *du_dt;  // last force of each particle
  float *vpx, *vpy, *vpz, *up;        // predicted at t_next (scratch)
  int32_t* bin;
  int64_t* t_begin;
  const int32_t* bin_new;  // proposed bins (nullptr: keep)
  uint8_t* act;            // active mask (scratch, input order)
  uint8_t* sync;           // synchronisation flags (nullptr: none; cleared)
  const int32_t* wake;     // wake-up bins (nullptr: no wake-up pass)
  // largest |v|^2 of the drift and largest h after it (float bits, reset by
  // the caller; nullptr: not taken)
  unsigned *vmax2_bits, *hmax_bits;
  // prediction of h, rho, P and c in the drift (predict != 0)
  int predict;
  float gamma;  // adiabatic index
  float *h, *rho, *P, *c;
  const float* div_v;
  unsigned long long* t_next;
  int32_t* status;
};
// The wake-up pass's view of the cells of the last uniform build.
struct WakeArgs {
  int64_t n;
  const sphk::GridDev* grid;
  const int32_t *cell_start, *perm, *key;
  const double *x, *y, *z;
  const float* h;
  double gamma;  // H / h of the kernel
  const uint8_t* act;
  const int32_t* bin;
  int32_t* wake;  // written: -1, or the largest bin_i - 2 above bin_j
  // sorted copies of this sub-step's loops: the active mask, and the
  // cell-relative positions with H (the force gather's records)
  const uint8_t* act_s;
  const float4* pos4;
  int32_t* cellmin;            // scratch, one per cell
  const int32_t* total_cells;  // device count of the build's cells
};
cudaError_t launch_hier_next(const HierArgs& a, cudaStream_t st);
cudaError_t launch_hier_drift(const HierArgs& a, cudaStream_t st);
cudaError_t launch_hier_kick(const HierArgs& a, cudaStream_t st);
// prop[i] = bin[i] where act[i] == 0 and i is not flagged for synchronisation
// (the limiter's input for the particles that keep their step)
cudaError_t launch_hier_held_bins(const HierArgs& a, int32_t* prop, cudaStream_t st);
// The wake-up limiter's neighbour pass, and the early end of the steps of the
// woken and the synchronised particles.
cudaError_t launch_hier_wake(const WakeArgs& a, cudaStream_t st);
cudaError_t launch_hier_interrupt(const HierArgs& a, cudaStream_t st);

// Time bins (timebins.cu): the CFL bins of n particles (input order), and the
// sorted limiter records E[s].x = bin of perm[s].
cudaError_t launch_time_bins(int64_t n, const float* h, const float* v_sig, float c, float dt_max, int max_bin,
                             int32_t* bins, cudaStream_t st);
cudaError_t launch_gather_bins(int64_t n, const int32_t* perm, const int32_t* bins, float4* fE, cudaStream_t st);

// SPHENIX per-particle steps (sphenix.cu).  The viscosity update of every
// particle (input order): alpha_v in/out, div_v_prev in (the divergence of the
// previous evaluation) and out (set to div_v); sim_offset / n_sims map a
// particle to its simulation's dt when x.dt_dev is given.
struct SphenixAlphaArgs {
  int64_t n_total;
  int n_sims;
  const int64_t* sim_offset;
  const float *h, *c, *div_v, *v_sig;
  float *div_v_prev, *alpha_v;
  float gamma_k;  // H / h of the kernel
};
cudaError_t launch_sphenix_alpha_v(const SphenixAlphaArgs& a, const sphk::SphenixDev& x, cudaStream_t st);
// Sorted copies E[s] = (u, alpha_V, P, alpha_c) of particle perm[s].
cudaError_t launch_gather_sphenix(int64_t n_total, const int32_t* perm, const float* u, const float* alpha_v,
                                  const float* P, const float* alpha_c, float4* fE, cudaStream_t st);

// Nested-grid build (tree.cu), after launch_build produced the top cells
// (counts and cell_start; no cell sort).
struct TreeBuildArgs {
  int n_sims;
  int64_t n_total;
  int64_t cap_cells;
  int n_leaf;
  double margin;
  const int64_t* sim_offset;
  const sphk::GridDev* grid;
  const double *x, *y, *z;
  const float* h;
  const int32_t* cell_key;    // top cell of each particle (launch_build's key)
  const int32_t* cell_start;  // top cells' ranges (valid in source order too)
  uint64_t *key64, *key64_b, *key64_c;  // n each (scratch)
  uint64_t* skey;             // n: source keys in source order
  int32_t* perm;              // n: source order -> pool index
  int32_t* tgt;               // n: target order -> source index
  int32_t *rv, *hist;         // radix scratch
  int32_t *flag, *leaf_of;    // n each
  int32_t* scan_tmp;          // n / 1024 + 2
  sphk::TreeLeaf* leaves;     // n + 1: target groups, start in target order
  int32_t* n_leaves;          // 1 (device)
  sphk::TreeRange* ranges;    // 27 n: source-order ranges of each group
  int8_t* level;              // n (source order): level of each particle
  float* leaf_side;           // n (source order): cell side of each particle's level
  float gamma_k = sphk::kGammaK;  // H / h of the kernel
};
cudaError_t launch_tree_build(const TreeBuildArgs& a, cudaStream_t st);

// Tree-order copies for the tree loops: fine integer position, offset from
// the fine sub-cell corner with the mass, (v, u), starting h, list radius.
struct TreeGatherArgs {
  int64_t n_total;
  int n_sims;
  const int32_t* perm;
  const uint64_t* skey;
  const sphk::GridDev* grid;
  const double *x, *y, *z;
  const float *m, *vx, *vy, *vz, *u, *h;
  const float* leaf_side;
  float list_reach;  // list radius / starting support
  int4* fine;
  float4 *rel, *vel4;
  float *hs, *lrad;
  float gamma_k = sphk::kGammaK;  // H / h of the kernel
};
cudaError_t launch_tree_gather(const TreeGatherArgs& a, cudaStream_t st);

// Density on the leaves (tree_loops.cu).  Lists hold packed (tree index,
// periodic shift) entries, kTreeListRegion per (4 ti + lane); list_cnt 0xffff
// marks a target whose sums were taken without a list.  Pairs that only the
// larger support reaches are emitted as reverse pairs and ordered by
// receiver into rev_start / rev.
struct TreeDensityArgs {
  int n_sims;
  int num_sms;
  int64_t n_total;
  const sphk::GridDev* grid;
  const int32_t* tgt;  // target order -> source index
  const sphk::TreeLeaf* leaves;
  const int32_t* n_leaves;
  const sphk::TreeRange* ranges;
  const int4* fine;
  const float4 *rel, *vel4;
  const float *hs, *lrad, *leaf_side;
  const int32_t* perm;
  int32_t* status;
  unsigned long long* pairs;
  float *h, *rho, *f, *div_v, *curl_v, *P, *c, *B;
  int32_t* n_iter;
  uint32_t* lists;
  uint16_t* list_cnt;
  uint64_t* rev_raw;   // rev_cap emitted pairs (receiver << 32 | packed source)
  unsigned long long* rev_count;  // 1: pairs emitted (may exceed rev_cap)
  int32_t* rev_start;  // n + 1: per-receiver counts, then their exclusive scan
  int32_t* rev_fill;   // n: scatter cursors
  uint32_t* rev;       // rev_cap: packed sources ordered by (receiver, source)
  int64_t rev_cap;
  int32_t* scan_tmp;   // (n + 1) / 1024 + 2
  int32_t* work;       // 1: group counter (reset by the launcher)
  // targets whose support outgrew their level, re-solved one level coarser
  const uint64_t* skey;        // n: source keys
  const int32_t* cell_start;   // top cells' ranges
  const int8_t* level;         // n: level of each particle
  int32_t *fb_list, *fb_count;  // n, 1
  int8_t* fb_level;            // n: level of the fallback solve
  int32_t* fb_work;            // 1
  unsigned long long* list_free;  // 1: targets summed without a list (counted with pairs)
  // masked loops: 1 per target in tree order (nullptr: every target), and
  // its exclusive prefix sums (n + 1; a group without a masked particle in
  // its 27 cells is skipped)
  const uint8_t* act = nullptr;
  const int32_t* act_pre = nullptr;
};
cudaError_t launch_tree_density(const TreeDensityArgs& a, const sphk::PhysDev& ph, cudaStream_t st);
// The mask in tree order: out[k] = active[perm[k]]; with pre (n + 1 int32,
// scan scratch tmp of (n + 1) / 1024 + 2) also its exclusive prefix sums.
cudaError_t launch_tree_mask(int64_t n, const int32_t* perm, const uint8_t* active, uint8_t* out, int32_t* pre,
                             int32_t* tmp, cudaStream_t st);

struct TreeForceArgs {
  int n_sims;
  int num_sms;
  const sphk::GridDev* grid;
  const int32_t* tgt;
  const sphk::TreeLeaf* leaves;
  const int32_t* n_leaves;
  const sphk::TreeRange* ranges;
  const int4* fine;
  const float4* rel;
  const float *lrad, *leaf_side;
  const int32_t* perm;
  const float4* rec;  // 4 float4 per source, as GatherForceArgs::rec
  const uint32_t* lists;
  const uint16_t* list_cnt;
  const int32_t* rev_start;
  const uint32_t* rev;
  unsigned long long* pairs;
  float *ax, *ay, *az, *du_dt, *v_sig;
  int32_t* work;  // 1: group counter (reset by the launcher)
  int64_t n_total;
  const uint64_t* skey;
  const int32_t* cell_start;
  const int32_t *fb_list, *fb_count;
  const int8_t* fb_level;
  int32_t* fb_work;
  // SPHENIX: (u, alpha_V, P, alpha_c) per source in tree order; the gradient
  // pass writes alpha_c (input order) and, if given, lap u
  const float4* fE = nullptr;
  float* alpha_c_out = nullptr;
  float* lap_u = nullptr;
  // masked loops: 1 per target in tree order (nullptr: every target)
  const uint8_t* act = nullptr;
  // the time-step limiter (fE.x = each source's bin): bins in input order
  int32_t* bins_out = nullptr;
  // the wake-up pass (fE.x = each source's bin): per input-order particle
  // outside the mask, the largest bin - 2 of a masked neighbour above its bin
  int32_t* wake = nullptr;
};
cudaError_t launch_tree_force(const TreeForceArgs& a, const sphk::PhysDev& ph, cudaStream_t st);
cudaError_t launch_tree_sphenix_force(const TreeForceArgs& a, const sphk::PhysDev& ph, const sphk::SphenixDev& x,
                                      cudaStream_t st);
cudaError_t launch_tree_sphenix_gradient(const TreeForceArgs& a, const sphk::PhysDev& ph,
                                         const sphk::SphenixDev& x, cudaStream_t st);
// The first time-step limiter over the nested grids' force pairs (a.fE,
// a.bins_out), and the wake-up pass (a.fE, a.act, a.wake).
cudaError_t launch_tree_limit(const TreeForceArgs& a, const sphk::PhysDev& ph, cudaStream_t st);
cudaError_t launch_tree_wake(const TreeForceArgs& a, const sphk::PhysDev& ph, cudaStream_t st);
// Exclusive scan of m int32 in place with a host-known length (radix.cu);
// tmp holds m / 1024 + 2 entries.
cudaError_t scan_exclusive_host_n(int32_t* a, int64_t m, int32_t* tmp, cudaStream_t st);

// Time integration over a pool (step.cu).
struct StepArgs {
  int n_sims;
  int64_t n_total;
  int num_sms;
  const int64_t* sim_offset;
  const double* box;
  double cfl;
  double gamma_k = sphk::kGammaKd;  // H / h of the kernel
  double *x, *y, *z;
  float *vx, *vy, *vz, *u;
  const float* m;
  const float* h;
  float *ax, *ay, *az, *du_dt, *v_sig;
  float *vpx, *vpy, *vpz, *up;  // predicted velocity / energy (scratch)
  double* dt;                   // per simulation
  unsigned* dt_bits;  // per simulation scratch (min of h / v_sig as FP32 bits)
  // per simulation: 0.5 dt and dt / 3 rounded to FP32, written by launch_dt
  // with dt (the kicks read them instead of each thread deriving them in
  // FP64, which this GPU runs at a small fraction of its FP32 rate)
  float* dt_f;
  int32_t* status;
  // starting guess of the next density loop: h_guess = h (1 + div_v dt / 3)
  // (nullptr: keep h)
  float* h_guess = nullptr;
  const float* div_v = nullptr;
};
cudaError_t launch_dt(const StepArgs& a, cudaStream_t st);  // uses a.dt_bits scratch
cudaError_t launch_kick_drift(const StepArgs& a, cudaStream_t st);
cudaError_t launch_kick(const StepArgs& a, cudaStream_t st);
cudaError_t launch_conservation(int n_sims, const int64_t* sim_offset, const float* m, const float* vx,
                                const float* vy, const float* vz, const float* ax, const float* ay,
                                const float* az, const float* du_dt, double* out, cudaStream_t st);

}  // namespace sphh
