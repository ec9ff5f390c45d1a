/*
 * sph.h -- C ABI of the GB300 (sm_103a) SPH neighbour-loop library.
 *
 * The library computes the hot path of the SPH solver of SWIFT (Schaller et
 * al., MNRAS 2024): particles are binned into a periodic cell grid whose cells
 * are at least the kernel support wide (Sec. 2.1, the Verlet-list grid); the
 * density loop solves every particle's smoothing length by Newton-Raphson
 * (Sec. 3.1.1, eqs. "numberdensity" and "partition") and accumulates the
 * density, its h-derivative and the velocity divergence and curl (Sec. 3.1.2);
 * the force loop then accumulates the pressure acceleration, the
 * Balsara-switched artificial viscosity and du/dt of the "Minimal"
 * density-energy flavour (Sec. 3.2, eqs. "densityenergy", "basicartvisc",
 * "alpha", "nuij", "balsara"); a kick-drift-kick step with one global
 * time-step (Sec. 2.4, operators of Sec. 5.4 with a = 1) ties them together.
 *
 * Conventions shared by every entry point
 *  - Pointers to particle data are DEVICE pointers owned by the caller; the
 *    library never frees them.  Arrays are structure-of-arrays, indexed by the
 *    caller's particle index ("input order").  Positions are double in
 *    [0, L); every other per-particle array is float.
 *  - Work is enqueued on the stream given to sph_create; calls return when the
 *    work is enqueued unless the context was created with SPH_FLAG_SYNC, in
 *    which case they wait for the stream and report device-side status.
 *  - Return values: SPH_OK (0) or a negative SPH_E_* code; no call throws,
 *    aborts or traps.  Device-side conditions (smoothing length not converged,
 *    a support larger than the cell, ...) are OR-ed into a status word that
 *    sph_status() returns and clears.
 *  - Kernel: the cubic spline by default, in the Dehnen & Aly (2012) form
 *    W(r,h) = w(r/H)/H^3, H = gamma_K h, gamma_K = 1.825742 (Sec. 3.1, eq.
 *    "kernel"); sph_params.kernel selects the quartic spline or the Wendland
 *    C2 kernel instead (SPH_KERNEL_*).
 *  - One context per stream; a context is not thread-safe.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
enum {
  SPH_OK = 0,
  SPH_E_INVAL = -1,     /* bad argument (NULL pointer, negative size, ...)   */
  SPH_E_NOMEM = -2,     /* device allocation of context scratch failed       */
  SPH_E_H_NOCONV = -3,  /* some smoothing length did not converge            */
  SPH_E_REBUILD = -4,   /* some support H exceeds its cell: rebuild needed   */
  SPH_E_BOX = -5,       /* the largest support exceeds half the box          */
  SPH_E_TIMEOUT = -6,   /* a bounded device wait expired                     */
  SPH_E_CUDA = -7,      /* a CUDA runtime call failed                        */
  SPH_E_CAPACITY = -8   /* a fixed-size limit of the library was exceeded    */
};

/* ---- device status bits (sph_status) ------------------------------------ */
enum {
  SPH_ST_H_NOCONV = 1,  /* Newton-Raphson hit max_h_iter                     */
  SPH_ST_REBUILD = 2,   /* a converged H is larger than the cell size        */
  SPH_ST_BOX = 4,       /* a support larger than half the box was needed     */
  SPH_ST_CAPACITY = 8,  /* a cell held more particles than a kernel handles  */
  SPH_ST_NEG_U = 16     /* a kick made some internal energy negative         */
};

/* ---- context flags ------------------------------------------------------ */
enum {
  SPH_FLAG_SYNC = 1,        /* wait after each call, return device status    */
  SPH_FLAG_COUNT_PAIRS = 2, /* count in-support pairs (diagnostics, slower)  */
  SPH_FLAG_TIMING = 4,      /* record CUDA events around each kernel group   */
  SPH_FLAG_TREE = 8,        /* nested grids below the top cells (Sec. 2.1 and
                               9.1) for smoothing lengths that span decades   */
  SPH_FLAG_AXIS_SORT = 16,  /* uniform grid: sorted interactions (Sec. 2.2).
                               After each density gather, every cell's
                               particles are ranked along the 13 axes that
                               link it to its neighbours (kAxes x n u16 of
                               context scratch); the density filter walks
                               each neighbour cell along its axis, nearest
                               first, and stops where the distance along the
                               axis reaches the search radius.  Same
                               neighbour sets as without the flag, summed in
                               another order.  Ignored with SPH_FLAG_TREE.  */
  SPH_FLAG_SYMMETRIC = 32   /* uniform grid, cubic spline, Minimal force:
                               each pair within reach is evaluated once
                               (Sec. 2.1, the pair terms are antisymmetric).
                               The density publishes only the neighbours
                               later in sorted order; the force keeps the
                               target's side and writes the partner's side
                               as a record, and the records are grouped by
                               receiver and added in order of their source,
                               so results do not depend on scheduling and a
                               simulation's result is the same alone or in a
                               pool.  Needs context scratch for 64 records
                               (40 bytes each) per particle; more pairs set
                               SPH_ST_CAPACITY.  Masked loops, SPHENIX calls
                               and the other kernels keep the gather form
                               (they then filter the cells themselves).  */
};

/* Smoothing kernels (Sec. 3.1), W(r, h) = w(r/H)/H^3, H = gamma_K h, in the
 * Dehnen & Aly (2012) convention (h is twice the kernel's standard deviation
 * per dimension):
 *   SPH_KERNEL_CUBIC        16/pi [(1-q)^3 - 4 (1/2-q)_+^3],         gamma_K = 1.825742
 *   SPH_KERNEL_QUARTIC      15625/(512 pi) [(1-q)^4 - 5 (3/5-q)_+^4 + 10 (1/5-q)_+^4],
 *                                                                     gamma_K = 2.018932
 *   SPH_KERNEL_WENDLAND_C2  21/(2 pi) (1-q)^4 (1 + 4q),               gamma_K = 1.936492
 * The kernel sets gamma_K everywhere it enters: cell sizes, the smoothing-
 * length equation, the loops and the time-step. */
enum { SPH_KERNEL_CUBIC = 0, SPH_KERNEL_QUARTIC = 1, SPH_KERNEL_WENDLAND_C2 = 2 };

/* Kernel groups timed with SPH_FLAG_TIMING (index into sph_kernel_times). */
enum {
  SPH_T_BUILD = 0,      /* cell grid, keys, counting sort, in-cell order   */
  SPH_T_GATHER = 1,     /* sorted cell-relative copies for the loops       */
  SPH_T_DENSITY = 2,    /* density loop with the smoothing-length solve    */
  SPH_T_FORCE = 3,      /* force loop                                      */
  SPH_T_INTEGRATE = 4,  /* time-step reduction, kicks and drift            */
  SPH_T_COUNT = 5
};

/* Physical and numerical parameters.  sph_default_params fills the values of
 * the paper's "Minimal" flavour: gamma = 5/3, eta = 1.2348 (~48 neighbours),
 * alpha_V = 0.8, beta = 3, epsilon = 1e-4 (Sec. 3.2), the paper's default
 * relative smoothing-length tolerance h_tol = 1e-4 (Sec. 3.1.1), plus
 * max_h_iter = 30, C_CFL = 0.1 and a 5 % cell margin. */
typedef struct sph_params {
  double box_size;     /* side L of the periodic cubic box (> 0)                  */
  double gamma;        /* ratio of specific heats, eq. "eos"                      */
  double eta;          /* resolution parameter of eq. "partition"                 */
  double alpha_v;      /* viscosity constant alpha_V, eq. "balsara"               */
  double beta_v;       /* signal-velocity constant beta                           */
  double eps_balsara;  /* epsilon of eq. "balsara"                                */
  double h_tol;        /* Newton-Raphson stops when the correction |dh| <= h_tol h;
                          that last correction is applied (error ~ 2 h_tol^2)     */
  double cfl;          /* C_CFL of the global time-step                           */
  double cell_margin;  /* cells are >= (1 + cell_margin) * gamma_K * max h        */
  int32_t max_h_iter;  /* iteration cap of the smoothing-length solve             */
  int32_t flags;       /* SPH_FLAG_*                                              */
  int32_t n_leaf;      /* SPH_FLAG_TREE: a cell with at most n_leaf particles is
                          not split (>= 1)                                        */
  int32_t kernel;      /* SPH_KERNEL_*                                            */
  int32_t lanes_per_target; /* uniform-grid loops: 0 = automatic (four lanes per
                          target in rounds of up to 8 targets, else two), 2 or
                          4 = that many lanes for every target (a tuning knob;
                          results agree to rounding, as the lanes split the sums) */
} sph_params;

/* Opaque context: holds the stream, the parameters and the device scratch
 * (cell keys, cell offsets, sorted particle copies), grown on demand. */
typedef struct sph_ctx sph_ctx;

/* Cell lists of one simulation, produced by sph_build_cells.  Device pointers
 * into context scratch, valid until the next sph_build_cells/sph_step on the
 * same context.  cell_start[c] .. cell_start[c+1] is the range of sorted
 * positions of cell c = kx + n_c (ky + n_c kz); perm[s] is the input index of
 * the particle at sorted position s; inside a cell the input indices ascend. */
typedef struct sph_cells {
  int64_t n;                 /* particles binned                                  */
  int32_t n_c;               /* cells per side (host copy; needs SPH_FLAG_SYNC or
                                sph_cells_sync, else -1)                          */
  const int32_t* n_c_dev;    /* device: cells per side                            */
  const int32_t* cell_start; /* device: n_c^3 + 1 offsets                         */
  const int32_t* perm;       /* device: n                                         */
} sph_cells;

/* Input particles of one simulation (device pointers, length n). */
typedef struct sph_particles {
  int64_t n;
  const double *x, *y, *z;    /* positions in [0, L)                              */
  const float *vx, *vy, *vz;  /* velocities                                       */
  const float *m;             /* masses                                           */
  const float *u;             /* internal energy per unit mass                    */
} sph_particles;

/* Outputs of the density loop (device pointers, length n, input order).
 * n_iter may be NULL. */
typedef struct sph_density_out {
  float *h;        /* converged smoothing length                                   */
  float *rho;      /* density rho_i = sum_j m_j W(r_ij, h_i), self included        */
  float *f;        /* f_i = [1 + h_i/(3 rho_i) d rho_i/dh]^-1                       */
  float *div_v;    /* velocity divergence                                          */
  float *curl_v;   /* norm of the velocity curl                                    */
  float *P;        /* pressure (gamma - 1) u rho                                   */
  float *c;        /* sound speed sqrt(gamma P / rho)                              */
  float *balsara;  /* Balsara switch B_i                                           */
  int32_t *n_iter; /* Newton-Raphson passes used (optional)                        */
} sph_density_out;

/* Outputs of the force loop (device pointers, length n, input order). */
typedef struct sph_force_out {
  float *ax, *ay, *az;  /* acceleration                                            */
  float *du_dt;         /* internal energy rate                                    */
  float *v_sig;         /* max_j signal velocity over neighbours                   */
} sph_force_out;

/* State of a pool of independent simulations advanced together by sph_step.
 * All arrays are device pointers over the whole pool (length n_total);
 * simulation s owns particles [sim_offset[s], sim_offset[s+1]) and lives in a
 * periodic cube of side box_size[s].  a, du/dt and v_sig hold the previous
 * force evaluation on entry (run sph_density + sph_force once to start) and
 * the new one on exit; the density outputs are refreshed too. */
typedef struct sph_pool {
  int32_t n_sims;
  int64_t n_total;
  const int64_t* sim_offset;  /* device, n_sims + 1, ascending, [0] = 0            */
  const double* box_size;     /* device, n_sims                                    */
  double *x, *y, *z;          /* in/out positions                                  */
  float *vx, *vy, *vz;        /* in/out velocities                                 */
  float *u;                   /* in/out internal energy                            */
  const float *m;             /* masses                                            */
  float *h;                   /* in/out smoothing length (warm start)              */
  float *ax, *ay, *az, *du_dt, *v_sig;             /* in/out force results         */
  float *rho, *f, *div_v, *curl_v, *P, *c, *balsara; /* out density results        */
  double *dt;                 /* device, n_sims: time-step taken by each sim       */
  int32_t *n_iter;            /* optional (NULL): Newton-Raphson passes            */
} sph_pool;

void sph_default_params(sph_params* p);

/* Creates a context bound to `stream` (a cudaStream_t; NULL = legacy default
 * stream).  Allocates nothing on the device until the first call that needs
 * scratch.  Returns SPH_E_INVAL for bad parameters. */
int sph_create(sph_ctx** ctx, const sph_params* p, void* stream);
void sph_destroy(sph_ctx* ctx);
const char* sph_error_string(int code);

/* Device status word accumulated since the last call (SPH_ST_* bits); waits
 * for the context's stream, then clears the word. */
int sph_status(sph_ctx* ctx, int32_t* status_out);

/* Bins n particles into the cell grid (Sec. 2.1).  The grid has
 * n_c = max(1, floor(L / ((1 + cell_margin) gamma_K max_i h_i))) cells per
 * side (capped so that n_c^3 <= 8 n + 216), computed on the device; a
 * support (1 + cell_margin) gamma_K max h above L/2 sets SPH_ST_BOX (and
 * SPH_E_BOX when synchronous), since the minimum image would no longer be
 * unique.  Cell coordinates are k = floor(fl(fl(x n_c) / L)), clamped
 * to n_c - 1 (IEEE double, round to nearest); the order inside a cell is
 * ascending input index, so the lists are exactly reproducible.
 *
 * With SPH_FLAG_TREE the cells of this grid are the top level of nested
 * grids: below each, a cell is split into 8 children until it holds at most
 * n_leaf particles, or its children would be narrower than (1 + cell_margin)
 * times the largest support inside it, or it is 1/1024 of the top cell.
 * cell_start still delimits the top cells, but inside a top cell the order is
 * the Morton order of the 1024^3 sub-cells (ties: ascending input index), so
 * that every cell of every level is one contiguous range. */
int sph_build_cells(sph_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                    const float* h, sph_cells* out);

/* Allocates the context's scratch for up to n_total particles in up to
 * n_sims simulations (and the nested-grid scratch with SPH_FLAG_TREE), so that
 * later calls of that size allocate nothing: use it before capturing a CUDA
 * graph or before serving requests whose latency matters.  Waits for the
 * stream when it has to reallocate.  The paper has no counterpart (a
 * deployment aid). */
int sph_reserve(sph_ctx* ctx, int64_t n_total, int32_t n_sims);

/* Waits for the stream and fills out->n_c from the device. */
int sph_cells_sync(sph_ctx* ctx, sph_cells* cells);

/* Copies the cell lists of `cells` into caller buffers (host or device;
 * cell_start_dst holds n_c^3 + 1 entries, perm_dst holds n).  Waits for the
 * stream; fills cells->n_c. */
int sph_cells_copy(sph_ctx* ctx, sph_cells* cells, int32_t* cell_start_dst, int32_t* perm_dst);

/* Density loop with the smoothing-length solve (Sec. 3.1).  h_in is the
 * starting guess (may alias out->h).  Each particle's h is iterated with
 * Newton-Raphson on n_hat(h) - (eta/h)^3, using dn_hat/dh, until the relative
 * correction is below h_tol (the last correction is applied, and the outputs
 * are evaluated at that final h); H is capped at the cell size (a particle that would
 * need more sets SPH_ST_REBUILD and returns twice its capped h in out->h:
 * rebuild the cells from out->h and call again, which at least doubles the
 * cells that particle needs).  Sums are accumulated in FP32 on coordinates relative to the
 * particle's cell; the convergence test runs in FP64.  With SPH_FLAG_TREE the
 * cell is the particle's leaf, and coordinates are relative to the leaf with
 * an exact integer part (1/1024 of a top cell), so precision follows the
 * leaf's size. */
int sph_density(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in, const float* h_in,
                sph_density_out* out);

/* Force loop (Sec. 3.2) over all pairs with r_ij < max(H_i, H_j), reading the
 * density results d (h, rho, f, P, c, balsara; input order). */
int sph_force(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in,
              const sph_density_out* d, sph_force_out* out);

/* The loops on an active subset (Sec. 2.4, the per-particle time-step
 * hierarchy: only the particles whose step ends are updated, and every other
 * particle is a neighbour at its drifted position).  active: device uint8,
 * length n, input order; nonzero marks a particle to update.  Outputs are
 * written for the active particles only; the others keep their contents.
 * sph_force_active reads the density results of every particle (the inactive
 * ones from their last update).  On the uniform grid the force reuses the
 * neighbour lists of the preceding sph_density_active on the same cells when
 * it is given the same mask pointer (whose contents must not change in
 * between); else it filters its own.  On the nested grids (SPH_FLAG_TREE) the
 * force needs them: it takes the same mask pointer as the preceding density
 * on the same cells, or follows an unmasked density (else SPH_E_INVAL); the
 * density also walks the inactive particles' lists at their current supports,
 * for the pairs an active particle receives from a larger inactive support
 * (its outputs stay untouched).  The outputs of an active particle equal those
 * of the unmasked loops up to the order of the FP32 sums (a block deals its
 * active targets to lanes anew). */
int sph_density_active(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in, const float* h_in,
                       const uint8_t* active, sph_density_out* out);
int sph_force_active(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in,
                     const sph_density_out* d, const uint8_t* active, sph_force_out* out);

/* Time bins of the power-of-two time-step hierarchy (Sec. 2.4) with the first
 * time-step limiter (the SPH section's "Time-step limiter", Delta = 4), on the
 * cells of the last build (both grid modes; on the nested grids after an
 * unmasked density of that build, whose lists and reverse pairs it walks):
 *   dt_i  = C_CFL gamma_K h_i / v_sig,i        (FP32: fl(fl(c h_i) / v_sig,i),
 *                                               c = fl(C_CFL gamma_K))
 *   bin_i = smallest b in [0, max_bin] with dt_max 2^-b <= dt_i (max_bin if
 *           none; 0 where v_sig <= 0), i.e. a step dt_max 2^-bin_i <= dt_i;
 *   bin_i = max(bin_i, max_j bin_j - 2) over the force pairs j != i with
 *           r_ij < max(H_i, H_j), applied once (a step at most 4 times the
 *           smallest neighbour step).
 *   d       density results of every particle (h, and the force records)
 *   v_sig   device float, n: signal velocities (from sph_force)
 *   cfl > 0, dt_max > 0, 0 <= max_bin <= 62
 *   bins    device int32, n, input order: written
 * The limiter is a neighbour pass over the lists of the preceding density
 * (the force loop's template with a one-line pair function). */
int sph_time_bins(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in, const sph_density_out* d,
                  const float* v_sig, double cfl, double dt_max, int32_t max_bin, int32_t* bins);

/* One sub-step of the power-of-two time-step hierarchy (Sec. 2.4, "Local
 * time-step optimisations") for a single simulation (pool with n_sims = 1;
 * both grid modes).  Time runs on integer ticks, tau = dt_max / 2^max_bin each; a
 * particle in bin b takes steps of 2^(max_bin - b) ticks starting at
 * t_begin[i] (a multiple of that length).  In this mode the pool's vx, vy, vz
 * and u are the particle's half-kicked values for its current step, and its
 * a, du/dt, v_sig and density results are those of its last evaluation.  The
 * call:
 *   t_next = min_i (t_begin_i + step_i)                  (returned, host)
 *   every particle drifts from t_now to t_next; the loops see the predicted
 *   v_half + a (t_next - t_begin - step/2) tau (u alike);
 *   the particles whose step ends at t_next are active: the cells are rebuilt,
 *   the density and force run for them (sph_density_active / sph_force_active),
 *   then each gets the second half kick over its old step, a new bin (with
 *   SPH_HIER_ADAPT: that of sph_time_bins with params.cfl, limited against the
 *   bins the inactive neighbours hold; else its old bin; in both cases
 *   shortened until the new step divides t_next), the first half kick over
 *   its new step, and t_begin = t_next.
 * The second and third time-step limiters of the SPH section ("Time-step
 * limiter") end the current step of an inactive particle j at t_next: its v
 * and u become the predicted ones at t_next, it takes a new bin (shortened
 * until its step divides t_next), the first half kick over that step, and
 * t_begin = t_next.
 *   SPH_HIER_WAKEUP (Saitoh & Makino 2009): after the active particles have
 *     their new bins, every inactive j within r_ij < max(H_i, H_j) of an
 *     active i (uniform grid: FP64 minimum-image distance; nested grids: the
 *     force pairs of the sub-step, decided in FP32 like the force's) whose
 *     step is more than 4 times longer, bin_j < bin_i - 2, is woken with bin
 *     max_i (bin_i - 2);
 *   sync (device uint8, n, or NULL): flags of particles to synchronise, say
 *     those a source term changed between sub-steps.  A flagged inactive
 *     particle ends its step with its CFL bin (SPH_HIER_ADAPT; the limiter of
 *     the active particles then sees that bin) or its held bin, raised to its
 *     wake-up bin if it has one.  Every flag is cleared (set to 0).
 * SPH_HIER_PREDICT: the drift also carries every particle's h and density
 * over [t_now, t_next] with its last velocity divergence held (dh/dt =
 * h div_v / 3, continuity drho/dt = -rho div_v: h e^(div_v dt/3),
 * rho e^(-div_v dt), in place in the pool), and sets P = (gamma - 1) u rho and
 * c = sqrt(gamma P / rho) at the predicted u; the inactive particles enter the
 * loops with these values, the active ones start their h solve from them.
 * SPH_HIER_KEEP_CELLS: the cells are rebuilt only when they may no longer hold
 * every pair: while the largest support (gamma_K max h after the drift) plus
 * twice the drift bound since the last build (max |v| dt summed over the
 * sub-steps) stays below a cell side, the sub-step keeps the cells of the last
 * build of this call's kind (positions taken relative to the cell each particle
 * is filed in, nearest periodic image) and caps the supports of the density
 * at the cell less twice the drift bound; a support reaching that cap rebuilds
 * and repeats the density.  The results then differ from a fresh build's by
 * the FP32 rounding of the relative positions only.  Between calls the pool's
 * positions must change only through sph_hier_substep (any other build on the
 * context, or a different n, rebuilds).  Uniform grid only (SPH_E_INVAL with
 * SPH_FLAG_TREE: the nested grids are rebuilt every sub-step).
 * bins (int32) and t_begin (int64) are device arrays of n, updated in place;
 * 0 <= max_bin <= 40; options: SPH_HIER_* bits (others: SPH_E_INVAL).  With
 * SPH_FLAG_SYNC a density that needs larger cells is rebuilt and repeated.
 * Waits for the stream (it returns t_next). */
enum {
  SPH_HIER_ADAPT = 1,   /* new bins from the CFL condition and the first limiter */
  SPH_HIER_WAKEUP = 2,  /* the wake-up limiter                                   */
  SPH_HIER_PREDICT = 4,    /* prediction of h, rho, P, c in the drift (below)    */
  SPH_HIER_KEEP_CELLS = 8  /* keep the cells of an earlier sub-step (below)      */
};
int sph_hier_substep(sph_ctx* ctx, const sph_pool* pool, int32_t* bins, int64_t* t_begin, double dt_max,
                     int32_t max_bin, int64_t t_now, int32_t options, uint8_t* sync, int64_t* t_next_out);

/* The same sub-step with the tick on the device: *tick (device int64) is the
 * current tick t_now on entry and is replaced by t_next on the stream.  Nothing
 * waits for the stream, so a CUDA graph can capture the call and replay it,
 * each replay one more sub-step (small sub-steps are launch-bound).  Not with
 * SPH_HIER_KEEP_CELLS, SPH_FLAG_SYNC or SPH_FLAG_TIMING (SPH_E_INVAL).  The
 * first call on a context allocates its scratch: make it before a capture. */
int sph_hier_substep_dev(sph_ctx* ctx, const sph_pool* pool, int32_t* bins, int64_t* t_begin, double dt_max,
                         int32_t max_bin, int64_t* tick, int32_t options, uint8_t* sync);

/* One kick-drift-kick step of every simulation of the pool (Sec. 2.4):
 *   dt = C_CFL min_i H_i / v_sig,i per simulation (FP64 reduction),
 *   half kick of v and u, drift of x in FP64 with periodic wrap, prediction
 *   of v and u for the loops, cell rebuild, density, force, half kick.
 * n_sims = 1 is the plain path; n_sims > 1 runs every loop as one launch over
 * all simulations.  With SPH_FLAG_SYNC, a step whose density reports
 * SPH_ST_REBUILD is rebuilt with larger cells and repeated internally. */
int sph_step(sph_ctx* ctx, const sph_pool* pool);

/* ---- SPHENIX flavour (Sec. 3.3) ------------------------------------------
 * The default flavour of the paper: a viscosity parameter alpha_V,i carried
 * by each particle and evolved with a shock indicator (eqs. "sphenix_visc1"
 * to "sphenix_visc4"), the pair parameter alpha_V,ij = (alpha_V,i +
 * alpha_V,j)/2 (B_i + B_j)/2 (eq. "av_ij"), and artificial conduction with a
 * parameter alpha_c,i evolved from the Laplacian of u and limited near shocks
 * (eqs. "art_cond", "artconddt", "condshocklimiter", "conductionlimiter").
 * An evaluation is: sph_density, then sph_sphenix_gradient (viscosity
 * update, then a third neighbour loop over r < H_i that computes lap u and
 * updates alpha_c), then sph_force_sphenix.  Where the paper's equations are
 * garbled or silent, the library reads them as follows:
 *   viscosity:  rate = (div_v - div_v_prev)/dt (0 if dt = 0),
 *               S = H^2 max(0, -rate),
 *               alpha_loc = alpha_V,max S/(v_sig^2 + S) (0 if S = 0), with
 *               v_sig from the previous force evaluation;
 *               alpha_V <- alpha_loc if that is larger, else
 *               alpha_loc + (alpha_V - alpha_loc) exp(-ell c dt / H);
 *   gradient:   lap u_i = 2 sum_{j != i, r < H_i} (m_j/rho_j)(u_i - u_j) W'(r, h_i)/r,
 *               v_c,i = max_j v_c,ij,
 *               v_c,ij = |v_ij . x_ij|/r + sqrt(2 |P_i - P_j|/(rho_i + rho_j)),
 *               alpha_V,max,i = max(alpha_V,i, max_j alpha_V,j);
 *   conduction: alpha_c += dt [beta_c H lap u / sqrt(u) - (alpha_c - alpha_c,min) v_c,i / H]
 *               (no source where u <= 0), then limited to
 *               [alpha_c,min, alpha_c,max (1 - alpha_V,max,i / alpha_V,max)];
 *   force:      du_i/dt += alpha_c,ij v_c,ij m_j (u_i - u_j)
 *                          [f_i W'(r, h_i) + f_j W'(r, h_j)] / (rho_i + rho_j)
 *               over the force pairs, alpha_c,ij = (P_i alpha_c,i + P_j alpha_c,j)/(P_i + P_j)
 *               (0 if P_i + P_j = 0).
 * Both grid modes: with SPH_FLAG_TREE the gradient pass and the force walk
 * the nested grids' lists and reverse pairs (the gradient pass only the
 * lists: it reaches r < H_i, inside each target's list radius). */
typedef struct sph_sphenix_params {
  double alpha_v_max;  /* alpha_V,max (2)                               */
  double ell;          /* viscosity decay length ell (0.05)             */
  double beta_c;       /* beta_c of eq. "artconddt" (1)                 */
  double alpha_c_min;  /* alpha_c,min (0)                               */
  double alpha_c_max;  /* alpha_c,max of eq. "condshocklimiter" (1)     */
} sph_sphenix_params;

/* Per-particle SPHENIX arrays of one simulation (device, length n, input order). */
typedef struct sph_sphenix_state {
  float *alpha_v;       /* in/out: viscosity parameter alpha_V,i               */
  float *alpha_c;       /* in/out: conduction parameter alpha_c,i              */
  float *div_v_prev;    /* in: the divergence of the previous evaluation;
                           out: this evaluation's (d->div_v)                   */
  const float *v_sig;   /* in: the signal velocity of the previous force       */
  float *lap_u;         /* out, optional (NULL): lap u                         */
} sph_sphenix_state;

void sph_sphenix_default_params(sph_sphenix_params* x);

/* Between sph_density and sph_force_sphenix on the same cells: updates
 * st->alpha_v over the step dt (>= 0), then runs the gradient pass and
 * updates st->alpha_c over dt.  d holds this evaluation's density results. */
int sph_sphenix_gradient(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in,
                         const sph_density_out* d, const sph_sphenix_params* x, double dt,
                         sph_sphenix_state* st);
/* SPHENIX force loop: sph_force with the viscosity parameters alpha_v and the
 * conduction term with the parameters alpha_c (device, input order), both as
 * left by sph_sphenix_gradient. */
int sph_force_sphenix(sph_ctx* ctx, const sph_cells* cells, const sph_particles* in,
                      const sph_density_out* d, const float* alpha_v, const float* alpha_c,
                      sph_force_out* out);
/* sph_step with the SPHENIX force evaluation (density, viscosity update over
 * the step's dt, gradient pass, SPHENIX force), for a pool.  pool->div_v and
 * pool->v_sig hold the previous evaluation's values on entry (as after
 * sph_density + sph_sphenix_gradient + sph_force_sphenix); alpha_v and
 * alpha_c are device arrays of n_total (pool order), updated in place. */
int sph_step_sphenix(sph_ctx* ctx, const sph_pool* pool, const sph_sphenix_params* x, float* alpha_v,
                     float* alpha_c);

/* FP64 conservation sums of a pool after a force evaluation, per simulation:
 * out[4 s + 0..2] = sum m a, out[4 s + 3] = sum m (v . a + du/dt) with the
 * velocities given (device array out of 4 n_sims doubles). */
int sph_conservation(sph_ctx* ctx, const sph_pool* pool, double* out);

/* Friends-of-friends groups (Sec. 7.1) of n particles in the periodic box of
 * side params.box_size.  Particles i and j are friends when their
 * minimum-image distance is below the linking length b:
 *   d = x_i - x_j per axis, wrapped once into [-L/2, L/2],
 *   dx*dx + dy*dy + dz*dz < b*b   (FP64, evaluated left to right);
 * a group is a connected component of that relation.
 *   x, y, z   device FP64, n each, in [0, L)
 *   link_len  b, 0 < b <= L/3 (else SPH_E_INVAL / SPH_E_BOX)
 *   group     device int32, n, written: group[i] = the smallest index of i's
 *             group (so group[i] == i marks one particle per group)
 * The search reuses the cell build with cells at least b wide (it replaces
 * the context's current cells).  Asynchronous on the context's stream;
 * with SPH_FLAG_SYNC it waits and returns the device status
 * (SPH_E_CAPACITY if a bounded union-find loop gave up). */
int sph_fof(sph_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
            double link_len, int32_t* group);

/* With SPH_FLAG_TIMING: waits for the stream, then returns the summed device
 * time in milliseconds (ms_out[SPH_T_COUNT]) and the number of timed launches
 * of each group (calls_out[SPH_T_COUNT], may be NULL) since the last query,
 * and resets both. */
int sph_kernel_times(sph_ctx* ctx, double* ms_out, int64_t* calls_out);

/* Number of pairs counted by the last density and force launches when the
 * context has SPH_FLAG_COUNT_PAIRS (waits for the stream):
 * out[0] = density pairs r < H_i (self included, last Newton pass),
 * out[1] = force pairs r < max(H_i, H_j), j != i. */
int sph_pair_counts(sph_ctx* ctx, int64_t* out);

/* Moves the particle fields (x .. balsara; not dt or n_iter) of n_ranges
 * whole simulations between two pools (device arrays, enqueued on `stream`,
 * a cudaStream_t): simulation r occupies offsets[r] .. offsets[r+1] of
 * `packed` (offsets[0] = 0, offsets[n_ranges] <= packed->n_total) and the
 * same number of particles from starts[r] on in `spread`.  to_packed = 1
 * copies spread -> packed (gathering a batch out of a store), 0 copies back.
 * Only sim_offset-free fields are touched; the ranges must not overlap.  The
 * paper has no counterpart: it serves many resident simulations. */
int sph_pool_move(const sph_pool* spread, const sph_pool* packed, int32_t n_ranges, const int64_t* starts,
                  const int64_t* offsets, int32_t to_packed, void* stream);

/* Diagnostics of the last nested-grid build and density (SPH_FLAG_TREE; waits
 * for the stream): out[0] = target groups, out[1] = targets that left their
 * group for the per-target kernel (a list overflow or a support past the list
 * radius; needs SPH_FLAG_COUNT_PAIRS, else 0), out[2] = reverse pairs emitted,
 * out[3] = targets solved by the per-target kernel (those, and the ones
 * re-solved at a coarser level).  All zero without nested grids. */
int sph_tree_counts(sph_ctx* ctx, int64_t* out);

/* Cell build for callers that cannot allocate device memory (code running in
 * another framework's memory arena, loops whose allocator must not
 * synchronise the device, plugins that are only handed buffers).  The paper
 * has no counterpart: this is a deployment variant of sph_build_cells.
 *
 * It computes the same grid and the same lists as sph_build_cells on a
 * context with the cubic-spline kernel (the default), the uniform grid (no
 * SPH_FLAG_TREE) and the same box_size and cell_margin: bit-identical
 * cell_start and perm.  The cells are sized for the cubic spline's support
 * H = 1.825742 h; a caller of the quartic or Wendland C2 kernel passes h
 * scaled by gamma_K(kernel) / 1.825742, or uses sph_build_cells.  All of its
 * scratch is one fixed array compiled into the library (about 3.1 MB, held
 * by every GPU that loads the library until the process exits); it calls no
 * allocating routine.
 *   n              particles, 0 <= n <= 65536 (more: SPH_E_CAPACITY)
 *   x, y, z, h     device inputs (length n)
 *   cell_start     device output, cell_start_cap >= 8 n + 217 entries; the
 *                  first n_c^3 + 1 are written
 *   perm           device output (length n)
 *   n_c_out        optional device int32: cells per side
 *   status_out     optional device int32: SPH_ST_* bits of this build
 *   stream         cudaStream_t (NULL = legacy default stream)
 * The first call on a device resolves the address of the fixed array on that
 * device (with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * it again on a device after cudaDeviceReset (the kept address would be
 * stale).  Every call on a device shares the array: calls whose work
 * overlaps on the GPU (different streams, or different host threads) race
 * and corrupt each other's results.  Returns SPH_OK when the work is
 * enqueued. */
int sph_build_cells_static(int64_t n, const double* x, const double* y, const double* z,
                           const float* h, double box_size, double cell_margin,
                           int32_t* cell_start, int64_t cell_start_cap, int32_t* perm,
                           int32_t* n_c_out, int32_t* status_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
