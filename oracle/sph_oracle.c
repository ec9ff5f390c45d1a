/*
 * sph_oracle.c -- plain, serial, FP64 CPU oracle for the SPH neighbour loops of
 * SWIFT (Schaller et al., "SWIFT: A modern highly-parallel gravity and smoothed
 * particle hydrodynamics solver", MNRAS 2024), Sec. 2.1 (cell grid) and
 * Sec. 3.1-3.2 ("Minimal" density-energy SPH with Balsara-switched viscosity).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg.  The library never links, loads or calls it, and it shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is evaluated in double precision straight from the definitions:
 * no blocking, no fusion, no reordering.  Neighbour candidates come from a
 * plain bucket grid (a range search that returns every particle within the
 * requested radius, checked against O(N^2) brute force by the tests) or, on
 * request, from brute force itself.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *  - kernel: cubic spline in the Dehnen & Aly (2012) form W(r,h)=w(r/H)/H^3,
 *    H = gamma_K h, gamma_K = 1.825742, w(q) = 16/pi [(1-q)^3 - 4 (1/2-q)_+^3]
 *    (Sec. 3.1, eq. "kernel"; the paper cites the form but prints no w);
 *  - the number density includes the self term j = i (eq. "numberdensity");
 *  - smoothed divergence / curl use velocity differences (Sec. 3.1.2);
 *    the curl sign is fixed so that rigid rotation with angular velocity
 *    omega returns +2 omega (only its norm enters the Balsara switch);
 *  - f_i = [1 + h_i/(3 rho_i) d rho_i/dh]^-1 (Sec. 3.2 with the inverse that
 *    the comoving form in Sec. 5 prints);
 *  - second pressure term and viscosity use grad_i W(r_ij, h_j);
 *    nu_ij divides by the mean density (rho_i + rho_j)/2;
 *    alpha_ij = alpha_V (B_i + B_j)/2; du/dt viscosity uses the symmetric
 *    nu_ij/4 v_ij.(f_i G_i + f_j G_j) (Sec. 3.2, eqs. "basicartvisc",
 *    "alpha", "nuij", "balsara");
 *  - c_i = sqrt(gamma P_i / rho_i) (not printed; ideal-gas sound speed).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* --------------------------------------------------------------------------
 * Kernels (Sec. 3.1, eq. "kernel"): W(r, h) = w(q)/H^3, q = r/H, H = gamma_K h,
 * in the Dehnen & Aly (2012) convention, where h is twice the kernel's
 * standard deviation per dimension, so gamma_K = sqrt(3 / (4 <q^2>)) with
 * <q^2> = int 4 pi q^4 w(q) dq.  The paper names the cubic spline (the
 * default), the quartic spline and the Wendland C2 kernel (Sec. 3.1):
 *   0 cubic:       w = 16/pi [(1-q)^3 - 4 (1/2-q)_+^3],             gamma_K = 1.825742
 *   1 quartic:     w = 15625/(512 pi) [(1-q)^4 - 5 (3/5-q)_+^4
 *                                      + 10 (1/5-q)_+^4],            gamma_K = 2.018932
 *   2 Wendland C2: w = 21/(2 pi) (1-q)^4 (1+4q),                      gamma_K = 1.936492
 * (w = 0 for q >= 1).  The kernel of every call is set by oracle_set_kernel.
 * -------------------------------------------------------------------------- */
static int or_kernel = 0;
static double OR_GAMMA_K = 1.825742;

int oracle_set_kernel(int k) {
  static const double gam[3] = {1.825742, 2.018932, 1.936492};
  if (k < 0 || k > 2) return -1;
  or_kernel = k;
  OR_GAMMA_K = gam[k];
  return 0;
}

double oracle_gamma_k(void) { return OR_GAMMA_K; }

static double or_pos(double x) { return x > 0.0 ? x : 0.0; }

double oracle_w(double q) {
  if (q >= 1.0) return 0.0;
  double a = 1.0 - q;
  if (or_kernel == 1) {
    double b = or_pos(0.6 - q), c = or_pos(0.2 - q);
    return (15625.0 / (512.0 * OR_PI)) * (a * a * a * a - 5.0 * b * b * b * b + 10.0 * c * c * c * c);
  }
  if (or_kernel == 2) return (21.0 / (2.0 * OR_PI)) * a * a * a * a * (1.0 + 4.0 * q);
  double w = a * a * a;
  if (q < 0.5) {
    double b = 0.5 - q;
    w -= 4.0 * b * b * b;
  }
  return (16.0 / OR_PI) * w;
}

double oracle_dw_dq(double q) {
  if (q >= 1.0) return 0.0;
  double a = 1.0 - q;
  if (or_kernel == 1) {
    double b = or_pos(0.6 - q), c = or_pos(0.2 - q);
    return (15625.0 / (512.0 * OR_PI)) * (-4.0) * (a * a * a - 5.0 * b * b * b + 10.0 * c * c * c);
  }
  if (or_kernel == 2) return (21.0 / (2.0 * OR_PI)) * (-20.0) * q * a * a * a;
  double d = -3.0 * a * a;
  if (q < 0.5) {
    double b = 0.5 - q;
    d += 12.0 * b * b;
  }
  return (16.0 / OR_PI) * d;
}

/* W(r, h) and dW/dr(r, h). */
static double or_W(double r, double h) {
  double H = OR_GAMMA_K * h;
  return oracle_w(r / H) / (H * H * H);
}
static double or_dWdr(double r, double h) {
  double H = OR_GAMMA_K * h;
  return oracle_dw_dq(r / H) / (H * H * H * H);
}
/* dW/dh at fixed r: W = w(r/H)/H^3 -> dW/dh = -(3 W + r dW/dr)/h. */
static double or_dWdh(double r, double h) {
  return -(3.0 * or_W(r, h) + r * or_dWdr(r, h)) / h;
}

/* --------------------------------------------------------------------------
 * Periodic helpers.
 * -------------------------------------------------------------------------- */
/* One wrap of a coordinate into [0, L). */
double oracle_wrap(double x, double L) {
  if (x < 0.0) x += L;
  if (x >= L) x -= L;
  return x;
}
/* Minimum-image component of a displacement. */
static double or_min_image(double d, double L) {
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}

/* --------------------------------------------------------------------------
 * Cell grid (Sec. 2.1, the Verlet-list grid): cell coordinate
 *   k = floor( fl(fl(x * n_c) / L) ), clamped to n_c - 1,
 * cell id = kx + n_c (ky + n_c kz); particles ordered by cell id, ties kept in
 * ascending input index (a stable counting sort).
 * -------------------------------------------------------------------------- */
int32_t oracle_cell_coord(double x, double L, int32_t n_c) {
  double s = (x * (double)n_c) / L;
  int32_t k = (int32_t)floor(s);
  if (k < 0) k = 0;
  if (k > n_c - 1) k = n_c - 1;
  return k;
}

int oracle_build_cells(int64_t n, const double* x, const double* y, const double* z,
                       double L, int32_t n_c, int32_t* cell_start, int32_t* perm) {
  if (n < 0 || n_c < 1) return -1;
  int64_t n_cells = (int64_t)n_c * n_c * n_c;
  int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t* count = (int64_t*)calloc((size_t)n_cells + 1, sizeof(int64_t));
  if (!key || !count) { free(key); free(count); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    int32_t kx = oracle_cell_coord(x[i], L, n_c);
    int32_t ky = oracle_cell_coord(y[i], L, n_c);
    int32_t kz = oracle_cell_coord(z[i], L, n_c);
    key[i] = kx + n_c * (ky + n_c * kz);
    count[key[i] + 1] += 1;
  }
  for (int64_t c = 0; c < n_cells; ++c) count[c + 1] += count[c];
  for (int64_t c = 0; c <= n_cells; ++c) cell_start[c] = (int32_t)count[c];
  /* stable placement: walk the input in order */
  for (int64_t i = 0; i < n; ++i) {
    perm[count[key[i]]] = (int32_t)i;
    count[key[i]] += 1;
  }
  free(key);
  free(count);
  return 0;
}

/* --------------------------------------------------------------------------
 * Depth-first order of the nested grids (Sec. 2.1 and Sec. 9.1: particles of
 * every cell of every level of the octree below a top cell are contiguous).
 * Each top cell is split 10 times (1024 sub-cells per side); a particle's
 * sub-cell on one axis is g = floor(1024 fl(fl(x n_c) / L)), clamped to its
 * top cell k: g in [1024 k, 1024 k + 1023].  Inside a top cell, particles are
 * ordered by the child index (x bit + 2 y bit + 4 z bit) at depth 1, then at
 * depth 2, ... depth 10, i.e. by the number whose base-8 digits are those
 * child indices; ties keep ascending input index.  Top cells come in
 * ascending cell id (kx + n_c (ky + n_c kz)).
 * -------------------------------------------------------------------------- */
static int32_t or_fine(double x, double L, int32_t n_c, int32_t k) {
  double s = (x * (double)n_c) / L;
  double g = floor(s * 1024.0);
  double lo = 1024.0 * (double)k, hi = lo + 1023.0;
  if (g < lo) g = lo;
  if (g > hi) g = hi;
  return (int32_t)(g - lo);
}

typedef struct {
  uint64_t key;
  int32_t idx;
} or_tkey;

static int or_tkey_cmp(const void* a, const void* b) {
  const or_tkey* p = (const or_tkey*)a;
  const or_tkey* q = (const or_tkey*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx ? 1 : 0);
}

int oracle_tree_order(int64_t n, const double* x, const double* y, const double* z, double L, int32_t n_c,
                      int32_t* cell_start, int32_t* perm) {
  if (n < 0 || n_c < 1) return -1;
  int64_t n_cells = (int64_t)n_c * n_c * n_c;
  or_tkey* t = (or_tkey*)malloc(sizeof(or_tkey) * (size_t)(n > 0 ? n : 1));
  int64_t* count = (int64_t*)calloc((size_t)n_cells + 1, sizeof(int64_t));
  if (!t || !count) { free(t); free(count); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    int32_t kx = oracle_cell_coord(x[i], L, n_c);
    int32_t ky = oracle_cell_coord(y[i], L, n_c);
    int32_t kz = oracle_cell_coord(z[i], L, n_c);
    int32_t gx = or_fine(x[i], L, n_c, kx), gy = or_fine(y[i], L, n_c, ky), gz = or_fine(z[i], L, n_c, kz);
    uint64_t digits = 0;
    for (int d = 1; d <= 10; ++d) {
      int b = 10 - d; /* bit of the sub-cell coordinate chosen at depth d */
      uint64_t child = (uint64_t)(((gx >> b) & 1) + 2 * ((gy >> b) & 1) + 4 * ((gz >> b) & 1));
      digits = digits * 8 + child;
    }
    int64_t cell = kx + (int64_t)n_c * (ky + (int64_t)n_c * kz);
    t[i].key = ((uint64_t)cell << 30) + digits;
    t[i].idx = (int32_t)i;
    count[cell + 1] += 1;
  }
  qsort(t, (size_t)n, sizeof(or_tkey), or_tkey_cmp);
  for (int64_t c = 0; c < n_cells; ++c) count[c + 1] += count[c];
  for (int64_t c = 0; c <= n_cells; ++c) cell_start[c] = (int32_t)count[c];
  for (int64_t i = 0; i < n; ++i) perm[i] = t[i].idx;
  free(t);
  free(count);
  return 0;
}

/* --------------------------------------------------------------------------
 * Range search: a bucket grid over the periodic box.  or_collect returns
 * every particle j whose minimum-image distance to point p is < R (and, if
 * skip >= 0, j != skip), with its displacement p - x_j.
 * -------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  double L;
  const double *x, *y, *z;
  int32_t ng;
  double g;
  int32_t* start; /* ng^3 + 1 */
  int32_t* idx;   /* n */
  int brute;
} or_grid;

typedef struct {
  int64_t len, cap;
  int32_t* j;
  double *dx, *dy, *dz, *r;
} or_list;

static int or_list_push(or_list* l, int32_t j, double dx, double dy, double dz, double r) {
  if (l->len == l->cap) {
    int64_t cap = l->cap ? 2 * l->cap : 256;
    int32_t* nj = (int32_t*)realloc(l->j, sizeof(int32_t) * cap);
    if (!nj) return -2;
    l->j = nj;
    double* a = (double*)realloc(l->dx, sizeof(double) * cap); if (!a) return -2; l->dx = a;
    a = (double*)realloc(l->dy, sizeof(double) * cap); if (!a) return -2; l->dy = a;
    a = (double*)realloc(l->dz, sizeof(double) * cap); if (!a) return -2; l->dz = a;
    a = (double*)realloc(l->r, sizeof(double) * cap); if (!a) return -2; l->r = a;
    l->cap = cap;
  }
  l->j[l->len] = j;
  l->dx[l->len] = dx;
  l->dy[l->len] = dy;
  l->dz[l->len] = dz;
  l->r[l->len] = r;
  l->len += 1;
  return 0;
}
static void or_list_free(or_list* l) {
  free(l->j); free(l->dx); free(l->dy); free(l->dz); free(l->r);
  memset(l, 0, sizeof(*l));
}

static int32_t or_grid_coord(const or_grid* G, double x) {
  int32_t k = (int32_t)floor(x / G->g);
  if (k < 0) k = 0;
  if (k > G->ng - 1) k = G->ng - 1;
  return k;
}

static int or_grid_build(or_grid* G, int64_t n, double L, const double* x, const double* y,
                         const double* z, double r_hint, int brute) {
  memset(G, 0, sizeof(*G));
  G->n = n; G->L = L; G->x = x; G->y = y; G->z = z; G->brute = brute;
  int32_t ng = 1;
  if (r_hint > 0.0) {
    double t = floor(L / r_hint);
    ng = t < 1.0 ? 1 : (t > 96.0 ? 96 : (int32_t)t);
  }
  G->ng = ng;
  G->g = L / ng;
  int64_t nc = (int64_t)ng * ng * ng;
  G->start = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
  G->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* key = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!G->start || !G->idx || !key) { free(key); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = or_grid_coord(G, x[i]) + ng * (or_grid_coord(G, y[i]) + ng * or_grid_coord(G, z[i]));
    key[i] = c;
    G->start[c + 1] += 1;
  }
  for (int64_t c = 0; c < nc; ++c) G->start[c + 1] += G->start[c];
  int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
  if (!fill) { free(key); return -2; }
  memcpy(fill, G->start, sizeof(int32_t) * (size_t)nc);
  for (int64_t i = 0; i < n; ++i) G->idx[fill[key[i]]++] = (int32_t)i;
  free(fill);
  free(key);
  return 0;
}
static void or_grid_free(or_grid* G) { free(G->start); free(G->idx); }

/* Axis range of buckets overlapping [c - R, c + R]; each bucket once. */
static void or_axis_range(const or_grid* G, double c, double R, int32_t* lo, int32_t* hi, int* all) {
  int32_t a = (int32_t)floor((c - R) / G->g);
  int32_t b = (int32_t)floor((c + R) / G->g);
  if (b - a + 1 >= G->ng) { *all = 1; *lo = 0; *hi = G->ng - 1; }
  else { *all = 0; *lo = a; *hi = b; }
}

static int or_collect(const or_grid* G, double px, double py, double pz, double R, int64_t skip,
                      or_list* out) {
  out->len = 0;
  double L = G->L;
  if (G->brute) {
    for (int64_t j = 0; j < G->n; ++j) {
      if (j == skip) continue;
      double dx = or_min_image(px - G->x[j], L);
      double dy = or_min_image(py - G->y[j], L);
      double dz = or_min_image(pz - G->z[j], L);
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r < R && or_list_push(out, (int32_t)j, dx, dy, dz, r)) return -2;
    }
    return 0;
  }
  int32_t lo[3], hi[3];
  int all[3];
  or_axis_range(G, px, R, &lo[0], &hi[0], &all[0]);
  or_axis_range(G, py, R, &lo[1], &hi[1], &all[1]);
  or_axis_range(G, pz, R, &lo[2], &hi[2], &all[2]);
  int32_t ng = G->ng;
  for (int32_t kz = lo[2]; kz <= hi[2]; ++kz) {
    int32_t cz = ((kz % ng) + ng) % ng;
    for (int32_t ky = lo[1]; ky <= hi[1]; ++ky) {
      int32_t cy = ((ky % ng) + ng) % ng;
      for (int32_t kx = lo[0]; kx <= hi[0]; ++kx) {
        int32_t cx = ((kx % ng) + ng) % ng;
        int32_t c = cx + ng * (cy + ng * cz);
        for (int32_t s = G->start[c]; s < G->start[c + 1]; ++s) {
          int32_t j = G->idx[s];
          if (j == skip) continue;
          double dx = or_min_image(px - G->x[j], L);
          double dy = or_min_image(py - G->y[j], L);
          double dz = or_min_image(pz - G->z[j], L);
          double r = sqrt(dx * dx + dy * dy + dz * dz);
          if (r < R && or_list_push(out, j, dx, dy, dz, r)) return -2;
        }
      }
    }
  }
  return 0;
}

/* --------------------------------------------------------------------------
 * Public data records (mirrored by oracle/__init__.py with ctypes).
 * -------------------------------------------------------------------------- */
typedef struct {
  int64_t n;
  double L;                     /* periodic cubic box side */
  const double *x, *y, *z;      /* positions in [0, L) */
  const double *vx, *vy, *vz;   /* velocities */
  const double *m;              /* masses */
  const double *u;              /* internal energy per unit mass */
} oracle_particles;

typedef struct {
  double gamma;        /* ratio of specific heats */
  double eta;          /* resolution parameter of eq. "partition" */
  double alpha_v;      /* viscosity constant alpha_V */
  double beta_v;       /* signal-velocity constant beta */
  double eps_balsara;  /* epsilon of eq. "balsara" */
  double h_tol;        /* relative tolerance on h of the Newton-Raphson solve */
  int32_t max_iter;    /* iteration cap of the solve */
  int32_t brute;       /* 1: O(N^2) neighbour search; 0: bucket grid */
} oracle_config;

typedef struct {      /* per target */
  double *h, *rho, *drho_dh, *n_hat, *dn_dh;
  double *div_v, *curl_x, *curl_y, *curl_z, *curl_norm;
  double *f, *P, *c, *B;
  int32_t *n_ngb;     /* neighbours with r < H_i, self included */
  int32_t *n_iter;    /* Newton-Raphson iterations used */
} oracle_density_out;

typedef struct {      /* per particle, all n: density results the force reads */
  const double *h, *rho, *f, *P, *c, *B;
} oracle_density_state;

typedef struct {      /* per target */
  double *ax, *ay, *az, *du_dt, *v_sig;
  int32_t *n_pairs;   /* j != i with r_ij < max(H_i, H_j) */
} oracle_force_out;

/* Median of the positive entries of v (for the bucket size hint only),
 * by Hoare's selection. */
static double or_median(const double* v, int64_t n) {
  if (n <= 0) return 0.0;
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  if (!t) return 0.0;
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i)
    if (v[i] > 0.0) t[k++] = v[i];
  double m = 0.0;
  if (k > 0) {
    int64_t lo = 0, hi = k - 1, want = k / 2;
    while (lo < hi) {
      double piv = t[lo + (hi - lo) / 2];
      int64_t i = lo, j = hi;
      while (i <= j) {
        while (t[i] < piv) ++i;
        while (t[j] > piv) --j;
        if (i <= j) { double x = t[i]; t[i] = t[j]; t[j] = x; ++i; --j; }
      }
      if (want <= j) hi = j;
      else if (want >= i) lo = i;
      else break;
    }
    m = t[want];
  }
  free(t);
  return m;
}

/* Number density n_hat(h) and its derivative (Sec. 3.1.1) over a candidate
 * list of distances; the self term (r = 0) is part of the list. */
static void or_nhat(const or_list* l, double h, double* n_hat, double* dn_dh) {
  double H = OR_GAMMA_K * h;
  double s = 0.0, d = 0.0;
  for (int64_t k = 0; k < l->len; ++k) {
    double r = l->r[k];
    if (r >= H) continue;
    s += or_W(r, h);
    d += or_dWdh(r, h);
  }
  *n_hat = s;
  *dn_dh = d;
}

/* Sums of the density loop for target i at smoothing length h over the list l
 * (which must hold every particle within gamma_K h, the self term included),
 * then the per-particle factors f_i, P_i, c_i and B_i (Sec. 3.1-3.2). */
static void or_density_sums(const oracle_particles* P, const oracle_config* C, int64_t i, double h,
                            const or_list* l_, oracle_density_out* out, int64_t t) {
  const or_list l = *l_;
  double H = OR_GAMMA_K * h;
  double nh = 0, dn = 0, rho = 0, drho = 0, div = 0, cx = 0, cy = 0, cz = 0;
  int32_t nngb = 0;
  for (int64_t k = 0; k < l.len; ++k) {
    double r = l.r[k];
    if (r >= H) continue;
    int32_t j = l.j[k];
    double W = or_W(r, h);
    double dWh = or_dWdh(r, h);
    nngb += 1;
    nh += W;
    dn += dWh;
    rho += P->m[j] * W;
    drho += P->m[j] * dWh;
    if (r > 0.0) {
      /* grad_i W_ij = dW/dr * x_ij / r, x_ij = x_i - x_j */
      double g = or_dWdr(r, h) / r;
      double gx = g * l.dx[k], gy = g * l.dy[k], gz = g * l.dz[k];
      double ux = P->vx[i] - P->vx[j], uy = P->vy[i] - P->vy[j], uz = P->vz[i] - P->vz[j];
      div -= P->m[j] * (ux * gx + uy * gy + uz * gz);
      cx += P->m[j] * (uy * gz - uz * gy);
      cy += P->m[j] * (uz * gx - ux * gz);
      cz += P->m[j] * (ux * gy - uy * gx);
    }
  }
  div /= rho; cx /= rho; cy /= rho; cz /= rho;
  double curl = sqrt(cx * cx + cy * cy + cz * cz);
  double fi = 1.0 / (1.0 + h / (3.0 * rho) * drho);
  double Pi = (C->gamma - 1.0) * P->u[i] * rho;
  double ci = sqrt(C->gamma * Pi / rho);
  double Bi = fabs(div) / (fabs(div) + curl + C->eps_balsara * ci / h);
  out->h[t] = h; out->rho[t] = rho; out->drho_dh[t] = drho;
  out->n_hat[t] = nh; out->dn_dh[t] = dn;
  out->div_v[t] = div; out->curl_x[t] = cx; out->curl_y[t] = cy; out->curl_z[t] = cz;
  out->curl_norm[t] = curl;
  out->f[t] = fi; out->P[t] = Pi; out->c[t] = ci; out->B[t] = Bi;
  out->n_ngb[t] = nngb;
}

/* --------------------------------------------------------------------------
 * Density loop with the smoothing-length solve (Sec. 3.1.1-3.1.2, eqs.
 * "numberdensity", "partition", "eos", "balsara").
 *
 * For each target i the smoothing length is the root of
 *     f(h) = n_hat(h) - (eta / h)^3,
 * found by Newton-Raphson with f'(h) = dn_hat/dh + 3 eta^3 / h^4 (the
 * derivative the paper prints), safeguarded by a bisection bracket, until
 * |dh| <= h_tol h.  h0 holds a starting guess for every particle.
 * -------------------------------------------------------------------------- */
int oracle_density(const oracle_particles* P, const oracle_config* C, const double* h0,
                   int64_t n_t, const int64_t* targets, oracle_density_out* out) {
  int64_t n = P->n;
  double L = P->L;
  double eta3 = C->eta * C->eta * C->eta;
  or_grid G;
  double hint = OR_GAMMA_K * or_median(h0, n);
  int err = or_grid_build(&G, n, L, P->x, P->y, P->z, hint, C->brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets ? targets[t] : t;
    double xi = P->x[i], yi = P->y[i], zi = P->z[i];
    double h = h0[i];
    double lo = 0.0, hi = INFINITY;
    double Rcap = 0.4999 * L;  /* minimum image needs the support below L/2 */
    double R = 1.25 * OR_GAMMA_K * h;
    if (R > Rcap) R = Rcap;
    err = or_collect(&G, xi, yi, zi, R, -1, &l);
    int32_t it = 0;
    for (; it < C->max_iter && !err; ++it) {
      if (OR_GAMMA_K * h > R) {
        if (OR_GAMMA_K * h >= Rcap) { err = -5; break; }   /* support would wrap the box */
        R = 1.5 * OR_GAMMA_K * h;
        if (R > Rcap) R = Rcap;
        err = or_collect(&G, xi, yi, zi, R, -1, &l);
        if (err) break;
      }
      double nh, dn;
      or_nhat(&l, h, &nh, &dn);
      double f = nh - eta3 / (h * h * h);
      double fp = dn + 3.0 * eta3 / (h * h * h * h);
      if (f < 0.0) lo = h; else hi = h;
      if (f == 0.0) break;
      /* converged when the Newton correction is below the tolerance */
      if (fp > 0.0 && fabs(f / fp) <= C->h_tol * h) { h -= f / fp; ++it; break; }
      double hn = h - f / fp;
      /* safeguards (they move the path, not the root): at most a factor of 2
       * per step, and bisection whenever the step leaves the bracket */
      if (hn > 2.0 * h) hn = 2.0 * h;
      if (hn < 0.5 * h) hn = 0.5 * h;
      if (!(fp > 0.0) || !(hn > lo) || !(hn < hi))
        hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
      double dh = fabs(hn - h);
      h = hn;
      if (dh <= C->h_tol * h) { ++it; break; }
    }
    if (err) break;
    if (it >= C->max_iter) { err = -3; break; }
    if (OR_GAMMA_K * h > R) {
      if (OR_GAMMA_K * h >= Rcap) { err = -5; break; }
      R = OR_GAMMA_K * h * 1.0001;
      if (R > Rcap) R = Rcap;
      err = or_collect(&G, xi, yi, zi, R, -1, &l);
      if (err) break;
    }
    or_density_sums(P, C, i, h, &l, out, t);
    out->n_iter[t] = it;
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}

/* Density-loop sums at a given smoothing length h[t] per target (no solve);
 * n_iter is set to 0.  Used to check derivatives with respect to h. */
int oracle_density_at(const oracle_particles* P, const oracle_config* C, const double* h_t,
                      int64_t n_t, const int64_t* targets, oracle_density_out* out) {
  int64_t n = P->n;
  double L = P->L;
  or_grid G;
  double hint = OR_GAMMA_K * or_median(h_t, n_t);
  int err = or_grid_build(&G, n, L, P->x, P->y, P->z, hint, C->brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets ? targets[t] : t;
    double R = 1.0001 * OR_GAMMA_K * h_t[t];
    if (R >= 0.5 * L) { err = -5; break; }
    err = or_collect(&G, P->x[i], P->y[i], P->z[i], R, -1, &l);
    if (err) break;
    or_density_sums(P, C, i, h_t[t], &l, out, t);
    out->n_iter[t] = 0;
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}

/* --------------------------------------------------------------------------
 * Force loop (Sec. 3.2, eqs. "densityenergy", "basicartvisc", "alpha",
 * "nuij", "balsara").  For each target i, over j != i with
 * r_ij < max(H_i, H_j), with x_ij = x_i - x_j, v_ij = v_i - v_j,
 * G_i = dW/dr(r_ij, h_i) / r_ij and G_j = dW/dr(r_ij, h_j) / r_ij:
 *   mu_ij    = min(v_ij . x_ij, 0) / r_ij
 *   vsig_ij  = c_i + c_j - beta mu_ij
 *   nu_ij    = -alpha_V (B_i + B_j)/2 mu_ij vsig_ij / ((rho_i + rho_j)/2)
 *   a_i     -= m_j [ f_i P_i/rho_i^2 G_i + f_j P_j/rho_j^2 G_j
 *                    + nu_ij/2 (f_i G_i + f_j G_j) ] x_ij
 *   du_i/dt += m_j [ f_i P_i/rho_i^2 G_i + nu_ij/4 (f_i G_i + f_j G_j) ] v_ij . x_ij
 *   vsig_i   = max_j vsig_ij
 * -------------------------------------------------------------------------- */
int oracle_force(const oracle_particles* P, const oracle_config* C, const oracle_density_state* S,
                 int64_t n_t, const int64_t* targets, oracle_force_out* out) {
  int64_t n = P->n;
  double L = P->L;
  double hmax = 0.0;
  for (int64_t j = 0; j < n; ++j) hmax = S->h[j] > hmax ? S->h[j] : hmax;
  double Hmax = OR_GAMMA_K * hmax;
  if (Hmax >= 0.5 * L) return -5;
  or_grid G;
  int err = or_grid_build(&G, n, L, P->x, P->y, P->z, OR_GAMMA_K * or_median(S->h, n), C->brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets ? targets[t] : t;
    err = or_collect(&G, P->x[i], P->y[i], P->z[i], Hmax, i, &l);
    if (err) break;
    double hi = S->h[i], Hi = OR_GAMMA_K * hi;
    double rhoi = S->rho[i], fi = S->f[i], Pi = S->P[i], ci = S->c[i], Bi = S->B[i];
    double ax = 0, ay = 0, az = 0, du = 0, vsig = 0;
    int32_t np = 0;
    for (int64_t k = 0; k < l.len; ++k) {
      int32_t j = l.j[k];
      double r = l.r[k];
      double hj = S->h[j], Hj = OR_GAMMA_K * hj;
      if (!(r < (Hi > Hj ? Hi : Hj))) continue;
      np += 1;
      double dx = l.dx[k], dy = l.dy[k], dz = l.dz[k];
      double vx = P->vx[i] - P->vx[j], vy = P->vy[i] - P->vy[j], vz = P->vz[i] - P->vz[j];
      double vdotx = vx * dx + vy * dy + vz * dz;
      double Gi = or_dWdr(r, hi) / r;
      double Gj = or_dWdr(r, hj) / r;
      double rhoj = S->rho[j], fj = S->f[j], Pj = S->P[j], cj = S->c[j], Bj = S->B[j];
      double mu = vdotx < 0.0 ? vdotx / r : 0.0;
      double vs = ci + cj - C->beta_v * mu;
      double alpha = C->alpha_v * 0.5 * (Bi + Bj);
      double nu = -alpha * mu * vs / (0.5 * (rhoi + rhoj));
      double pi_term = fi * Pi / (rhoi * rhoi) * Gi;
      double pj_term = fj * Pj / (rhoj * rhoj) * Gj;
      double visc = fi * Gi + fj * Gj;
      double s = P->m[j] * (pi_term + pj_term + 0.5 * nu * visc);
      ax -= s * dx; ay -= s * dy; az -= s * dz;
      du += P->m[j] * (pi_term + 0.25 * nu * visc) * vdotx;
      if (vs > vsig) vsig = vs;
    }
    out->ax[t] = ax; out->ay[t] = ay; out->az[t] = az;
    out->du_dt[t] = du; out->v_sig[t] = vsig;
    out->n_pairs[t] = np;
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}

/* --------------------------------------------------------------------------
 * Neighbour collection for tests: for each target, every j (j != target)
 * with minimum-image distance < R_t.  Writes up to cap indices per target
 * into nbr[t * cap + k] and the count into cnt[t] (which may exceed cap).
 * -------------------------------------------------------------------------- */
int oracle_neighbours(const oracle_particles* P, int64_t n_t, const int64_t* targets, const double* R,
                      int32_t brute, int64_t cap, int32_t* nbr, int64_t* cnt) {
  or_grid G;
  double hint = or_median(R, n_t);
  int err = or_grid_build(&G, P->n, P->L, P->x, P->y, P->z, hint, brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets[t];
    if (R[t] >= 0.5 * P->L) { err = -5; break; }
    err = or_collect(&G, P->x[i], P->y[i], P->z[i], R[t], i, &l);
    if (err) break;
    cnt[t] = l.len;
    for (int64_t k = 0; k < l.len && k < cap; ++k) nbr[t * cap + k] = l.j[k];
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}

/* --------------------------------------------------------------------------
 * One kick-drift-kick step with a single global time-step (Sec. 2.4 leapfrog,
 * Sec. 5.4 operators with a = 1), in the order:
 *   dt     = C_CFL min_i H_i / vsig_i            (from the previous force)
 *   v     += a dt/2,   u += du/dt dt/2           (first half kick)
 *   x      = wrap(x + v dt)                      (drift)
 *   v_pred = v + a dt/2, u_pred = u + du/dt dt/2 (prediction for the loops)
 *   density (h warm-started) and force on x, v_pred, u_pred
 *   v     += a_new dt/2, u += du/dt_new dt/2     (second half kick)
 * All arrays are in/out over the n particles.  The caller holds a, du/dt and
 * vsig from the previous force evaluation.
 * -------------------------------------------------------------------------- */
int oracle_step(int64_t n, double L, const oracle_config* C, double cfl,
                double* x, double* y, double* z, double* vx, double* vy, double* vz,
                const double* m, double* u, double* h,
                double* ax, double* ay, double* az, double* du_dt, double* v_sig,
                double* rho_out, double* dt_out) {
  double dt = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double cand = cfl * OR_GAMMA_K * h[i] / v_sig[i];
    if (cand < dt) dt = cand;
  }
  if (!(dt > 0.0) || isinf(dt)) return -4;
  double* vpx = (double*)malloc(sizeof(double) * n);
  double* vpy = (double*)malloc(sizeof(double) * n);
  double* vpz = (double*)malloc(sizeof(double) * n);
  double* up = (double*)malloc(sizeof(double) * n);
  int err = (!vpx || !vpy || !vpz || !up) ? -2 : 0;
  for (int64_t i = 0; i < n && !err; ++i) {
    vx[i] += 0.5 * dt * ax[i]; vy[i] += 0.5 * dt * ay[i]; vz[i] += 0.5 * dt * az[i];
    u[i] += 0.5 * dt * du_dt[i];
    x[i] = oracle_wrap(x[i] + vx[i] * dt, L);
    y[i] = oracle_wrap(y[i] + vy[i] * dt, L);
    z[i] = oracle_wrap(z[i] + vz[i] * dt, L);
    vpx[i] = vx[i] + 0.5 * dt * ax[i]; vpy[i] = vy[i] + 0.5 * dt * ay[i]; vpz[i] = vz[i] + 0.5 * dt * az[i];
    up[i] = u[i] + 0.5 * dt * du_dt[i];
  }
  double *hd = 0, *rho = 0, *drho = 0, *nh = 0, *dn = 0, *div = 0, *c3 = 0, *cn = 0, *f = 0, *Pr = 0,
         *cs = 0, *B = 0;
  int32_t *nn = 0, *ni = 0, *np = 0;
  if (!err) {
    hd = (double*)malloc(sizeof(double) * n); rho = (double*)malloc(sizeof(double) * n);
    drho = (double*)malloc(sizeof(double) * n); nh = (double*)malloc(sizeof(double) * n);
    dn = (double*)malloc(sizeof(double) * n); div = (double*)malloc(sizeof(double) * n);
    c3 = (double*)malloc(sizeof(double) * 3 * n); cn = (double*)malloc(sizeof(double) * n);
    f = (double*)malloc(sizeof(double) * n); Pr = (double*)malloc(sizeof(double) * n);
    cs = (double*)malloc(sizeof(double) * n); B = (double*)malloc(sizeof(double) * n);
    nn = (int32_t*)malloc(sizeof(int32_t) * n); ni = (int32_t*)malloc(sizeof(int32_t) * n);
    np = (int32_t*)malloc(sizeof(int32_t) * n);
    if (!hd || !rho || !drho || !nh || !dn || !div || !c3 || !cn || !f || !Pr || !cs || !B || !nn ||
        !ni || !np)
      err = -2;
  }
  if (!err) {
    oracle_particles Pp = {n, L, x, y, z, vpx, vpy, vpz, m, up};
    oracle_density_out D = {hd, rho, drho, nh, dn, div, c3, c3 + n, c3 + 2 * n, cn, f, Pr, cs, B, nn, ni};
    err = oracle_density(&Pp, C, h, n, 0, &D);
    if (!err) {
      oracle_density_state S = {hd, rho, f, Pr, cs, B};
      oracle_force_out F = {ax, ay, az, du_dt, v_sig, np};
      err = oracle_force(&Pp, C, &S, n, 0, &F);
    }
    if (!err) {
      for (int64_t i = 0; i < n; ++i) {
        h[i] = hd[i];
        if (rho_out) rho_out[i] = rho[i];
        vx[i] += 0.5 * dt * ax[i]; vy[i] += 0.5 * dt * ay[i]; vz[i] += 0.5 * dt * az[i];
        u[i] += 0.5 * dt * du_dt[i];
      }
    }
  }
  free(vpx); free(vpy); free(vpz); free(up);
  free(hd); free(rho); free(drho); free(nh); free(dn); free(div); free(c3); free(cn); free(f);
  free(Pr); free(cs); free(B); free(nn); free(ni); free(np);
  if (dt_out) *dt_out = dt;
  return err;
}

/* --------------------------------------------------------------------------
 * Friends-of-friends groups (Sec. 7.1).  Particles i and j are friends when
 * their minimum-image distance in the periodic box of side L is below the
 * linking length b:
 *   d = x_i - x_j per axis, wrapped once into [-L/2, L/2] (or_min_image),
 *   r2 = dx*dx + dy*dy + dz*dz (left to right, no contraction),  r2 < b*b.
 * Groups are the connected components of the friendship graph, found with
 * union-find: every friend pair merges the sets of its two particles.  The
 * root of a set is kept at its smallest index (the larger root is hooked
 * below the smaller), so group[i] = the smallest index of i's group.
 * Candidates: a grid of n_c = floor(L / b) cells per side (at most
 * cbrt(8 n + 216), at least 3, so cells are at least b wide and the 27
 * neighbour cells of a cell are distinct), each pair tested once from the
 * particle of smaller index.  Returns -1 when b > L/3 (fewer than 3 cells).
 * -------------------------------------------------------------------------- */
static int64_t or_find(int64_t* parent, int64_t i) {
  while (parent[i] != i) {
    parent[i] = parent[parent[i]]; /* path halving */
    i = parent[i];
  }
  return i;
}

int oracle_fof(int64_t n, const double* x, const double* y, const double* z, double L, double b,
               int32_t* group) {
  if (n < 0 || !(L > 0.0) || !(b > 0.0)) return -1;
  if (n == 0) return 0;
  int64_t n_c = (int64_t)floor(L / b);
  if (n_c < 3) return -1;
  const double lim = 8.0 * (double)n + 216.0;
  while (n_c > 3 && (double)n_c * (double)n_c * (double)n_c > lim) --n_c;
  const int64_t n_cells = n_c * n_c * n_c;
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* start = (int64_t*)calloc((size_t)n_cells + 1, sizeof(int64_t));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_cells);
  int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!key || !start || !order || !fill || !parent) {
    free(key); free(start); free(order); free(fill); free(parent);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t kx = oracle_cell_coord(x[i], L, (int32_t)n_c);
    int64_t ky = oracle_cell_coord(y[i], L, (int32_t)n_c);
    int64_t kz = oracle_cell_coord(z[i], L, (int32_t)n_c);
    key[i] = kx + n_c * (ky + n_c * kz);
    start[key[i] + 1] += 1;
    parent[i] = i;
  }
  for (int64_t c = 0; c < n_cells; ++c) start[c + 1] += start[c];
  for (int64_t c = 0; c < n_cells; ++c) fill[c] = start[c];
  for (int64_t i = 0; i < n; ++i) order[fill[key[i]]++] = i;
  const double b2 = b * b;
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = key[i];
    int64_t kx = k % n_c, ky = (k / n_c) % n_c, kz = k / (n_c * n_c);
    for (int64_t oz = -1; oz <= 1; ++oz)
      for (int64_t oy = -1; oy <= 1; ++oy)
        for (int64_t ox = -1; ox <= 1; ++ox) {
          int64_t cx = (kx + ox + n_c) % n_c, cy = (ky + oy + n_c) % n_c, cz = (kz + oz + n_c) % n_c;
          int64_t c = cx + n_c * (cy + n_c * cz);
          for (int64_t t = start[c]; t < start[c + 1]; ++t) {
            int64_t j = order[t];
            if (j <= i) continue;
            double dx = or_min_image(x[i] - x[j], L);
            double dy = or_min_image(y[i] - y[j], L);
            double dz = or_min_image(z[i] - z[j], L);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < b2)) continue;
            int64_t ri = or_find(parent, i), rj = or_find(parent, j);
            if (ri == rj) continue;
            if (ri < rj) parent[rj] = ri; else parent[ri] = rj;
          }
        }
  }
  for (int64_t i = 0; i < n; ++i) group[i] = (int32_t)or_find(parent, i);
  free(key); free(start); free(order); free(fill); free(parent);
  return 0;
}

/* --------------------------------------------------------------------------
 * SPHENIX flavour (Sec. 3.3): a time-dependent viscosity parameter per
 * particle (eqs. "sphenix_visc1" to "sphenix_visc4"), the pair viscosity
 * parameter of eq. "av_ij", and artificial conduction (eqs. "art_cond",
 * "artconddt", "condshocklimiter", "conductionlimiter").  The dissipationless
 * part and the form of the viscosity terms are those of oracle_force.
 *
 * Readings (the paper prints these equations with typos or leaves a
 * quantity undefined):
 *  - viscosity update: alpha_V relaxes from alpha_V(t) towards alpha_loc
 *    with the factor exp(-ell c_i dt / H_i), and jumps to alpha_loc when
 *    alpha_loc is larger (the printed minus sign would drive alpha negative);
 *    the rate of the divergence is (div_v - div_v_prev) / dt, zero when
 *    dt = 0; alpha_loc = 0 when S_i = 0; v_sig,i is the signal velocity of
 *    the previous force evaluation;
 *  - gradient pass (after the viscosity update), over j != i with r < H_i:
 *      lap_u_i = 2 sum_j (m_j / rho_j) (u_i - u_j) (dW/dr)(r_ij, h_i) / r_ij
 *    (the second-derivative estimate of Brookshaw 1985, which the paper
 *    uses but does not print), v_c,i = max_j v_c,ij, and
 *    alpha_V,max,i = max(alpha_V,i, max_j alpha_V,j) (updated values);
 *  - conduction update: one explicit Euler step of eq. "artconddt" over dt,
 *    the source term taken as zero when u_i <= 0, then the result limited to
 *    [alpha_c,min, alpha_c,max (1 - alpha_V,max,i / alpha_V,max)];
 *    alpha_c,max = 1 (eq. "condshocklimiter"; the second bound of 2 in the
 *    text is read as a typo), alpha_c,min = 0;
 *  - conduction term, over the force pairs (r < max(H_i, H_j), j != i):
 *      du_i/dt += alpha_c,ij v_c,ij m_j (u_i - u_j)
 *                 [f_i dW/dr(r, h_i) + f_j dW/dr(r, h_j)] / (rho_i + rho_j)
 *    i.e. the kernel gradients of eq. "art_cond" projected on x_ij / r_ij
 *    (the printed f_ij and grad_j W_ji, which would cancel, are read as
 *    f_i grad_i W(h_i) + f_j grad_i W(h_j)); v_c,ij uses rho_i + rho_j (the
 *    printed rho_j + rho_j is a typo); alpha_c,ij = 0 when P_i + P_j = 0.
 * -------------------------------------------------------------------------- */
typedef struct {
  double alpha_v_max;  /* alpha_V,max, eq. "sphenix_visc2" (2)        */
  double ell;          /* viscosity decay length, eq. "sphenix_visc1" (0.05) */
  double beta_c;       /* beta_c of eq. "artconddt" (1)                */
  double alpha_c_min;  /* alpha_c,min (0)                              */
  double alpha_c_max;  /* alpha_c,max of eq. "condshocklimiter" (1)    */
} oracle_sphenix_config;

typedef struct {      /* per target */
  double *lap_u, *v_c, *alpha_v_ngb, *alpha_c;
} oracle_sphenix_gradient_out;

/* Viscosity parameter of each of the n particles after a step dt. */
void oracle_sphenix_alpha_v(int64_t n, const oracle_sphenix_config* X, double dt, const double* h,
                            const double* c, const double* div_v, const double* div_v_prev,
                            const double* v_sig, const double* alpha_in, double* alpha_out) {
  for (int64_t i = 0; i < n; ++i) {
    double H = OR_GAMMA_K * h[i];
    double rate = dt > 0.0 ? (div_v[i] - div_v_prev[i]) / dt : 0.0;
    double S = H * H * (-rate > 0.0 ? -rate : 0.0);
    double loc = S > 0.0 ? X->alpha_v_max * S / (v_sig[i] * v_sig[i] + S) : 0.0;
    double a = alpha_in[i];
    if (loc > a)
      alpha_out[i] = loc;
    else
      alpha_out[i] = loc + (a - loc) * exp(-X->ell * c[i] * dt / H);
  }
}

/* Conduction signal speed of a pair (x_ij, v_ij . x_ij, r). */
static double or_v_cond(double vdotx, double r, double Pi, double Pj, double rhoi, double rhoj) {
  return fabs(vdotx) / r + sqrt(2.0 * fabs(Pi - Pj) / (rhoi + rhoj));
}

/* Gradient pass and conduction-parameter update for the given targets.
 * alpha_v holds the updated viscosity parameters of all n particles,
 * alpha_c_in the conduction parameters before the step. */
int oracle_sphenix_gradient(const oracle_particles* P, const oracle_config* C, const oracle_sphenix_config* X,
                            const oracle_density_state* S, const double* alpha_v, const double* alpha_c_in,
                            double dt, int64_t n_t, const int64_t* targets, oracle_sphenix_gradient_out* out) {
  int64_t n = P->n;
  double L = P->L;
  or_grid G;
  int err = or_grid_build(&G, n, L, P->x, P->y, P->z, OR_GAMMA_K * or_median(S->h, n), C->brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets ? targets[t] : t;
    double hi = S->h[i], Hi = OR_GAMMA_K * hi;
    if (Hi >= 0.5 * L) { err = -5; break; }
    err = or_collect(&G, P->x[i], P->y[i], P->z[i], Hi, i, &l);
    if (err) break;
    double lap = 0.0, vc = 0.0, avmax = alpha_v[i];
    for (int64_t k = 0; k < l.len; ++k) {
      int32_t j = l.j[k];
      double r = l.r[k];
      if (!(r > 0.0)) continue;
      double vdotx = (P->vx[i] - P->vx[j]) * l.dx[k] + (P->vy[i] - P->vy[j]) * l.dy[k] +
                     (P->vz[i] - P->vz[j]) * l.dz[k];
      lap += P->m[j] / S->rho[j] * (P->u[i] - P->u[j]) * or_dWdr(r, hi) / r;
      double v = or_v_cond(vdotx, r, S->P[i], S->P[j], S->rho[i], S->rho[j]);
      if (v > vc) vc = v;
      if (alpha_v[j] > avmax) avmax = alpha_v[j];
    }
    lap *= 2.0;
    double src = P->u[i] > 0.0 ? X->beta_c * Hi * lap / sqrt(P->u[i]) : 0.0;
    double rate = src - (alpha_c_in[i] - X->alpha_c_min) * vc / Hi;
    double a = alpha_c_in[i] + dt * rate;
    double cap = X->alpha_c_max * (1.0 - avmax / X->alpha_v_max);
    if (a > cap) a = cap;
    if (a < X->alpha_c_min) a = X->alpha_c_min;
    out->lap_u[t] = lap;
    out->v_c[t] = vc;
    out->alpha_v_ngb[t] = avmax;
    out->alpha_c[t] = a;
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}

/* Force loop of SPHENIX for the given targets: oracle_force with
 * alpha_ij = (alpha_V,i + alpha_V,j)/2 (B_i + B_j)/2 and the conduction term
 * added to du/dt (du_cond, optional, receives the conduction part alone). */
int oracle_sphenix_force(const oracle_particles* P, const oracle_config* C, const oracle_density_state* S,
                         const double* alpha_v, const double* alpha_c, int64_t n_t, const int64_t* targets,
                         oracle_force_out* out, double* du_cond) {
  int64_t n = P->n;
  double L = P->L;
  double hmax = 0.0;
  for (int64_t j = 0; j < n; ++j) hmax = S->h[j] > hmax ? S->h[j] : hmax;
  double Hmax = OR_GAMMA_K * hmax;
  if (Hmax >= 0.5 * L) return -5;
  or_grid G;
  int err = or_grid_build(&G, n, L, P->x, P->y, P->z, OR_GAMMA_K * or_median(S->h, n), C->brute);
  if (err) { or_grid_free(&G); return err; }
  or_list l = {0};
  for (int64_t t = 0; t < n_t && !err; ++t) {
    int64_t i = targets ? targets[t] : t;
    err = or_collect(&G, P->x[i], P->y[i], P->z[i], Hmax, i, &l);
    if (err) break;
    double hi = S->h[i], Hi = OR_GAMMA_K * hi;
    double rhoi = S->rho[i], fi = S->f[i], Pi = S->P[i], ci = S->c[i], Bi = S->B[i];
    double ax = 0, ay = 0, az = 0, du = 0, cond = 0, vsig = 0;
    int32_t np = 0;
    for (int64_t k = 0; k < l.len; ++k) {
      int32_t j = l.j[k];
      double r = l.r[k];
      double hj = S->h[j], Hj = OR_GAMMA_K * hj;
      if (!(r < (Hi > Hj ? Hi : Hj))) continue;
      np += 1;
      double dx = l.dx[k], dy = l.dy[k], dz = l.dz[k];
      double vx = P->vx[i] - P->vx[j], vy = P->vy[i] - P->vy[j], vz = P->vz[i] - P->vz[j];
      double vdotx = vx * dx + vy * dy + vz * dz;
      double Gi = or_dWdr(r, hi) / r;
      double Gj = or_dWdr(r, hj) / r;
      double rhoj = S->rho[j], fj = S->f[j], Pj = S->P[j], cj = S->c[j], Bj = S->B[j];
      double mu = vdotx < 0.0 ? vdotx / r : 0.0;
      double vs = ci + cj - C->beta_v * mu;
      double alpha = 0.5 * (alpha_v[i] + alpha_v[j]) * 0.5 * (Bi + Bj);
      double nu = -alpha * mu * vs / (0.5 * (rhoi + rhoj));
      double pi_term = fi * Pi / (rhoi * rhoi) * Gi;
      double pj_term = fj * Pj / (rhoj * rhoj) * Gj;
      double visc = fi * Gi + fj * Gj;
      double s = P->m[j] * (pi_term + pj_term + 0.5 * nu * visc);
      ax -= s * dx; ay -= s * dy; az -= s * dz;
      du += P->m[j] * (pi_term + 0.25 * nu * visc) * vdotx;
      double ac = Pi + Pj > 0.0 ? (Pi * alpha_c[i] + Pj * alpha_c[j]) / (Pi + Pj) : 0.0;
      double vc = or_v_cond(vdotx, r, Pi, Pj, rhoi, rhoj);
      double gsum = fi * or_dWdr(r, hi) + fj * or_dWdr(r, hj);
      cond += ac * vc * P->m[j] * (P->u[i] - P->u[j]) * gsum / (rhoi + rhoj);
      if (vs > vsig) vsig = vs;
    }
    out->ax[t] = ax; out->ay[t] = ay; out->az[t] = az;
    out->du_dt[t] = du + cond; out->v_sig[t] = vsig;
    out->n_pairs[t] = np;
    if (du_cond) du_cond[t] = cond;
  }
  or_list_free(&l);
  or_grid_free(&G);
  return err;
}
