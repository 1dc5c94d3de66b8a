/*
 * FP64 Monte-Carlo ray-tracing estimator through finite volumes (test infrastructure).
 *
 * This file is part of the CPU oracle.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg build or call it; the CUDA library shares no code
 * with it.
 *
 * It follows Section 3 of Collange, Daumas and Defour: rays are traced cell by
 * cell through isothermal homogeneous finite volumes (Fig. "Monte-Carlo
 * ray-tracing"); across a length l of a cell the transmitted power is multiplied
 * by exp(-kappa l), the Beer-Lambert first term of Eq. (I), and the power lost
 * in the cell is tallied there; the host averages the effect of the rays.  The
 * emission source is the Planck function of Eq. (planck) (second term of
 * Eq. (I)), integrated over the cell volume and the sphere of directions.
 *
 * Readings (the paper gives no sampling details):
 *  - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *    (seed_lo, seed_hi), counter = (ray_lo, ray_hi, call, enclosure);
 *  - call 0 -> emission cell c = floor(u0 * ncells / 2^32), wavenumber index
 *    j = floor(u1 * n_nu / 2^32), in-cell fractions fx, fy from u2, u3
 *    (f = (u >> 8) * 2^-24); call 1 -> fz from word 0 and the first
 *    Marsaglia (1972) pair from words 1, 2; later calls give two pairs each;
 *  - the geometry (position, direction, cell traversal after Amanatides and
 *    Woo 1987) is specified in IEEE binary32 round-to-nearest arithmetic with no
 *    contraction, so this file must be compiled with -ffp-contract=off; the
 *    physics (kappa interpolation, weights, attenuation, tallies) is binary64;
 *  - ties between axes step the lowest axis (x < y < z) and produce a
 *    zero-length visit; cold black walls absorb what reaches them ("escaped").
 *  - weight of a ray = 4 pi V kappa(nu_j, T_c) I_b(nu_j, T_c) dnu * ncells * n_nu / N.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Philox4x32-10 from its published definition ---------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---- inputs ------------------------------------------------------------- */
typedef struct {
  int32_t nx, ny, nz, pad;
  double hx, hy, hz;
  const float *T, *p, *x; /* p, x may be NULL (table's reference values) */
} og_grid;

typedef struct {
  double nu_min, dnu;
  int64_t n_nu;
  int32_t nT, pad;
  double T_min, T_max, p_ref, x_ref;
} og_spec;

typedef struct {
  const double *kappa;     /* [nT][ncol] (or [ncells][ncol] when per_cell), cm^-1 */
  int64_t ncol;
  const int64_t *col_of_j; /* [n_nu] column of each j (-1 absent), NULL = identity */
  int32_t per_cell;        /* 1: kappa holds each cell's own value at its state */
  int32_t pad;
} og_table;

enum { OG_OK = 0, OG_E_COLUMN = 1, OG_E_ARGS = 2, OG_E_NOMEM = 3 };
enum { OG_MODE_EMIT = 0, OG_MODE_BEAM = 1 };

/* CODATA 2018 */
static const double OG_H = 6.62607015e-34, OG_C = 299792458.0, OG_KB = 1.380649e-23;
static const double OG_PI = 3.14159265358979323846;

typedef struct {
  const og_grid *g;
  const og_spec *s;
  const og_table *t;
  int32_t *cell_k;
  float *cell_frac, *cell_s;
  int64_t ncells;
  float h[3];
  int fin[3];
  int n[3];
} og_ctx;

/* T-bracket and density scale per cell, specified in binary32. */
static void cell_prep(og_ctx *C) {
  const og_grid *g = C->g;
  const og_spec *s = C->s;
  float Tmin_f = (float)s->T_min;
  float dT_f = s->nT >= 2 ? (float)((s->T_max - s->T_min) / (double)(s->nT - 1)) : 1.0f;
  float den_f = (float)(s->p_ref * s->x_ref);
  float pref_f = (float)s->p_ref, xref_f = (float)s->x_ref;
  for (int64_t c = 0; c < C->ncells; ++c) {
    int k = 0;
    float frac = 0.0f;
    if (s->nT >= 2) {
      float u = (g->T[c] - Tmin_f) / dT_f;
      float fl = floorf(u);
      if (fl < 0.0f) fl = 0.0f;
      if (fl > (float)(s->nT - 2)) fl = (float)(s->nT - 2);
      k = (int)fl;
      frac = u - fl;
      if (frac < 0.0f) frac = 0.0f;
      if (frac > 1.0f) frac = 1.0f;
    }
    float sc = 1.0f;
    if (g->p || g->x) {
      float pc = g->p ? g->p[c] : pref_f;
      float xc = g->x ? g->x[c] : xref_f;
      float num = pc * xc;
      sc = num / den_f;
    }
    C->cell_k[c] = k;
    C->cell_frac[c] = frac;
    C->cell_s[c] = sc;
  }
}

/* kappa of cell c at table column col [cm^-1]: linear in T between nodes times
 * the density scale; or, for a per-cell table (kappa evaluated by the caller at
 * each cell's own T, p, x), the cell's own row as given. */
static double cell_kappa(const og_ctx *C, int64_t c, int64_t col) {
  const double *K = C->t->kappa;
  int64_t nc = C->t->ncol;
  if (C->t->per_cell) return K[c * nc + col];
  int k = C->cell_k[c];
  double fr = (double)C->cell_frac[c];
  double v;
  if (C->s->nT >= 2)
    v = (1.0 - fr) * K[(int64_t)k * nc + col] + fr * K[(int64_t)(k + 1) * nc + col];
  else
    v = K[col];
  return (double)C->cell_s[c] * v;
}

static double planck(double nu_cm, double T) {
  double nu = 100.0 * nu_cm;
  double c2 = OG_H * OG_C / OG_KB;
  return 2.0 * OG_H * OG_C * OG_C * nu * nu * nu / expm1(c2 * nu / T);
}

static inline float u24(uint32_t u) { return (float)(u >> 8) * 0x1p-24f; }

typedef struct {
  int32_t ix[3];
  float pos[3], dir[3];
  int64_t j;
  double w;
} og_ray;

#define OG_MAX_PHILOX_CALLS 64

/* Isotropic direction by Marsaglia's method from one pair of words. */
static int marsaglia(uint32_t ua, uint32_t ub, float dir[3]) {
  float a = 2.0f * u24(ua) - 1.0f;
  float b = 2.0f * u24(ub) - 1.0f;
  float aa = a * a;
  float bb = b * b;
  float s = aa + bb;
  if (s >= 1.0f || s == 0.0f) return 0;
  float q = sqrtf(1.0f - s);
  dir[0] = (2.0f * a) * q;
  dir[1] = (2.0f * b) * q;
  dir[2] = 1.0f - 2.0f * s;
  return 1;
}

static int sample_ray(const og_ctx *C, uint64_t seed, uint32_t encl, uint64_t r,
                      uint64_t n_total, int mode, og_ray *R) {
  const og_grid *g = C->g;
  const og_spec *s = C->s;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(r >> 32), 0u, encl};
  uint32_t v[4];
  int64_t c;
  float f[3];
  if (mode == OG_MODE_BEAM) {
    R->j = (int64_t)(r % (uint64_t)s->n_nu);
    R->ix[0] = 0; R->ix[1] = g->ny / 2; R->ix[2] = g->nz / 2;
    R->pos[0] = 0.0f;
    for (int a = 1; a < 3; ++a)
      R->pos[a] = C->fin[a] ? ((float)R->ix[a] + 0.5f) * C->h[a] : 0.0f;
    R->dir[0] = 1.0f; R->dir[1] = 0.0f; R->dir[2] = 0.0f;
    R->w = 1.0;
    return OG_OK;
  }
  oracle_philox(ctr, key, v);
  c = (int64_t)(((uint64_t)v[0] * (uint64_t)C->ncells) >> 32);
  R->j = (int64_t)(((uint64_t)v[1] * (uint64_t)s->n_nu) >> 32);
  f[0] = u24(v[2]);
  f[1] = u24(v[3]);
  ctr[2] = 1u;
  oracle_philox(ctr, key, v);
  f[2] = u24(v[0]);
  int ok = marsaglia(v[1], v[2], R->dir);
  for (uint32_t call = 2; !ok && call < OG_MAX_PHILOX_CALLS; ++call) {
    ctr[2] = call;
    oracle_philox(ctr, key, v);
    ok = marsaglia(v[0], v[1], R->dir);
    if (!ok) ok = marsaglia(v[2], v[3], R->dir);
  }
  if (!ok) { R->dir[0] = 0.0f; R->dir[1] = 0.0f; R->dir[2] = 1.0f; }
  R->ix[0] = (int32_t)(c % g->nx);
  R->ix[1] = (int32_t)((c / g->nx) % g->ny);
  R->ix[2] = (int32_t)(c / ((int64_t)g->nx * g->ny));
  for (int a = 0; a < 3; ++a)
    R->pos[a] = C->fin[a] ? ((float)R->ix[a] + f[a]) * C->h[a] : 0.0f;
  /* emission weight, binary64 */
  int64_t col = C->t->col_of_j ? C->t->col_of_j[R->j] : R->j;
  if (col < 0 || col >= C->t->ncol) return OG_E_COLUMN;
  double kap = cell_kappa(C, c, col);
  double T = (double)g->T[c];
  double nu = s->nu_min + (double)R->j * s->dnu;
  double V = 1.0;
  if (C->fin[0]) V *= g->hx;
  if (C->fin[1]) V *= g->hy;
  if (C->fin[2]) V *= g->hz;
  double scale = (double)C->ncells * (double)s->n_nu / (double)n_total;
  R->w = 4.0 * OG_PI * V * (100.0 * kap) * planck(nu, T) * (100.0 * s->dnu) * scale;
  return OG_OK;
}

typedef struct {
  int64_t n_rec;
  int32_t max_vis;
  int32_t *cells;
  float *ds;
  int32_t *nvis;
} og_rec;

/* Walk one ray to a wall; deposit into absorbed[]; return the escaped power. */
static int walk(const og_ctx *C, const og_ray *R, int tau_cut, double *absorbed,
                uint64_t *steps, int64_t rec_row, const og_rec *rec, double *escaped) {
  int64_t col = C->t->col_of_j ? C->t->col_of_j[R->j] : R->j;
  if (col < 0 || col >= C->t->ncol) return OG_E_COLUMN;
  int i[3] = {R->ix[0], R->ix[1], R->ix[2]};
  int step[3];
  float invd[3], tmax[3];
  for (int a = 0; a < 3; ++a) {
    if (!C->fin[a] || R->dir[a] == 0.0f) {
      step[a] = 0; invd[a] = 0.0f; tmax[a] = INFINITY;
    } else {
      step[a] = R->dir[a] > 0.0f ? 1 : -1;
      invd[a] = 1.0f / R->dir[a];
      float plane = (float)(i[a] + (step[a] > 0 ? 1 : 0)) * C->h[a];
      tmax[a] = (plane - R->pos[a]) * invd[a];
    }
  }
  float t = 0.0f;
  double tau = 0.0;
  int nv = 0;
  int64_t nx = C->n[0], nxy = (int64_t)C->n[0] * C->n[1];
  for (;;) {
    int a = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
    float tn = tmax[a];
    float ds = tn - t;
    int64_t cell = i[0] + nx * i[1] + nxy * i[2];
    double kap = cell_kappa(C, cell, col);
    double opt = kap > 0.0 ? kap * 100.0 * (double)ds : 0.0;
    double dep = R->w * exp(-tau) * (-expm1(-opt));
    absorbed[cell] += dep;
    tau += opt;
    if (rec && rec_row >= 0) {
      if (nv < rec->max_vis) {
        rec->cells[rec_row * rec->max_vis + nv] = (int32_t)cell;
        rec->ds[rec_row * rec->max_vis + nv] = ds;
      }
    }
    ++nv;
    if (tn == INFINITY) break;          /* never reaches a wall */
    if (tau_cut && tau > 100.0) break;  /* optional cut: lost fraction < 4e-44 */
    t = tn;
    i[a] += step[a];
    if (i[a] < 0 || i[a] >= C->n[a]) break;
    float plane = (float)(i[a] + (step[a] > 0 ? 1 : 0)) * C->h[a];
    tmax[a] = (plane - R->pos[a]) * invd[a];
  }
  if (rec && rec_row >= 0) rec->nvis[rec_row] = nv;
  *steps += (uint64_t)nv;
  *escaped = R->w * exp(-tau);
  return OG_OK;
}

static int ctx_init(og_ctx *C, const og_grid *g, const og_spec *s, const og_table *t) {
  memset(C, 0, sizeof(*C));
  C->g = g; C->s = s; C->t = t;
  C->ncells = (int64_t)g->nx * g->ny * g->nz;
  double hh[3] = {g->hx, g->hy, g->hz};
  int nn[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a) {
    C->fin[a] = isfinite(hh[a]) ? 1 : 0;
    C->h[a] = (float)hh[a];
    C->n[a] = nn[a];
  }
  C->cell_k = (int32_t *)malloc(sizeof(int32_t) * C->ncells);
  C->cell_frac = (float *)malloc(sizeof(float) * C->ncells);
  C->cell_s = (float *)malloc(sizeof(float) * C->ncells);
  if (!C->cell_k || !C->cell_frac || !C->cell_s) return OG_E_NOMEM;
  cell_prep(C);
  return OG_OK;
}

static void ctx_free(og_ctx *C) {
  free(C->cell_k); free(C->cell_frac); free(C->cell_s);
}

typedef struct {
  const og_ctx *C;
  uint64_t seed, r0, r1, n_total, ray_begin;
  uint32_t encl;
  int mode, tau_cut;
  double *absorbed;
  double emitted, escaped;
  uint64_t steps;
  const og_rec *rec;
  double *rec_esc, *rec_w;
  int err;
} og_job;

static void *run_job(void *arg) {
  og_job *J = (og_job *)arg;
  og_ray R;
  for (uint64_t r = J->r0; r < J->r1; ++r) {
    int e = sample_ray(J->C, J->seed, J->encl, r, J->n_total, J->mode, &R);
    if (e) { J->err = e; return NULL; }
    int64_t row = -1;
    if (J->rec && (int64_t)(r - J->ray_begin) < J->rec->n_rec) row = (int64_t)(r - J->ray_begin);
    double esc = 0.0;
    e = walk(J->C, &R, J->tau_cut, J->absorbed, &J->steps, row, J->rec, &esc);
    if (e) { J->err = e; return NULL; }
    J->emitted += R.w;
    J->escaped += esc;
    if (row >= 0) {
      if (J->rec_esc) J->rec_esc[row] = esc;
      if (J->rec_w) J->rec_w[row] = R.w;
    }
  }
  return NULL;
}

/* Trace rays [ray_begin, ray_begin + n_rays) of an N = n_total estimate.
 * absorbed[ncells] and scalars[3] (emitted, absorbed, escaped) are ACCUMULATED. */
int oracle_trace(const og_grid *g, const og_spec *s, const og_table *t, uint64_t seed,
                 uint32_t encl, uint64_t ray_begin, uint64_t n_rays, uint64_t n_total,
                 int mode, int tau_cut, int nthreads, double *absorbed, double *scalars,
                 uint64_t *steps, int64_t n_rec, int32_t max_vis, int32_t *rec_cells,
                 float *rec_ds, int32_t *rec_n, double *rec_esc, double *rec_w) {
  if (!g || !s || !t || !absorbed || !scalars || n_total == 0) return OG_E_ARGS;
  og_ctx C;
  int e = ctx_init(&C, g, s, t);
  if (e) { ctx_free(&C); return e; }
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > n_rays) nthreads = n_rays > 0 ? (int)n_rays : 1;
  og_rec rec = {n_rec, max_vis, rec_cells, rec_ds, rec_n};
  og_job *jobs = (og_job *)calloc((size_t)nthreads, sizeof(og_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); ctx_free(&C); return OG_E_NOMEM; }
  for (int k = 0; k < nthreads; ++k) {
    og_job *J = &jobs[k];
    J->C = &C; J->seed = seed; J->encl = encl; J->mode = mode; J->tau_cut = tau_cut;
    J->n_total = n_total; J->ray_begin = ray_begin;
    J->r0 = ray_begin + n_rays * (uint64_t)k / (uint64_t)nthreads;
    J->r1 = ray_begin + n_rays * (uint64_t)(k + 1) / (uint64_t)nthreads;
    J->absorbed = (double *)calloc((size_t)C.ncells, sizeof(double));
    J->rec = (n_rec > 0 && rec_cells) ? &rec : NULL;
    J->rec_esc = rec_esc; J->rec_w = rec_w;
    if (!J->absorbed) { e = OG_E_NOMEM; }
  }
  if (!e) {
    for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, run_job, &jobs[k]);
    run_job(&jobs[0]);
    for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
    for (int k = 0; k < nthreads; ++k) {
      if (jobs[k].err) e = jobs[k].err;
      for (int64_t c = 0; c < C.ncells; ++c) absorbed[c] += jobs[k].absorbed[c];
      scalars[0] += jobs[k].emitted;
      scalars[2] += jobs[k].escaped;
      if (steps) *steps += jobs[k].steps;
    }
    double tot = 0.0;
    for (int k = 0; k < nthreads; ++k)
      for (int64_t c = 0; c < C.ncells; ++c) tot += jobs[k].absorbed[c];
    scalars[1] += tot;
  }
  for (int k = 0; k < nthreads; ++k) free(jobs[k].absorbed);
  free(jobs); free(th);
  ctx_free(&C);
  return e;
}

/* Sample rays only: cell (flat), j, position, direction and weight. */
int oracle_sample_rays(const og_grid *g, const og_spec *s, const og_table *t, uint64_t seed,
                       uint32_t encl, uint64_t ray_begin, uint64_t n, uint64_t n_total, int mode,
                       int64_t *cell, int64_t *j, float *pos, float *dir, double *w) {
  og_ctx C;
  int e = ctx_init(&C, g, s, t);
  if (e) { ctx_free(&C); return e; }
  og_ray R;
  for (uint64_t k = 0; k < n && !e; ++k) {
    e = sample_ray(&C, seed, encl, ray_begin + k, n_total, mode, &R);
    cell[k] = R.ix[0] + (int64_t)g->nx * (R.ix[1] + (int64_t)g->ny * R.ix[2]);
    j[k] = R.j;
    for (int a = 0; a < 3; ++a) { pos[3 * k + a] = R.pos[a]; dir[3 * k + a] = R.dir[a]; }
    if (w) w[k] = R.w;
  }
  ctx_free(&C);
  return e;
}

/* Only the emission indices (cell, j) of rays: no table needed. */
void oracle_emission_indices(int64_t ncells, int64_t n_nu, uint64_t seed, uint32_t encl,
                             uint64_t ray_begin, uint64_t n, int64_t *cell, int64_t *j) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint64_t k = 0; k < n; ++k) {
    uint64_t r = ray_begin + k;
    uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(r >> 32), 0u, encl}, v[4];
    oracle_philox(ctr, key, v);
    cell[k] = (int64_t)(((uint64_t)v[0] * (uint64_t)ncells) >> 32);
    j[k] = (int64_t)(((uint64_t)v[1] * (uint64_t)n_nu) >> 32);
  }
}

/* Walk explicitly given rays (brute-force quadrature of the estimator). */
int oracle_walk_rays(const og_grid *g, const og_spec *s, const og_table *t, int64_t n,
                     const int32_t *ix3, const float *pos, const float *dir, const int64_t *j,
                     const double *w, double *absorbed, double *escaped) {
  og_ctx C;
  int e = ctx_init(&C, g, s, t);
  if (e) { ctx_free(&C); return e; }
  uint64_t steps = 0;
  og_ray R;
  for (int64_t k = 0; k < n && !e; ++k) {
    for (int a = 0; a < 3; ++a) {
      R.ix[a] = ix3[3 * k + a]; R.pos[a] = pos[3 * k + a]; R.dir[a] = dir[3 * k + a];
    }
    R.j = j[k];
    R.w = w[k];
    double esc = 0.0;
    e = walk(&C, &R, 0, absorbed, &steps, -1, NULL, &esc);
    escaped[k] = esc;
  }
  ctx_free(&C);
  return e;
}

/* Cell T bracket and density scale (for tests). */
int oracle_cell_prep(const og_grid *g, const og_spec *s, int32_t *k, float *frac, float *sc) {
  og_table t = {NULL, 0, NULL, 0, 0};
  og_ctx C;
  int e = ctx_init(&C, g, s, &t);
  if (!e) {
    memcpy(k, C.cell_k, sizeof(int32_t) * C.ncells);
    memcpy(frac, C.cell_frac, sizeof(float) * C.ncells);
    memcpy(sc, C.cell_s, sizeof(float) * C.ncells);
  }
  ctx_free(&C);
  return e;
}


/* ---- Spectrally resolved marching of Eq. (I) along given rays -------------
 * For each ray (start position inside the grid, direction) and each spectral
 * sample nu_j, the intensity entering with I_in(nu_j) crosses the cells of the
 * same binary32 walk; across a cell of length l:
 *   I <- I exp(-kappa l) + I_b(nu_j, T_cell) (1 - exp(-kappa l))      (Eq. I)
 * with kappa the cell's table value (cm^-1, times 100 per m).  I_out is the
 * intensity leaving the grid; power[r] = sum_j (I_in - I_out) dnu (m^-1), the
 * reduction of Section 3.  Binary64 physics.                                  */
int oracle_march(const og_grid *g, const og_spec *s, const og_table *t, int64_t n,
                 const float *pos, const float *dir, const double *I_in, double *I_out,
                 double *power) {
  og_ctx C;
  int e = ctx_init(&C, g, s, t);
  if (e) { ctx_free(&C); return e; }
  int maxv = g->nx + g->ny + g->nz + 4;
  int64_t *cells = (int64_t *)malloc(sizeof(int64_t) * (size_t)maxv);
  double *len = (double *)malloc(sizeof(double) * (size_t)maxv);
  if (!cells || !len) { free(cells); free(len); ctx_free(&C); return OG_E_NOMEM; }
  int64_t nx = C.n[0], nxy = (int64_t)C.n[0] * C.n[1];
  for (int64_t r = 0; r < n && !e; ++r) {
    int i[3], step[3];
    float invd[3], tmax[3], p[3], d[3];
    for (int a = 0; a < 3; ++a) {
      p[a] = pos[3 * r + a];
      d[a] = dir[3 * r + a];
      i[a] = C.fin[a] ? (int)floorf(p[a] / C.h[a]) : 0;
      if (i[a] < 0) i[a] = 0;
      if (i[a] >= C.n[a]) i[a] = C.n[a] - 1;
      if (!C.fin[a] || d[a] == 0.0f) {
        step[a] = 0; invd[a] = 0.0f; tmax[a] = INFINITY;
      } else {
        step[a] = d[a] > 0.0f ? 1 : -1;
        invd[a] = 1.0f / d[a];
        float plane = (float)(i[a] + (step[a] > 0 ? 1 : 0)) * C.h[a];
        tmax[a] = (plane - p[a]) * invd[a];
      }
    }
    int nv = 0;
    float tt = 0.0f;
    for (;;) {
      int a = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
      float tn = tmax[a];
      if (nv >= maxv) { e = OG_E_ARGS; break; }
      cells[nv] = i[0] + nx * i[1] + nxy * i[2];
      len[nv] = (double)(tn - tt);
      ++nv;
      if (tn == INFINITY) break;
      tt = tn;
      i[a] += step[a];
      if (i[a] < 0 || i[a] >= C.n[a]) break;
      float plane = (float)(i[a] + (step[a] > 0 ? 1 : 0)) * C.h[a];
      tmax[a] = (plane - p[a]) * invd[a];
    }
    double pw = 0.0;
    for (int64_t j = 0; j < s->n_nu && !e; ++j) {
      int64_t col = C.t->col_of_j ? C.t->col_of_j[j] : j;
      if (col < 0 || col >= C.t->ncol) { e = OG_E_COLUMN; break; }
      double nu = s->nu_min + (double)j * s->dnu;
      double I0 = I_in ? I_in[j] : 0.0, I = I0;
      for (int v = 0; v < nv; ++v) {
        double kap = cell_kappa(&C, cells[v], col);
        double a = kap > 0.0 ? kap * 100.0 * len[v] : 0.0;
        double Ib = planck(nu, (double)g->T[cells[v]]);
        double att = -expm1(-a);               /* 1 - exp(-a) */
        I = I * (1.0 - att) + Ib * att;
      }
      if (I_out) I_out[r * s->n_nu + j] = I;
      pw += (I0 - I) * (100.0 * s->dnu);
    }
    if (power) power[r] = pw;
  }
  free(cells); free(len); ctx_free(&C);
  return e;
}
