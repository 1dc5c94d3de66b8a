// Ray state, Philox ray sampling and one walk step, shared by the table walk,
// the on-the-fly line-by-line walk and the surrogate-network walk, so that all
// three trace the same rays (Section 3, Fig. ray; Eq. I first term).
#pragma once

#include "rt_common.cuh"

namespace rt {

struct CellParams {
  long long ncells;
  float Tmin, dT, den, pref, xref;
  int nT, has_px;
};

// Cell c's temperature bracket in the table (binary32: u = (T - T_min) / dT,
// k = clamp(floor u, 0, nT - 2), frac = clamp(u - k, 0, 1)), density scale
// (p x) / (p_ref x_ref) and T, packed as {frac, scale, T, k bits}.
__device__ __forceinline__ float4 cell_prep_one(const float *__restrict__ T, const float *__restrict__ p,
                                                const float *__restrict__ x, long long c,
                                                const CellParams &C, uint32_t *status) {
  const float Tc = T[c];
  int k = 0;
  float frac = 0.0f;
  if (!(Tc > 0.0f) || !isfinite(Tc)) status_or(status, RT_DEV_NONFINITE);
  if (C.nT >= 2) {
    const float u = __fdiv_rn(__fsub_rn(Tc, C.Tmin), C.dT);
    float fl = floorf(u);
    fl = fminf(fmaxf(fl, 0.0f), (float)(C.nT - 2));
    k = (int)fl;
    frac = fminf(fmaxf(__fsub_rn(u, fl), 0.0f), 1.0f);
  }
  float sc = 1.0f;
  if (C.has_px) {
    const float pc = p ? p[c] : C.pref;
    const float xc = x ? x[c] : C.xref;
    if (!(pc > 0.0f) || !isfinite(pc) || !(xc > 0.0f) || !isfinite(xc))
      status_or(status, RT_DEV_NONFINITE);
    sc = __fdiv_rn(__fmul_rn(pc, xc), C.den);
  }
  return make_float4(frac, sc, Tc, __int_as_float(k));
}

struct WalkParams {
  int n[3];
  int fin[3];
  float h[3];
  long long ncells, n_nu;
  int nT, mode, tau_cut, step_cap;
  int nu_major;  // walk table layout: 0 T-major, 1 wavenumber-major, 2 wavenumber-major node pairs
  unsigned long long ray_begin, n_rays;
  uint32_t seed_lo, seed_hi, enclosure;
  float nu_min, dnu;
  float w_scale;  // 4 pi V * 100 * (100 dnu) * ncells n_nu / N   [per (cm^-1 kappa) (I_b)]
  // Planck, wavenumber form, nu in m^-1
  float two_hc2, c2_m;
  // record
  long long rec_n;
  int rec_max;
};

struct RecordPtrs {
  int32_t *cells;
  float *ds;
  int32_t *nvis;
  float *weight, *escaped;
};

__device__ __forceinline__ float u24(uint32_t u) { return __fmul_rn(__uint2float_rn(u >> 8), 0x1p-24f); }

__device__ __forceinline__ bool marsaglia(uint32_t ua, uint32_t ub, float &dx, float &dy, float &dz) {
  const float a = __fsub_rn(__fmul_rn(2.0f, u24(ua)), 1.0f);
  const float b = __fsub_rn(__fmul_rn(2.0f, u24(ub)), 1.0f);
  const float s = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
  if (s >= 1.0f || s == 0.0f) return false;
  const float q = __fsqrt_rn(__fsub_rn(1.0f, s));
  dx = __fmul_rn(__fmul_rn(2.0f, a), q);
  dy = __fmul_rn(__fmul_rn(2.0f, b), q);
  dz = __fsub_rn(1.0f, __fmul_rn(2.0f, s));
  return true;
}

// kappa of a cell from the table, linear in T between its bracketing nodes, times
// the density scale.  T-major table: tab[k * n_nu + j].
__device__ __forceinline__ float cell_kappa(const float4 cd, const float *__restrict__ tab,
                                            long long n_nu, int nT, long long j) {
  const int k = __float_as_int(cd.w);
  const float v0 = __ldg(tab + (long long)k * n_nu + j);
  if (nT < 2) return cd.y * v0;
  const float v1 = __ldg(tab + (long long)(k + 1) * n_nu + j);
  return cd.y * fmaf(cd.x, v1, (1.0f - cd.x) * v0);
}

// The same from a wavenumber-major copy tabt[j * nT + k]: both nodes share a cache line.
__device__ __forceinline__ float cell_kappa_t(const float4 cd, const float *__restrict__ tabt, int nT,
                                              long long j) {
  const int k = __float_as_int(cd.w);
  const float *c = tabt + j * (long long)nT + k;
  const float v0 = __ldg(c);
  if (nT < 2) return cd.y * v0;
  const float v1 = __ldg(c + 1);
  return cd.y * fmaf(cd.x, v1, (1.0f - cd.x) * v0);
}

// The same from node pairs tabp[j * (nT - 1) + k] = {kappa_k, kappa_k+1}: one 8-byte load.
__device__ __forceinline__ float cell_kappa_p(const float4 cd, const float *__restrict__ tabp, int nT,
                                              long long j) {
  const int k = __float_as_int(cd.w);
  const float2 v = __ldg(reinterpret_cast<const float2 *>(tabp) + j * (long long)(nT - 1) + k);
  return cd.y * fmaf(cd.x, v.y, (1.0f - cd.x) * v.x);
}

// The same from the ray's row of node pairs, row = tabp + j (nT - 1).
__device__ __forceinline__ float cell_kappa_row(const float4 cd, const float2 *__restrict__ row) {
  const float2 v = __ldg(row + __float_as_int(cd.w));
  return cd.y * fmaf(cd.x, v.y, (1.0f - cd.x) * v.x);
}

// The same from the ray's row of a wavenumber-major table, row = tabt + j nT.
__device__ __forceinline__ float cell_kappa_row1(const float4 cd, const float *__restrict__ row, int nT) {
  const float *c = row + __float_as_int(cd.w);
  const float v0 = __ldg(c);
  if (nT < 2) return cd.y * v0;
  return cd.y * fmaf(cd.x, __ldg(c + 1), (1.0f - cd.x) * v0);
}

// kappa of a cell from the walk table in layout L (0 T-major, 1 wavenumber-major, 2 pairs).
template <int L>
__device__ __forceinline__ float cell_kappa_l(const float4 cd, const float *__restrict__ tab, int nT,
                                              long long n_nu, long long j) {
  if (L == 2) return cell_kappa_p(cd, tab, nT, j);
  if (L == 1) return cell_kappa_t(cd, tab, nT, j);
  return cell_kappa(cd, tab, n_nu, nT, j);
}

__device__ __forceinline__ float tmax_of(int i, int step, float h, float pos, float invd) {
  const float plane = __fmul_rn((float)(i + (step > 0 ? 1 : 0)), h);
  return __fmul_rn(__fsub_rn(plane, pos), invd);
}

// Emission weight 4 pi V kappa I_b(nu_j, T) dnu * ncells n_nu / N (Eq. planck,
// wavenumber form), kappa of the emitting cell in cm^-1.
__device__ __forceinline__ float emission_weight(const WalkParams &W, int j, float T, float kap) {
  const float nu_m = 100.0f * fmaf((float)j, W.dnu, W.nu_min);
  const float ib = W.two_hc2 * nu_m * nu_m * nu_m / expm1f(W.c2_m * nu_m / T);
  return W.w_scale * kap * ib;
}

// State of one ray between walk steps (registers of its lane).
// The step direction of an axis is the sign of its inverse direction cosine
// (an axis with a zero cosine, or unbounded, has tmax = inf and is never stepped).
struct Ray {
  int ix, iy, iz, cell, j, nv, row;
  float px, py, pz, ivx, ivy, ivz, tx, ty, tz, t, tau, tc, trans, w;
};

// Philox draws -> emission cell, wavenumber, position, direction, weight; DDA set-up.
// *cd_out (if given; walks with a table) receives the data of the first cell.
__device__ __forceinline__ void ray_init(const WalkParams &W, const float4 *__restrict__ cells,
                                         const float *__restrict__ tab, unsigned long long rr,
                                         bool record, Ray &R, float4 *cd_out = nullptr) {
  const unsigned long long r = W.ray_begin + rr;
  const long long nxy = (long long)W.n[0] * W.n[1];
  float dx, dy, dz;
  if (W.mode == RT_SRC_BEAM) {
    R.j = (int)(r % (unsigned long long)W.n_nu);
    R.ix = 0; R.iy = W.n[1] / 2; R.iz = W.n[2] / 2;
    R.px = 0.0f;
    R.py = W.fin[1] ? __fmul_rn(__fadd_rn((float)R.iy, 0.5f), W.h[1]) : 0.0f;
    R.pz = W.fin[2] ? __fmul_rn(__fadd_rn((float)R.iz, 0.5f), W.h[2]) : 0.0f;
    dx = 1.0f; dy = 0.0f; dz = 0.0f;
    R.w = 1.0f;
  } else {
    u32x4 ctr{(uint32_t)r, (uint32_t)(r >> 32), 0u, W.enclosure};
    u32x4 v = philox4x32_10(ctr, W.seed_lo, W.seed_hi);
    const long long c = (long long)(((unsigned long long)v.x * (unsigned long long)W.ncells) >> 32);
    R.j = (int)(((unsigned long long)v.y * (unsigned long long)W.n_nu) >> 32);
    const float fx = u24(v.z), fy = u24(v.w);
    ctr.z = 1u;
    v = philox4x32_10(ctr, W.seed_lo, W.seed_hi);
    const float fz = u24(v.x);
    bool ok = marsaglia(v.y, v.z, dx, dy, dz);
    for (uint32_t call = 2; !ok && call < 64u; ++call) {
      ctr.z = call;
      v = philox4x32_10(ctr, W.seed_lo, W.seed_hi);
      ok = marsaglia(v.x, v.y, dx, dy, dz);
      if (!ok) ok = marsaglia(v.z, v.w, dx, dy, dz);
    }
    if (!ok) { dx = 0.0f; dy = 0.0f; dz = 1.0f; }
    // cell index -> (ix, iy, iz) in 32-bit unsigned arithmetic (c < ncells < 2^31)
    const uint32_t cu = (uint32_t)c, n0 = (uint32_t)W.n[0], n1 = (uint32_t)W.n[1];
    const uint32_t q0 = cu / n0, q1 = q0 / n1;
    R.ix = (int)(cu - q0 * n0);
    R.iy = (int)(q0 - q1 * n1);
    R.iz = (int)q1;
    R.px = W.fin[0] ? __fmul_rn(__fadd_rn((float)R.ix, fx), W.h[0]) : 0.0f;
    R.py = W.fin[1] ? __fmul_rn(__fadd_rn((float)R.iy, fy), W.h[1]) : 0.0f;
    R.pz = W.fin[2] ? __fmul_rn(__fadd_rn((float)R.iz, fz), W.h[2]) : 0.0f;
    // emission weight from the table; walks without a table set it at their first step
    if (tab) {
      const float4 cd = cells[c];
      const float ke = W.nu_major == 2 ? cell_kappa_p(cd, tab, W.nT, R.j)
                       : (W.nu_major == 1 ? cell_kappa_t(cd, tab, W.nT, R.j)
                                          : cell_kappa(cd, tab, W.n_nu, W.nT, R.j));
      R.w = emission_weight(W, R.j, cd.z, ke);
      if (cd_out) *cd_out = cd;
    } else {
      R.w = -1.0f;
    }
  }
  R.ivx = R.ivy = R.ivz = 0.0f;
  R.tx = R.ty = R.tz = INFINITY;
  if (W.fin[0] && dx != 0.0f) { R.ivx = __fdiv_rn(1.0f, dx); R.tx = tmax_of(R.ix, dx > 0.0f ? 1 : -1, W.h[0], R.px, R.ivx); }
  if (W.fin[1] && dy != 0.0f) { R.ivy = __fdiv_rn(1.0f, dy); R.ty = tmax_of(R.iy, dy > 0.0f ? 1 : -1, W.h[1], R.py, R.ivy); }
  if (W.fin[2] && dz != 0.0f) { R.ivz = __fdiv_rn(1.0f, dz); R.tz = tmax_of(R.iz, dz > 0.0f ? 1 : -1, W.h[2], R.pz, R.ivz); }
  R.cell = (int)(R.ix + (long long)W.n[0] * R.iy + nxy * R.iz);
  if (cd_out && W.mode == RT_SRC_BEAM) *cd_out = cells[R.cell];
  R.row = (record && rr < (unsigned long long)W.rec_n) ? (int)rr : -1;
  R.t = 0.0f; R.tau = 0.0f; R.tc = 0.0f; R.trans = 1.0f;
  R.nv = 0;
}

// The wavenumber index of ray rr: the draw ray_init makes (Philox call 0, word 1),
// for grouping rays by wavenumber before a walk.
__device__ __forceinline__ int ray_nu_index(const WalkParams &W, unsigned long long rr) {
  const unsigned long long r = W.ray_begin + rr;
  const u32x4 v = philox4x32_10(u32x4{(uint32_t)r, (uint32_t)(r >> 32), 0u, W.enclosure}, W.seed_lo, W.seed_hi);
  return (int)(((unsigned long long)v.y * (unsigned long long)W.n_nu) >> 32);
}

// 1 - exp(-a) for a >= 0: below 1/4 its Taylor series to a^6 (truncation
// < a^7/5040, relative 5e-8 of the result), above it 1 - exp(-a) with the
// hardware exponential (relative error < 1.2e-6 at a = 1/4, falling with a).
__device__ __forceinline__ float one_minus_exp_neg(float a) {
  float p = __fmaf_rn(a, -1.0f / 720.0f, 1.0f / 120.0f);
  p = __fmaf_rn(a, p, -1.0f / 24.0f);
  p = __fmaf_rn(a, p, 1.0f / 6.0f);
  p = __fmaf_rn(a, p, -0.5f);
  p = __fmaf_rn(a, p, 1.0f);
  return a < 0.25f ? a * p : 1.0f - __expf(-a);
}

struct NoPrefetch {
  __device__ __forceinline__ void operator()(int) const {}
};

// One visit: deposit in the current cell (Eq. I, first term), advance to the next.
// Returns true when the ray has left the grid (or can never reach a wall).
// The next cell is found first and handed to pf (a walk may start loading its
// data) before the deposit arithmetic; the visit sequence is that of the
// binary32 DDA (nearest face, ties to the lowest axis, face distance
// recomputed from the start point).
// EARLY_EXIT selects returns at each stop condition (faster in the table walk)
// or one combined stop flag with an unconditional advance (faster in the
// batched walk); both give the same visits and deposits.
// AXES: the chosen axis's {n, cell stride, h bits} come from one 16-byte load of
// axes[axis] (a per-block shared-memory copy of the grid) instead of selects
// among constant-bank values.
// DARK: the caller knows the ray is dark and no optical-depth cut is requested, so
// the step is the DDA alone (same visits as the full step; kap is not read).
template <bool REC = true, bool EARLY_EXIT = true, bool AXES = false, bool DARK = false,
          typename Prefetch = NoPrefetch>
__device__ __forceinline__ bool ray_step(const WalkParams &W, float kap, double *__restrict__ absorbed,
                                         uint32_t *status, const RecordPtrs &rec, Ray &R,
                                         bool writes = true, Prefetch pf = Prefetch(),
                                         const int4 *axes = nullptr) {
  const bool a0 = R.tx <= R.ty && R.tx <= R.tz;
  const bool a1 = !a0 && R.ty <= R.tz;
  const float tn = a0 ? R.tx : (a1 ? R.ty : R.tz);
  const float iv = a0 ? R.ivx : (a1 ? R.ivy : R.ivz);
  const int st = iv > 0.0f ? 1 : -1;
  const int inew = (a0 ? R.ix : (a1 ? R.iy : R.iz)) + st;
  int nax, stride;
  float h;
  if (AXES) {
    const int4 c = axes[a0 ? 0 : (a1 ? 1 : 2)];
    nax = c.x;
    stride = c.y;
    h = __int_as_float(c.z);
  } else {
    nax = a0 ? W.n[0] : (a1 ? W.n[1] : W.n[2]);
    stride = a0 ? 1 : (a1 ? W.n[0] : W.n[0] * W.n[1]);
    h = a0 ? W.h[0] : (a1 ? W.h[1] : W.h[2]);
  }
  const bool inside = tn != INFINITY && (unsigned)inew < (unsigned)nax;  // 0 <= inew < nax
  const int cnext = R.cell + st * stride;
  if (inside) pf(cnext);

  const float ds = __fsub_rn(tn, R.t);
  const float trans0 = R.trans;
  // Once the transmission has underflowed to zero it stays zero (tau only grows): a
  // dark ray deposits nothing and its optical depth matters only to the optical-depth
  // cut, so without the cut it skips the depth sum and both exponentials (its visits,
  // deposits and escaped weight are those of the full update).
  if (!DARK && (trans0 != 0.0f || W.tau_cut)) {
    // the segment's optical depth; an unbounded segment (a ray that never reaches a
    // wall, ds = inf) is held at 1e30, which leaves a transmission of exactly 0 and
    // a deposit of w trans0, as an infinite depth would, without infinities in the sum
    const float a = kap > 0.0f ? fminf(__fmul_rn(__fmul_rn(kap, 100.0f), ds), 1e30f) : 0.0f;
    // compensated optical depth
    {
      const float y = __fsub_rn(a, R.tc);
      const float sum = __fadd_rn(R.tau, y);
      R.tc = __fsub_rn(__fsub_rn(sum, R.tau), y);
      R.tau = sum;
    }
    // deposit and transmission exp(-tau)
    if (trans0 != 0.0f) {
      const float dep = R.w * trans0 * one_minus_exp_neg(a);
      if (writes && dep != 0.0f) atomicAdd(absorbed + R.cell, (double)dep);
      R.trans = __expf(__fsub_rn(R.tc, R.tau));
    }
  }
  if (REC && writes && R.row >= 0 && R.nv < W.rec_max) {
    rec.cells[(long long)R.row * W.rec_max + R.nv] = R.cell;
    rec.ds[(long long)R.row * W.rec_max + R.nv] = ds;
  }
  ++R.nv;
  const bool cut = !DARK && W.tau_cut && R.tau > 100.0f;
  const bool capped = R.nv >= W.step_cap;
  if (EARLY_EXIT) {
    if (tn == INFINITY || cut) return true;
    if (capped) {
      if (writes) status_or(status, RT_DEV_STEPCAP);
      return true;
    }
    if (!inside) return true;
  } else {
    // a ray that stops keeps only w, trans, nv and row meaningful, so the advance
    // below need not be conditional
    if (writes && capped && tn != INFINITY && !cut) status_or(status, RT_DEV_STEPCAP);
  }
  R.t = tn;
  R.cell = cnext;
  const float ps = a0 ? R.px : (a1 ? R.py : R.pz);
  const float tm = tmax_of(inew, st, h, ps, iv);
  R.ix = a0 ? inew : R.ix;
  R.iy = a1 ? inew : R.iy;
  R.iz = (!a0 && !a1) ? inew : R.iz;
  R.tx = a0 ? tm : R.tx;
  R.ty = a1 ? tm : R.ty;
  R.tz = (!a0 && !a1) ? tm : R.tz;
  return !inside || cut || capped;
}

// Host: validation and walk parameters common to every walk (rt_trace.cu).
rt_status walk_setup(const rt_grid *grid, const rt_spectral *spec, uint64_t ray_begin,
                     uint64_t n_rays, uint64_t n_total, uint64_t seed, uint32_t enclosure,
                     int32_t flags, const rt_tally_buf *tally, const rt_record *record,
                     WalkParams *W, RecordPtrs *rp);
// Host: wavenumber-major copy tabt[j * nT + k] of a T-major table.
rt_status launch_transpose(const float *tab, int nT, long long n_nu, float *tabt, cudaStream_t st);
// Host: the walk's copy of a T-major table: node pairs (layout 2) when nT >= 2 and the
// pair table fits kPairTableBytes (so that it can stay in L2), else wavenumber-major (1).
constexpr size_t kPairTableBytes = size_t(64) << 20;
int walk_table_layout(int nT, long long n_nu);
size_t walk_table_bytes(int layout, int nT, long long n_nu);
rt_status launch_walk_table(int layout, const float *tab, int nT, long long n_nu, float *out, cudaStream_t st);
// Host: the CellParams of a spectral spec (table T grid, reference state).
CellParams cell_params(const rt_spectral *spec, long long ncells, int has_px);
// Host: rays [0, W.n_rays) grouped by band = (wavenumber index) / band_pts: per-band
// counts (n_bands words, reused as scatter cursors), band_start and item_start
// ([n_bands + 1]: first position of each band in the grouped order and first work
// item of `chunk` rays), and, if order is given, the rays' offsets grouped by band
// (within a band in arrival order).  One band: band_start = {0, n_rays}, no order.
rt_status band_plan(const WalkParams &W, int band_pts, long long n_bands, long long chunk,
                    unsigned long long *counts, long long *band_start, long long *item_start, uint32_t *order,
                    int sms, cudaStream_t st);
// Host: per-cell T bracket, density scale and T (float4 per cell).
rt_status cell_prep(const rt_grid *grid, const rt_spectral *spec, float4 *cells, uint32_t *status,
                    cudaStream_t st);

}  // namespace rt
