// Monte-Carlo ray tracing through finite volumes (Section 3, Fig. ray) and the
// final tally reduction.
//   k_cell_prep : per cell, the binary32 temperature bracket (k, frac) of the
//                 kappa table, the density scale (p x)/(p_ref x_ref) and T.
//   k_walk      : per ray, Philox draws -> emission cell, wavenumber, position,
//                 isotropic direction -> cell-by-cell walk with Beer-Lambert
//                 attenuation (Eq. I, first term), binary64 atomic deposits.
//   k_reduce / k_final : deterministic two-pass binary64 sum of the absorbed
//                 power and the energy balance.
#include <cmath>

#include "rt_common.cuh"

namespace rt {

rt_status validate_spec(const rt_spectral *s);

namespace {

constexpr int kWalkThreads = 256;
constexpr int kReduceBlocks = 256;

struct CellParams {
  long long ncells;
  float Tmin, dT, den, pref, xref;
  int nT, has_px;
};

__global__ void k_cell_prep(const float *__restrict__ T, const float *__restrict__ p,
                            const float *__restrict__ x, CellParams C, float4 *__restrict__ out,
                            uint32_t *status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C.ncells) return;
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
  out[c] = make_float4(frac, sc, Tc, __int_as_float(k));
}

struct WalkParams {
  int n[3];
  int fin[3];
  float h[3];
  long long ncells, n_nu;
  int nT, mode, tau_cut, step_cap;
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

__device__ __forceinline__ float cell_kappa(const float4 cd, const float *__restrict__ tab,
                                            long long n_nu, int nT, long long j) {
  const int k = __float_as_int(cd.w);
  const float v0 = __ldg(tab + (long long)k * n_nu + j);
  if (nT < 2) return cd.y * v0;
  const float v1 = __ldg(tab + (long long)(k + 1) * n_nu + j);
  return cd.y * fmaf(cd.x, v1, (1.0f - cd.x) * v0);
}

__device__ __forceinline__ float tmax_of(int i, int step, float h, float pos, float invd) {
  const float plane = __fmul_rn((float)(i + (step > 0 ? 1 : 0)), h);
  return __fmul_rn(__fsub_rn(plane, pos), invd);
}

// State of one ray between walk steps (registers of its lane).
struct Ray {
  int ix, iy, iz, sx, sy, sz, cell, j, nv, row;
  float px, py, pz, ivx, ivy, ivz, tx, ty, tz, t, tau, tc, trans, w;
};

// Philox draws -> emission cell, wavenumber, position, direction, weight; DDA set-up.
__device__ __forceinline__ void ray_init(const WalkParams &W, const float4 *__restrict__ cells,
                                         const float *__restrict__ tab, unsigned long long rr,
                                         bool record, Ray &R) {
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
    R.ix = (int)(c % W.n[0]);
    R.iy = (int)((c / W.n[0]) % W.n[1]);
    R.iz = (int)(c / nxy);
    R.px = W.fin[0] ? __fmul_rn(__fadd_rn((float)R.ix, fx), W.h[0]) : 0.0f;
    R.py = W.fin[1] ? __fmul_rn(__fadd_rn((float)R.iy, fy), W.h[1]) : 0.0f;
    R.pz = W.fin[2] ? __fmul_rn(__fadd_rn((float)R.iz, fz), W.h[2]) : 0.0f;
    // emission weight: 4 pi V kappa I_b(nu_j, T_c) dnu * ncells n_nu / N  (Eq. planck)
    const float4 cd = cells[c];
    const float kap = cell_kappa(cd, tab, W.n_nu, W.nT, R.j);
    const float nu_m = 100.0f * fmaf((float)R.j, W.dnu, W.nu_min);
    const float ib = W.two_hc2 * nu_m * nu_m * nu_m / expm1f(W.c2_m * nu_m / cd.z);
    R.w = W.w_scale * kap * ib;
  }
  R.sx = R.sy = R.sz = 0;
  R.ivx = R.ivy = R.ivz = 0.0f;
  R.tx = R.ty = R.tz = INFINITY;
  if (W.fin[0] && dx != 0.0f) { R.sx = dx > 0.0f ? 1 : -1; R.ivx = __fdiv_rn(1.0f, dx); R.tx = tmax_of(R.ix, R.sx, W.h[0], R.px, R.ivx); }
  if (W.fin[1] && dy != 0.0f) { R.sy = dy > 0.0f ? 1 : -1; R.ivy = __fdiv_rn(1.0f, dy); R.ty = tmax_of(R.iy, R.sy, W.h[1], R.py, R.ivy); }
  if (W.fin[2] && dz != 0.0f) { R.sz = dz > 0.0f ? 1 : -1; R.ivz = __fdiv_rn(1.0f, dz); R.tz = tmax_of(R.iz, R.sz, W.h[2], R.pz, R.ivz); }
  R.cell = (int)(R.ix + (long long)W.n[0] * R.iy + nxy * R.iz);
  R.row = (record && rr < (unsigned long long)W.rec_n) ? (int)rr : -1;
  R.t = 0.0f; R.tau = 0.0f; R.tc = 0.0f; R.trans = 1.0f;
  R.nv = 0;
}

// One visit: deposit in the current cell (Eq. I, first term), advance to the next.
// Returns true when the ray has left the grid (or can never reach a wall).
__device__ __forceinline__ bool ray_step(const WalkParams &W, const float4 *__restrict__ cells,
                                         const float *__restrict__ tab, double *__restrict__ absorbed,
                                         uint32_t *status, const RecordPtrs &rec, Ray &R) {
  int ax;
  float tn;
  if (R.tx <= R.ty && R.tx <= R.tz) { ax = 0; tn = R.tx; }
  else if (R.ty <= R.tz) { ax = 1; tn = R.ty; }
  else { ax = 2; tn = R.tz; }
  const float ds = __fsub_rn(tn, R.t);
  const float kap = cell_kappa(cells[R.cell], tab, W.n_nu, W.nT, R.j);
  const float a = kap > 0.0f ? __fmul_rn(__fmul_rn(kap, 100.0f), ds) : 0.0f;
  const float dep = R.w * R.trans * (-expm1f(-a));
  if (dep != 0.0f) atomicAdd(absorbed + R.cell, (double)dep);
  // compensated optical depth, transmission exp(-tau)
  if (a == INFINITY) {
    R.tau = INFINITY;
    R.trans = 0.0f;
  } else {
    const float y = __fsub_rn(a, R.tc);
    const float s = __fadd_rn(R.tau, y);
    R.tc = __fsub_rn(__fsub_rn(s, R.tau), y);
    R.tau = s;
    R.trans = expf(__fsub_rn(R.tc, R.tau));
  }
  if (R.row >= 0 && R.nv < W.rec_max) {
    rec.cells[(long long)R.row * W.rec_max + R.nv] = R.cell;
    rec.ds[(long long)R.row * W.rec_max + R.nv] = ds;
  }
  ++R.nv;
  if (tn == INFINITY) return true;
  if (W.tau_cut && R.tau > 100.0f) return true;
  if (R.nv >= W.step_cap) { status_or(status, RT_DEV_STEPCAP); return true; }
  R.t = tn;
  if (ax == 0) {
    R.ix += R.sx;
    if (R.ix < 0 || R.ix >= W.n[0]) return true;
    R.cell += R.sx;
    R.tx = tmax_of(R.ix, R.sx, W.h[0], R.px, R.ivx);
  } else if (ax == 1) {
    R.iy += R.sy;
    if (R.iy < 0 || R.iy >= W.n[1]) return true;
    R.cell += R.sy * W.n[0];
    R.ty = tmax_of(R.iy, R.sy, W.h[1], R.py, R.ivy);
  } else {
    R.iz += R.sz;
    if (R.iz < 0 || R.iz >= W.n[2]) return true;
    R.cell += R.sz * W.n[0] * W.n[1];
    R.tz = tmax_of(R.iz, R.sz, W.h[2], R.pz, R.ivz);
  }
  return false;
}

// Persistent walk: each warp owns a contiguous range of rays.  Lanes step their
// own rays; when half of the warp's lanes are idle (ballot), the idle lanes take
// the warp's next rays together, so ray set-up and stepping stay converged.
constexpr int kRefillIdle = 16;

__global__ void __launch_bounds__(kWalkThreads)
k_walk(const float4 *__restrict__ cells, const float *__restrict__ tab, WalkParams W,
       double *__restrict__ absorbed, double *__restrict__ scalars,
       unsigned long long *__restrict__ steps_out, uint32_t *status, RecordPtrs rec) {
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const unsigned long long wid = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long next = W.n_rays * wid / nwarps;
  const unsigned long long last = W.n_rays * (wid + 1) / nwarps;
  const bool record = rec.cells != nullptr;
  double em = 0.0, esc = 0.0;
  unsigned long long nsteps = 0;
  Ray R;
  bool active = false;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (next < last && (idle == 0xffffffffu || __popc(idle) >= kRefillIdle)) {
      const unsigned rank = __popc(idle & ((1u << lane) - 1u));
      if (!active && next + rank < last) {
        ray_init(W, cells, tab, next + rank, record, R);
        active = true;
      }
      next += __popc(idle);
    }
    if (!__any_sync(0xffffffffu, active)) break;
    if (active && ray_step(W, cells, tab, absorbed, status, rec, R)) {
      const float out = R.w * R.trans;
      em += (double)R.w;
      esc += (double)out;
      nsteps += (unsigned long long)R.nv;
      if (R.row >= 0) {
        rec.nvis[R.row] = R.nv;
        if (rec.weight) rec.weight[R.row] = R.w;
        if (rec.escaped) rec.escaped[R.row] = out;
      }
      active = false;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    em += __shfl_down_sync(0xffffffffu, em, o);
    esc += __shfl_down_sync(0xffffffffu, esc, o);
    nsteps += __shfl_down_sync(0xffffffffu, nsteps, o);
  }
  if (lane == 0) {
    if (em != 0.0) atomicAdd(scalars + 0, em);
    if (esc != 0.0) atomicAdd(scalars + 2, esc);
    if (nsteps) atomicAdd(steps_out, nsteps);
  }
}

__global__ void k_reduce(const double *__restrict__ a, long long n, double *__restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

__global__ void k_final(const double *__restrict__ partial, int np, double *__restrict__ scalars) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += partial[i];
  scalars[1] = s;
  const double e = scalars[0];
  scalars[3] = e != 0.0 ? fabs(e - s - scalars[2]) / e : 0.0;
}

rt_status validate_grid(const rt_grid *g) {
  if (!g) return fail(RT_E_INVAL, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(RT_E_INVAL, "grid dimensions must be >= 1");
  const long long nc = (long long)g->nx * g->ny * g->nz;
  if (nc > (1LL << 31) - 1) return fail(RT_E_INVAL, "grid has more than 2^31-1 cells");
  const double h[3] = {g->hx, g->hy, g->hz};
  for (int a = 0; a < 3; ++a)
    if (!(h[a] > 0) || std::isnan(h[a])) return fail(RT_E_INVAL, "grid cell sizes must be > 0 (or +inf)");
  if (!std::isfinite(g->hx) && !std::isfinite(g->hy) && !std::isfinite(g->hz))
    return fail(RT_E_INVAL, "grid needs at least one bounded axis");
  if (!g->T) return fail(RT_E_INVAL, "grid.T is NULL");
  return RT_OK;
}

}  // namespace

rt_status trace_impl(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                     uint64_t ray_begin, uint64_t n_rays, uint64_t n_total, uint64_t seed,
                     uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                     const rt_record *record, cudaStream_t st) {
  rt_status v = validate_grid(grid);
  if (v != RT_OK) return v;
  v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!kappa) return fail(RT_E_INVAL, "kappa is NULL");
  if (!tally || !tally->absorbed || !tally->scalars || !tally->steps || !tally->status)
    return fail(RT_E_INVAL, "tally buffer has a NULL pointer");
  const int mode = flags & 0xF;
  if (mode != RT_SRC_EMIT && mode != RT_SRC_BEAM) return fail(RT_E_INVAL, "flags: unknown source mode");
  if (flags & ~(0xF | RT_TAU_CUT)) return fail(RT_E_INVAL, "flags: unknown bits");
  if (n_total == 0 || n_rays > n_total) return fail(RT_E_INVAL, "n_rays_total must be >= n_rays and > 0");
  if (mode == RT_SRC_BEAM && !std::isfinite(grid->hx))
    return fail(RT_E_INVAL, "beam mode needs a bounded x axis");
  if (record) {
    if (record->n_rays < 0 || record->n_rays > (1LL << 31) - 1 ||
        (record->n_rays > 0 && (!record->cells || !record->ds || !record->n_visits ||
                                record->max_visits < 1)))
      return fail(RT_E_INVAL, "record: bad buffers");
  }
  if (n_rays == 0) return RT_OK;
  const long long nc = (long long)grid->nx * grid->ny * grid->nz;

  Scratch scr;
  v = scr.alloc((size_t)nc * sizeof(float4), st);
  if (v != RT_OK) return v;
  float4 *cells = scr.as<float4>();

  CellParams C;
  C.ncells = nc;
  C.Tmin = (float)spec->T_min;
  C.dT = spec->nT >= 2 ? (float)((spec->T_max - spec->T_min) / (double)(spec->nT - 1)) : 1.0f;
  C.den = (float)(spec->p_ref_atm * spec->x_ref);
  C.pref = (float)spec->p_ref_atm;
  C.xref = (float)spec->x_ref;
  C.nT = spec->nT;
  C.has_px = (grid->p_atm || grid->x) ? 1 : 0;
  k_cell_prep<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(grid->T, grid->p_atm, grid->x, C, cells,
                                                           tally->status);
  RT_CUDA_TRY(cudaGetLastError());

  WalkParams W;
  W.n[0] = grid->nx; W.n[1] = grid->ny; W.n[2] = grid->nz;
  const double h[3] = {grid->hx, grid->hy, grid->hz};
  double V = 1.0;
  for (int a = 0; a < 3; ++a) {
    W.fin[a] = std::isfinite(h[a]) ? 1 : 0;
    W.h[a] = (float)h[a];
    if (W.fin[a]) V *= h[a];
  }
  W.ncells = nc;
  W.n_nu = spec->n_nu;
  W.nT = spec->nT;
  W.mode = mode;
  W.tau_cut = (flags & RT_TAU_CUT) ? 1 : 0;
  W.step_cap = grid->nx + grid->ny + grid->nz + 4;
  W.ray_begin = ray_begin;
  W.n_rays = n_rays;
  W.seed_lo = (uint32_t)seed;
  W.seed_hi = (uint32_t)(seed >> 32);
  W.enclosure = enclosure;
  W.nu_min = (float)spec->nu_min;
  W.dnu = (float)spec->dnu;
  const double pi = 3.14159265358979323846;
  W.w_scale = (float)(4.0 * pi * V * 100.0 * (100.0 * spec->dnu) * (double)nc *
                      (double)spec->n_nu / (double)n_total);
  const double hP = 6.62607015e-34, cL = 299792458.0, kB = 1.380649e-23;
  W.two_hc2 = (float)(2.0 * hP * cL * cL);
  W.c2_m = (float)(hP * cL / kB);
  RecordPtrs rp{nullptr, nullptr, nullptr, nullptr, nullptr};
  W.rec_n = 0;
  W.rec_max = 0;
  if (record && record->n_rays > 0) {
    rp = RecordPtrs{record->cells, record->ds, record->n_visits, record->weight, record->escaped};
    W.rec_n = record->n_rays;
    W.rec_max = record->max_visits;
  }
  int dev = 0, sms = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  RT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk, kWalkThreads, 0));
  if (per_sm < 1) per_sm = 1;
  // persistent warps, each with a contiguous ray range of at least 64 rays
  unsigned long long want = (n_rays + 64ull * (kWalkThreads / 32) - 1) / (64ull * (kWalkThreads / 32));
  const unsigned long long cap = (unsigned long long)sms * (unsigned long long)per_sm;
  const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  k_walk<<<blocks, kWalkThreads, 0, st>>>(cells, kappa, W, tally->absorbed, tally->scalars,
                                          tally->steps, tally->status, rp);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status tally_impl(const rt_tally_buf *t, int64_t ncells, double *host_absorbed,
                     double *host_scalars, cudaStream_t st) {
  if (!t || !t->absorbed || !t->scalars || !t->steps || !t->status)
    return fail(RT_E_INVAL, "rt_tally: bad tally buffer");
  if (ncells < 1) return fail(RT_E_INVAL, "rt_tally: ncells must be >= 1");
  if (!host_scalars) return fail(RT_E_INVAL, "rt_tally: host_scalars is NULL");
  Scratch scr;
  rt_status v = scr.alloc(sizeof(double) * kReduceBlocks, st);
  if (v != RT_OK) return v;
  k_reduce<<<kReduceBlocks, 256, 0, st>>>(t->absorbed, ncells, scr.as<double>());
  RT_CUDA_TRY(cudaGetLastError());
  k_final<<<1, 32, 0, st>>>(scr.as<double>(), kReduceBlocks, t->scalars);
  RT_CUDA_TRY(cudaGetLastError());
  uint32_t bits = 0;
  RT_CUDA_TRY(cudaMemcpyAsync(host_scalars, t->scalars, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (host_absorbed)
    RT_CUDA_TRY(cudaMemcpyAsync(host_absorbed, t->absorbed, (size_t)ncells * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  RT_CUDA_TRY(cudaMemcpyAsync(&bits, t->status, sizeof(bits), cudaMemcpyDeviceToHost, st));
  RT_CUDA_TRY(cudaStreamSynchronize(st));
  return status_from_bits(bits);
}

}  // namespace rt

extern "C" {

rt_status rt_trace(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                   uint64_t ray_begin, uint64_t n_rays, uint64_t n_rays_total, uint64_t seed,
                   uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                   const rt_record *record, void *stream) {
  return rt::trace_impl(grid, kappa, spec, ray_begin, n_rays, n_rays_total, seed, enclosure, flags,
                        tally, record, (cudaStream_t)stream);
}

rt_status rt_tally(const rt_tally_buf *tally, int64_t ncells, double *host_absorbed,
                   double host_scalars[4], void *stream) {
  return rt::tally_impl(tally, ncells, host_absorbed, host_scalars, (cudaStream_t)stream);
}

}  // extern "C"
