// On-the-fly line-by-line walk: the Monte-Carlo walk of Section 3 with the
// absorption coefficient of each visited cell summed over the lines within the
// cutoff at that cell's own temperature, pressure and mole fraction (Eqs. S and
// tau evaluated per step, no table, no interpolation).  It is the plain
// line-by-line path that a table or the surrogate network replaces.
//   k_line_pack : per line, binary32 constants of Eq. S and the Doppler width.
//   k_walk_lbl  : one warp per ray; the lanes split the ray's line window, a
//                 warp sum gives kappa, and every lane advances the same ray
//                 state (lane 0 writes the deposits).
#include <cmath>

#include "rt_common.cuh"
#include "rt_walk.cuh"

namespace rt {

rt_status launch_line_geometry(const double *nu0, const double *S, const double *g, const double *E,
                               long long n, const rt_spectral *spec, int check, int4 *R,
                               unsigned long long *evals, uint32_t *status, cudaStream_t st);

namespace {

constexpr double kH = 6.62607015e-34, kC = 299792458.0, kKB = 1.380649e-23;
constexpr double kAmu = 1.66053906660e-27, kAtm = 101325.0, kPi = 3.14159265358979323846;

struct LineConst {
  float T_ref, q_exp, n_T, c2, doppler, u_coef, sqrt_ln2, inv_pi;
};

// L0 = {S_ref, gamma_ref, c2 nu0, 1 - exp(-c2 nu0 / T_ref)}, L1 = {c2 E hi, c2 E lo, nu0, 0}
__global__ void k_line_pack(const double *__restrict__ nu0, const double *__restrict__ S,
                            const double *__restrict__ g, const double *__restrict__ E, long long n,
                            double c2, double T_ref, float4 *__restrict__ L0, float4 *__restrict__ L1) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const float c2f = __double2float_rn(c2);
  const float nu = __double2float_rn(nu0[l]);
  const df c2E = df_mul(df_from_double(c2), df_from_double(E[l]));
  const float c2nu = c2f * nu;
  const float den = -expm1f(-c2nu / __double2float_rn(T_ref));
  L0[l] = make_float4(__double2float_rn(S[l]), __double2float_rn(g[l]), c2nu, den);
  L1[l] = make_float4(c2E.hi, c2E.lo, nu, 0.0f);
}

__device__ __forceinline__ long long first_hi_ge(const int4 *R, long long n, int j) {
  long long a = 0, b = n;
  while (a < b) {
    const long long m = (a + b) >> 1;
    if (R[m].y < j) a = m + 1; else b = m;
  }
  return a;
}
__device__ __forceinline__ long long first_lo_gt(const int4 *R, long long n, int j) {
  long long a = 0, b = n;
  while (a < b) {
    const long long m = (a + b) >> 1;
    if (R[m].x <= j) a = m + 1; else b = m;
  }
  return a;
}

// kappa [cm^-1] at wavenumber index j and state (T, p, x): lines [l0, l1) split over the warp
template <int PROFILE>
__device__ __forceinline__ float kappa_lbl(const int4 *__restrict__ R, const float4 *__restrict__ L0,
                                           const float4 *__restrict__ L1, long long l0, long long l1,
                                           int j, float T, float p, float x, const LineConst &K,
                                           float dnu, const WeidCoef &wc) {
  const int lane = threadIdx.x & 31;
  const float iT = __frcp_rn(T);
  const float d = __fsub_rn(__frcp_rn(K.T_ref), iT);         // 1/T_ref - 1/T
  const float tr = K.T_ref * iT;
  const float qr = powf(tr, K.q_exp);
  const float gfac = p * powf(tr, K.n_T);
  const float u_T = K.u_coef * x * p * iT;                  // number density, cm^-3
  const float sT = sqrtf(T);
  float acc = 0.0f, cmp = 0.0f;
  for (long long l = l0 + lane; l < l1; l += 32) {
    const int4 r = R[l];
    if (j < r.x || j > r.y) continue;
    const float4 a = L0[l], b = L1[l];
    const float boltz = expf(fmaf(b.x, d, b.y * d));
    const float stim = (1.0f - __expf(-a.z * iT)) / a.w;
    const float A = u_T * a.x * qr * boltz * stim;
    const float gam = a.y * gfac;
    const float u = (float)(j - r.z) + __int_as_float(r.w);   // offset in grid units
    float v;
    if (PROFILE == RT_PROFILE_LORENTZ) {
      const float gg = gam / dnu;
      v = A * (gg * K.inv_pi / dnu) / fmaf(u, u, gg * gg);
    } else {
      const float s = K.sqrt_ln2 / (b.z * sT * K.doppler);
      v = A * s * K.inv_pi * faddeeva_re(s * dnu * u, s * gam, wc);
    }
    const float yk = __fsub_rn(v, cmp);
    const float t = __fadd_rn(acc, yk);
    cmp = __fsub_rn(__fsub_rn(t, acc), yk);
    acc = t;
  }
  float s = __fsub_rn(acc, cmp);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <int PROFILE>
__global__ void __launch_bounds__(256)
k_walk_lbl(const int4 *__restrict__ R, const float4 *__restrict__ L0, const float4 *__restrict__ L1,
           long long n_lines, const float *__restrict__ T, const float *__restrict__ Pf,
           const float *__restrict__ Xf, float p_ref, float x_ref, LineConst K, WeidCoef wc,
           WalkParams W, double *__restrict__ absorbed, double *__restrict__ scalars,
           unsigned long long *__restrict__ steps_out, uint32_t *status, RecordPtrs rec) {
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const unsigned long long wid = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool record = rec.cells != nullptr;
  const bool lead = lane == 0;
  double em = 0.0, esc = 0.0;
  unsigned long long nsteps = 0;
  for (unsigned long long rr = wid; rr < W.n_rays; rr += nwarps) {
    Ray Ry;
    ray_init(W, nullptr, nullptr, rr, record, Ry);
    const long long l0 = first_hi_ge(R, n_lines, Ry.j);
    const long long l1 = first_lo_gt(R, n_lines, Ry.j);
    for (;;) {
      const float Tc = T[Ry.cell];
      const float pc = Pf ? Pf[Ry.cell] : p_ref;
      const float xc = Xf ? Xf[Ry.cell] : x_ref;
      const float kap = kappa_lbl<PROFILE>(R, L0, L1, l0, l1, Ry.j, Tc, pc, xc, K, W.dnu, wc);
      if (Ry.w < 0.0f) Ry.w = (W.mode == RT_SRC_BEAM) ? 1.0f : emission_weight(W, Ry.j, Tc, kap);
      if (ray_step(W, kap, absorbed, status, rec, Ry, lead)) break;
      if (Ry.trans == 0.0f && !W.tau_cut) {
        // dark (uniform over the warp's one ray): its remaining steps need no line sum
        while (!ray_step<true, true, false, true>(W, 0.0f, absorbed, status, rec, Ry, lead)) {
        }
        break;
      }
    }
    const float out = Ry.w * Ry.trans;
    em += (double)Ry.w;
    esc += (double)out;
    nsteps += (unsigned long long)Ry.nv;
    if (lead && Ry.row >= 0) {
      rec.nvis[Ry.row] = Ry.nv;
      if (rec.weight) rec.weight[Ry.row] = Ry.w;
      if (rec.escaped) rec.escaped[Ry.row] = out;
    }
  }
  if (lead) {
    if (em != 0.0) atomicAdd(scalars + 0, em);
    if (esc != 0.0) atomicAdd(scalars + 2, esc);
    if (nsteps) atomicAdd(steps_out, nsteps);
  }
}

}  // namespace

rt_status trace_lbl_impl(const rt_grid *grid, const rt_lines *lines, const rt_spectral *spec,
                         uint64_t ray_begin, uint64_t n_rays, uint64_t n_total, uint64_t seed,
                         uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                         const rt_record *record, cudaStream_t st) {
  WalkParams W;
  RecordPtrs rp;
  rt_status v = walk_setup(grid, spec, ray_begin, n_rays, n_total, seed, enclosure, flags, tally,
                           record, &W, &rp);
  if (v != RT_OK) return v;
  if (!lines || lines->n < 0 || (lines->n > 0 && (!lines->nu0 || !lines->S_ref || !lines->gamma_ref ||
                                                  !lines->E_lower)))
    return fail(RT_E_INVAL, "rt_trace_lbl: bad line list");
  if (lines->memory != RT_MEM_HOST && lines->memory != RT_MEM_DEVICE)
    return fail(RT_E_INVAL, "lines.memory must be RT_MEM_HOST or RT_MEM_DEVICE");
  if (!(lines->T_ref > 0) || !(lines->mass_amu > 0) || !std::isfinite(lines->n_T) || !std::isfinite(lines->q_exp))
    return fail(RT_E_INVAL, "lines: T_ref, mass_amu > 0 and finite exponents required");
  if (lines->memory == RT_MEM_HOST) {
    for (int64_t l = 1; l < lines->n; ++l)
      if (!(lines->nu0[l - 1] <= lines->nu0[l])) return fail(RT_E_UNSORTED, "rt_trace_lbl: lines not sorted");
  }
  if (n_rays == 0) return RT_OK;
  const long long n = lines->n;
  const size_t bl = (lines->memory == RT_MEM_HOST) ? 4 * (size_t)n * sizeof(double) : 0;
  const size_t oR = (bl + 255) & ~size_t(255);
  const size_t o0 = (oR + (size_t)n * 16 + 255) & ~size_t(255);
  const size_t o1 = (o0 + (size_t)n * 16 + 255) & ~size_t(255);
  Scratch scr;
  v = scr.alloc(o1 + (size_t)n * 16 + 16, st);
  if (v != RT_OK) return v;
  char *base = scr.as<char>();
  const double *d_nu0 = lines->nu0, *d_S = lines->S_ref, *d_g = lines->gamma_ref, *d_E = lines->E_lower;
  if (lines->memory == RT_MEM_HOST && n > 0) {
    double *d = reinterpret_cast<double *>(base);
    RT_CUDA_TRY(cudaMemcpyAsync(d, lines->nu0, n * 8, cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + n, lines->S_ref, n * 8, cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + 2 * n, lines->gamma_ref, n * 8, cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + 3 * n, lines->E_lower, n * 8, cudaMemcpyHostToDevice, st));
    d_nu0 = d; d_S = d + n; d_g = d + 2 * n; d_E = d + 3 * n;
  }
  int4 *R = reinterpret_cast<int4 *>(base + oR);
  float4 *L0 = reinterpret_cast<float4 *>(base + o0);
  float4 *L1 = reinterpret_cast<float4 *>(base + o1);
  const double c2 = 100.0 * kH * kC / kKB;
  if (n > 0) {
    v = launch_line_geometry(d_nu0, d_S, d_g, d_E, n, spec, lines->memory == RT_MEM_DEVICE ? 1 : 0, R,
                             nullptr, tally->status, st);
    if (v != RT_OK) return v;
    k_line_pack<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_nu0, d_S, d_g, d_E, n, c2, lines->T_ref, L0, L1);
    RT_CUDA_TRY(cudaGetLastError());
  }
  LineConst K;
  K.T_ref = (float)lines->T_ref;
  K.q_exp = (float)lines->q_exp;
  K.n_T = (float)lines->n_T;
  K.c2 = (float)c2;
  K.doppler = (float)(std::sqrt(2.0 * std::log(2.0) * kKB / (lines->mass_amu * kAmu)) / kC);
  K.u_coef = (float)(kAtm / kKB * 1e-6);
  K.sqrt_ln2 = (float)std::sqrt(std::log(2.0));
  K.inv_pi = (float)(1.0 / kPi);
  WeidCoef wc;
  weideman_coefficients(&wc);
  int dev = 0, sms = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned long long want = (n_rays + 7) / 8;
  const unsigned long long cap = (unsigned long long)sms * 8ull;
  const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  if (spec->profile == RT_PROFILE_LORENTZ)
    k_walk_lbl<RT_PROFILE_LORENTZ><<<blocks, 256, 0, st>>>(R, L0, L1, n, grid->T, grid->p_atm, grid->x,
        (float)spec->p_ref_atm, (float)spec->x_ref, K, wc, W, tally->absorbed, tally->scalars,
        tally->steps, tally->status, rp);
  else
    k_walk_lbl<RT_PROFILE_VOIGT><<<blocks, 256, 0, st>>>(R, L0, L1, n, grid->T, grid->p_atm, grid->x,
        (float)spec->p_ref_atm, (float)spec->x_ref, K, wc, W, tally->absorbed, tally->scalars,
        tally->steps, tally->status, rp);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

extern "C" rt_status rt_trace_lbl(const rt_grid *grid, const rt_lines *lines, const rt_spectral *spec,
                                  uint64_t ray_begin, uint64_t n_rays, uint64_t n_rays_total,
                                  uint64_t seed, uint32_t enclosure, int32_t flags,
                                  const rt_tally_buf *tally, const rt_record *record, void *stream) {
  return rt::trace_lbl_impl(grid, lines, spec, ray_begin, n_rays, n_rays_total, seed, enclosure, flags,
                            tally, record, (cudaStream_t)stream);
}
