// Spectrally resolved marching of Eq. (I) along rays (the paper's own kernel,
// Section 3 Listing "Parallel evaluation of (tau)-(planck)"): for every
// spectral sample nu_j, the intensity crossing a cell of length l becomes
//   I_out = I_in exp(-kappa l) + I_b(nu_j, T_cell) (1 - exp(-kappa l)),
// cell after cell, and the power lost by the beam is sum_j (I_in - I_out) dnu.
// The paper runs one full-screen pass per crossed cell over the spectral
// samples; here one block owns a slice of 1024 wavenumbers of one ray (four per
// thread) and loops over the ray's cells, so consecutive threads read consecutive
// table entries.
//   k_march_path : per ray, the binary32 walk (cells and lengths), as rt_trace.
//   k_march      : per (1024-wavenumber slice, ray), Eq. (I) over the cells, four
//                  wavenumbers per thread, and a binary64 block sum of
//                  (I_in - I_out) dnu.
#include <cmath>

#include "rt_common.cuh"
#include "rt_walk.cuh"

namespace rt {

rt_status validate_spec(const rt_spectral *s);

namespace {

struct MarchParams {
  int n[3], fin[3];
  float h[3];
  int max_vis;
  long long n_nu;
  int nT;
  float nu_min, dnu, two_hc2, c2_m, dnu_m;
};

__global__ void k_march_path(const float *__restrict__ pos, const float *__restrict__ dir,
                             long long n_paths, MarchParams M, int *__restrict__ vis_cell,
                             float *__restrict__ vis_len, int *__restrict__ nvis, uint32_t *status) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_paths) return;
  int i[3], st[3];
  float p[3], iv[3], tm[3];
  for (int a = 0; a < 3; ++a) {
    p[a] = pos[3 * r + a];
    const float d = dir[3 * r + a];
    i[a] = 0;
    if (M.fin[a]) {
      i[a] = (int)floorf(__fdiv_rn(p[a], M.h[a]));
      i[a] = min(max(i[a], 0), M.n[a] - 1);
    }
    if (!M.fin[a] || d == 0.0f) {
      st[a] = 0; iv[a] = 0.0f; tm[a] = INFINITY;
    } else {
      st[a] = d > 0.0f ? 1 : -1;
      iv[a] = __fdiv_rn(1.0f, d);
      tm[a] = tmax_of(i[a], st[a], M.h[a], p[a], iv[a]);
    }
  }
  float t = 0.0f;
  int nv = 0;
  const long long nx = M.n[0], nxy = (long long)M.n[0] * M.n[1];
  for (;;) {
    const int a = (tm[0] <= tm[1] && tm[0] <= tm[2]) ? 0 : (tm[1] <= tm[2] ? 1 : 2);
    const float tn = tm[a];
    if (nv >= M.max_vis) {
      status_or(status, RT_DEV_STEPCAP);
      break;
    }
    vis_cell[r * M.max_vis + nv] = (int)(i[0] + nx * i[1] + nxy * i[2]);
    vis_len[r * M.max_vis + nv] = __fsub_rn(tn, t);
    ++nv;
    if (tn == INFINITY) break;
    t = tn;
    i[a] += st[a];
    if (i[a] < 0 || i[a] >= M.n[a]) break;
    tm[a] = tmax_of(i[a], st[a], M.h[a], p[a], iv[a]);
  }
  nvis[r] = nv;
}

constexpr int kMarchThreads = 256;
constexpr int kMarchMaxVis = 1024;  // cells per path staged in shared memory at a time

// Paired binary32 arithmetic: two wavenumbers per thread, one f32x2 instruction
// for both (each half rounds as the scalar operation).
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// e^x for both halves as 2^(x log2 e): one paired multiply, then the MUFU base-2
// exponential (ex2.approx.ftz, about 2 ulp; a subnormal result is flushed to zero)
constexpr float kLog2e = 1.44269504088896341f;
__device__ __forceinline__ float2 exp2_ftz2(float2 x) {
  const float2 y = __fmul2_rn(x, dup2(kLog2e));
  float2 r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(y.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(y.y));
  return r;
}
// a / b for both halves as a times the MUFU reciprocal of b (rcp.approx.ftz)
__device__ __forceinline__ float2 div_ftz2(float2 a, float2 b) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(b.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(b.y));
  return __fmul2_rn(a, r);
}

// 1 - e^(-a) for a >= 0, both halves: below 1/4 the Taylor series to a^6
// (truncation < a^7/5040, relative 5e-8), above it one minus the hardware
// exponential (relative error below 1.2e-6 at a = 1/4, falling with a).
__device__ __forceinline__ float2 one_minus_exp_neg2(float2 a) {
  float2 p = __ffma2_rn(a, dup2(-1.0f / 720.0f), dup2(1.0f / 120.0f));
  p = __ffma2_rn(a, p, dup2(-1.0f / 24.0f));
  p = __ffma2_rn(a, p, dup2(1.0f / 6.0f));
  p = __ffma2_rn(a, p, dup2(-0.5f));
  p = __ffma2_rn(a, p, dup2(1.0f));
  const float2 s = __fmul2_rn(a, p);
  const float2 e = exp2_ftz2(neg2(a));
  return make_float2(a.x < 0.25f ? s.x : 1.0f - e.x, a.y < 0.25f ? s.y : 1.0f - e.y);
}

// e^x - 1 for x >= 0, both halves: the Taylor series below 1/4, else the hardware
// exponential minus one (same error bounds as above).
__device__ __forceinline__ float2 expm1_pos2(float2 x) {
  float2 p = __ffma2_rn(x, dup2(1.0f / 720.0f), dup2(1.0f / 120.0f));
  p = __ffma2_rn(x, p, dup2(1.0f / 24.0f));
  p = __ffma2_rn(x, p, dup2(1.0f / 6.0f));
  p = __ffma2_rn(x, p, dup2(0.5f));
  p = __ffma2_rn(x, p, dup2(1.0f));
  const float2 s = __fmul2_rn(x, p);
  const float2 e = exp2_ftz2(x);
  return make_float2(x.x < 0.25f ? s.x : e.x - 1.0f, x.y < 0.25f ? s.y : e.y - 1.0f);
}

// Block = 1024 wavenumbers (four per thread, as two pairs) of one path.  The
// path's cells are staged in shared memory with their per-cell constants folded:
// the optical depth of a crossing is a = A kappa_k + B kappa_k+1 with
// A = 100 l s (1 - frac), B = 100 l s frac (l the length in m, s the density
// scale), so one crossing costs the table loads, two paired multiply-adds for a,
// the two exponentials of Eq. I and Eq. planck, and the update
// I <- I + (1 - e^-a)(I_b - I), for each pair.
// VEC: 4 when n_nu is a multiple of 4 and the table 16-byte aligned (one 16-byte
// load per table row), 2 when n_nu is even and the table 8-byte aligned, else 1.
constexpr int kMarchPts = 4;

template <int VEC>
__global__ void __launch_bounds__(kMarchThreads, 6)
k_march(const float4 *__restrict__ cells, const float *__restrict__ tab, MarchParams M,
        const int *__restrict__ vis_cell, const float *__restrict__ vis_len, const int *__restrict__ nvis,
        const float *__restrict__ I_in, float *__restrict__ I_out, double *__restrict__ power) {
  __shared__ float4 s_c[kMarchMaxVis];      // {A, B, 1/T, 0}
  __shared__ long long s_row[kMarchMaxVis];  // k n_nu, the cell's lower table row
  __shared__ double s_red[kMarchThreads / 32];
  const long long r = blockIdx.y;
  const long long j0 = ((long long)blockIdx.x * kMarchThreads + threadIdx.x) * kMarchPts;
  bool ok[kMarchPts];
#pragma unroll
  for (int q = 0; q < kMarchPts; ++q) ok[q] = j0 + q < M.n_nu;
  const int nv = nvis[r];
  float2 pre[2], c2nu[2], I0[2], I[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float2 nu_m = make_float2(100.0f * fmaf((float)(j0 + 2 * h), M.dnu, M.nu_min),
                                    100.0f * fmaf((float)(j0 + 2 * h + 1), M.dnu, M.nu_min));
    pre[h] = __fmul2_rn(__fmul2_rn(__fmul2_rn(dup2(M.two_hc2), nu_m), nu_m), nu_m);
    c2nu[h] = __fmul2_rn(dup2(M.c2_m), nu_m);
    I0[h] = make_float2((ok[2 * h] && I_in) ? I_in[j0 + 2 * h] : 0.0f,
                        (ok[2 * h + 1] && I_in) ? I_in[j0 + 2 * h + 1] : 0.0f);
    I[h] = I0[h];
  }
  for (int v0 = 0; v0 < nv; v0 += kMarchMaxVis) {
    const int cnt = min(kMarchMaxVis, nv - v0);
    __syncthreads();
    for (int v = threadIdx.x; v < cnt; v += kMarchThreads) {
      const float4 cd = cells[vis_cell[r * M.max_vis + v0 + v]];
      const float w = 100.0f * vis_len[r * M.max_vis + v0 + v] * cd.y;
      s_c[v] = make_float4(w * (1.0f - cd.x), w * cd.x, __frcp_rn(cd.z), 0.0f);
      s_row[v] = (long long)__float_as_int(cd.w) * M.n_nu;
    }
    __syncthreads();
    if (ok[0]) {
      for (int v = 0; v < cnt; ++v) {
        const float4 c = s_c[v];
        const float *p0 = tab + s_row[v] + j0;
        float2 t0[2], t1[2];
        if (VEC == 4) {
          const float4 a0 = __ldg(reinterpret_cast<const float4 *>(p0));
          t0[0] = make_float2(a0.x, a0.y);
          t0[1] = make_float2(a0.z, a0.w);
          float4 a1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if (M.nT >= 2) a1 = __ldg(reinterpret_cast<const float4 *>(p0 + M.n_nu));
          t1[0] = make_float2(a1.x, a1.y);
          t1[1] = make_float2(a1.z, a1.w);
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            t1[h] = make_float2(0.0f, 0.0f);
            if (VEC == 2 && ok[2 * h]) {  // n_nu even: both points of the pair or neither
              t0[h] = __ldg(reinterpret_cast<const float2 *>(p0 + 2 * h));
              if (M.nT >= 2) t1[h] = __ldg(reinterpret_cast<const float2 *>(p0 + M.n_nu + 2 * h));
            } else {
              t0[h] = make_float2(ok[2 * h] ? __ldg(p0 + 2 * h) : 0.0f, ok[2 * h + 1] ? __ldg(p0 + 2 * h + 1) : 0.0f);
              if (M.nT >= 2)
                t1[h] = make_float2(ok[2 * h] ? __ldg(p0 + M.n_nu + 2 * h) : 0.0f,
                                    ok[2 * h + 1] ? __ldg(p0 + M.n_nu + 2 * h + 1) : 0.0f);
            }
          }
        }
        float2 a[2], xe[2], att[2], em1[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          a[h] = __ffma2_rn(dup2(c.y), t1[h], __fmul2_rn(dup2(c.x), t0[h]));  // optical depth
          xe[h] = __fmul2_rn(c2nu[h], dup2(c.z));                            // c2 nu / T
        }
        // 1 - exp(-a) and exp(x) - 1: the series runs only when one of the thread's
        // arguments is below 1/4 (each point takes the same form as in the helpers)
        if (fminf(fminf(a[0].x, a[0].y), fminf(a[1].x, a[1].y)) >= 0.25f) {
#pragma unroll
          for (int h = 0; h < 2; ++h) att[h] = __fadd2_rn(dup2(1.0f), neg2(exp2_ftz2(neg2(a[h]))));
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) att[h] = one_minus_exp_neg2(a[h]);
        }
        if (xe[0].x >= 0.25f) {  // the thread's lowest wavenumber has the lowest argument
#pragma unroll
          for (int h = 0; h < 2; ++h) em1[h] = __fadd2_rn(exp2_ftz2(xe[h]), dup2(-1.0f));
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) em1[h] = expm1_pos2(xe[h]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 ib = div_ftz2(pre[h], em1[h]);  // Eq. (planck)
          I[h] = __ffma2_rn(att[h], __fadd2_rn(ib, neg2(I[h])), I[h]);
        }
      }
    }
  }
  double d = 0.0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (ok[2 * h]) {
      if (I_out) I_out[r * M.n_nu + j0 + 2 * h] = I[h].x;
      d += (double)(I0[h].x - I[h].x);
    }
    if (ok[2 * h + 1]) {
      if (I_out) I_out[r * M.n_nu + j0 + 2 * h + 1] = I[h].y;
      d += (double)(I0[h].y - I[h].y);
    }
  }
  d *= (double)M.dnu_m;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kMarchThreads / 32; ++w) sum += s_red[w];
    atomicAdd(power + r, sum);
  }
}

}  // namespace

rt_status march_impl(const rt_grid *grid, const float *kappa, const rt_spectral *spec, int64_t n_paths,
                     const float *pos, const float *dir, const float *I_in, float *I_out,
                     double *power, int32_t *nvis_out, uint32_t *status, cudaStream_t st) {
  rt_status v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!grid || !grid->T || grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
    return fail(RT_E_INVAL, "rt_march: bad grid");
  if (n_paths < 0 || n_paths > 65535) return fail(RT_E_INVAL, "rt_march: n_paths must be in [0, 65535]");
  if (n_paths == 0) return RT_OK;  // no path: the buffers are not read and may be NULL
  if (!kappa || !pos || !dir || !power) return fail(RT_E_INVAL, "rt_march: NULL buffer");
  MarchParams M;
  const double h[3] = {grid->hx, grid->hy, grid->hz};
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  for (int a = 0; a < 3; ++a) {
    if (!(h[a] > 0)) return fail(RT_E_INVAL, "rt_march: cell sizes must be > 0");
    M.n[a] = n[a];
    M.fin[a] = std::isfinite(h[a]) ? 1 : 0;
    M.h[a] = (float)h[a];
  }
  M.max_vis = grid->nx + grid->ny + grid->nz + 4;
  M.n_nu = spec->n_nu;
  M.nT = spec->nT;
  M.nu_min = (float)spec->nu_min;
  M.dnu = (float)spec->dnu;
  const double hP = 6.62607015e-34, cL = 299792458.0, kB = 1.380649e-23;
  M.two_hc2 = (float)(2.0 * hP * cL * cL);
  M.c2_m = (float)(hP * cL / kB);
  M.dnu_m = (float)(100.0 * spec->dnu);
  const long long nc = (long long)grid->nx * grid->ny * grid->nz;
  const size_t b_cells = ((size_t)nc * sizeof(float4) + 255) & ~size_t(255);
  const size_t b_vis = ((size_t)n_paths * M.max_vis * 4 + 255) & ~size_t(255);
  Scratch scr;
  v = scr.alloc(b_cells + 2 * b_vis + (size_t)n_paths * 4, st);
  if (v != RT_OK) return v;
  char *base = scr.as<char>();
  float4 *cells = reinterpret_cast<float4 *>(base);
  int *vis_cell = reinterpret_cast<int *>(base + b_cells);
  float *vis_len = reinterpret_cast<float *>(base + b_cells + b_vis);
  int *nvis = reinterpret_cast<int *>(base + b_cells + 2 * b_vis);
  v = cell_prep(grid, spec, cells, status, st);
  if (v != RT_OK) return v;
  RT_CUDA_TRY(cudaMemsetAsync(power, 0, sizeof(double) * (size_t)n_paths, st));
  k_march_path<<<(unsigned)((n_paths + 127) / 128), 128, 0, st>>>(pos, dir, n_paths, M, vis_cell, vis_len,
                                                                 nvis, status);
  RT_CUDA_TRY(cudaGetLastError());
  const long long per_block = (long long)kMarchThreads * kMarchPts;
  dim3 g((unsigned)((spec->n_nu + per_block - 1) / per_block), (unsigned)n_paths);
  const uintptr_t ka = reinterpret_cast<uintptr_t>(kappa);
  const int vec = (spec->n_nu % 4 == 0 && (ka & 15u) == 0) ? 4 : ((spec->n_nu % 2 == 0 && (ka & 7u) == 0) ? 2 : 1);
  auto kernel = vec == 4 ? k_march<4> : (vec == 2 ? k_march<2> : k_march<1>);
  kernel<<<g, kMarchThreads, 0, st>>>(cells, kappa, M, vis_cell, vis_len, nvis, I_in, I_out, power);
  RT_CUDA_TRY(cudaGetLastError());
  if (nvis_out)
    RT_CUDA_TRY(cudaMemcpyAsync(nvis_out, nvis, sizeof(int32_t) * (size_t)n_paths, cudaMemcpyDeviceToDevice, st));
  return RT_OK;
}

}  // namespace rt

extern "C" rt_status rt_march(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                              int64_t n_paths, const float *pos, const float *dir, const float *I_in,
                              float *I_out, double *power, int32_t *nvis, uint32_t *status, void *stream) {
  return rt::march_impl(grid, kappa, spec, n_paths, pos, dir, I_in, I_out, power, nvis, status,
                        (cudaStream_t)stream);
}
