// Spectrally resolved marching of Eq. (I) along rays (the paper's own kernel,
// Section 3 Listing "Parallel evaluation of (tau)-(planck)"): for every
// spectral sample nu_j, the intensity crossing a cell of length l becomes
//   I_out = I_in exp(-kappa l) + I_b(nu_j, T_cell) (1 - exp(-kappa l)),
// cell after cell, and the power lost by the beam is sum_j (I_in - I_out) dnu.
// The paper runs one full-screen pass per crossed cell over the spectral
// samples; here one block owns a slice of 256 wavenumbers of one ray and loops
// over the ray's cells, so consecutive threads read consecutive table entries.
//   k_march_path : per ray, the binary32 walk (cells and lengths), as rt_trace.
//   k_march      : per (256-wavenumber slice, ray), Eq. (I) over the cells and
//                  a binary64 block sum of (I_in - I_out) dnu.
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

__global__ void __launch_bounds__(kMarchThreads)
k_march(const float4 *__restrict__ cells, const float *__restrict__ tab, MarchParams M,
        const int *__restrict__ vis_cell, const float *__restrict__ vis_len, const int *__restrict__ nvis,
        const float *__restrict__ I_in, float *__restrict__ I_out, double *__restrict__ power) {
  __shared__ float4 s_cd[kMarchMaxVis];
  __shared__ float s_len[kMarchMaxVis];
  __shared__ double s_red[kMarchThreads / 32];
  const long long r = blockIdx.y;
  const long long j = (long long)blockIdx.x * kMarchThreads + threadIdx.x;
  const bool valid = j < M.n_nu;
  const int nv = nvis[r];
  const float nu_m = 100.0f * fmaf((float)j, M.dnu, M.nu_min);
  const float pre = M.two_hc2 * nu_m * nu_m * nu_m;
  const float c2nu = M.c2_m * nu_m;
  const float I0 = (valid && I_in) ? I_in[j] : 0.0f;
  float I = I0;
  for (int v0 = 0; v0 < nv; v0 += kMarchMaxVis) {
    const int cnt = min(kMarchMaxVis, nv - v0);
    __syncthreads();
    for (int v = threadIdx.x; v < cnt; v += kMarchThreads) {
      s_cd[v] = cells[vis_cell[r * M.max_vis + v0 + v]];
      s_len[v] = vis_len[r * M.max_vis + v0 + v];
    }
    __syncthreads();
    if (valid) {
      for (int v = 0; v < cnt; ++v) {
        const float4 cd = s_cd[v];
        const int k = __float_as_int(cd.w);
        float kap = __ldg(tab + (long long)k * M.n_nu + j);
        if (M.nT >= 2) kap = fmaf(cd.x, __ldg(tab + (long long)(k + 1) * M.n_nu + j), (1.0f - cd.x) * kap);
        kap *= cd.y;
        const float a = kap > 0.0f ? kap * 100.0f * s_len[v] : 0.0f;
        const float att = -expm1f(-a);                  // 1 - exp(-kappa l)
        const float ib = pre / expm1f(c2nu / cd.z);     // Eq. (planck), wavenumber form
        I = fmaf(I, 1.0f - att, ib * att);
      }
    }
  }
  if (valid && I_out) I_out[r * M.n_nu + j] = I;
  double d = valid ? (double)(I0 - I) * (double)M.dnu_m : 0.0;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kMarchThreads / 32; ++w) s += s_red[w];
    atomicAdd(power + r, s);
  }
}

}  // namespace

rt_status march_impl(const rt_grid *grid, const float *kappa, const rt_spectral *spec, int64_t n_paths,
                     const float *pos, const float *dir, const float *I_in, float *I_out,
                     double *power, uint32_t *status, cudaStream_t st) {
  rt_status v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!grid || !grid->T || grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
    return fail(RT_E_INVAL, "rt_march: bad grid");
  if (!kappa || !pos || !dir || !power) return fail(RT_E_INVAL, "rt_march: NULL buffer");
  if (n_paths < 0 || n_paths > 65535) return fail(RT_E_INVAL, "rt_march: n_paths must be in [0, 65535]");
  if (n_paths == 0) return RT_OK;
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
  dim3 g((unsigned)((spec->n_nu + kMarchThreads - 1) / kMarchThreads), (unsigned)n_paths);
  k_march<<<g, kMarchThreads, 0, st>>>(cells, kappa, M, vis_cell, vis_len, nvis, I_in, I_out, power);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

extern "C" rt_status rt_march(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                              int64_t n_paths, const float *pos, const float *dir, const float *I_in,
                              float *I_out, double *power, uint32_t *status, void *stream) {
  return rt::march_impl(grid, kappa, spec, n_paths, pos, dir, I_in, I_out, power, status,
                        (cudaStream_t)stream);
}
