// Monte-Carlo ray tracing through finite volumes (Section 3, Fig. ray) and the
// final tally reduction.
//   k_cell_prep : per cell, the binary32 temperature bracket (k, frac) of the
//                 kappa table, the density scale (p x)/(p_ref x_ref) and T.
//   k_pair_table: the walk's copy of the table, {kappa_k, kappa_k+1} per
//                 (wavenumber, node), so a step's interpolation is one 8-byte load.
//   k_walk      : per ray, Philox draws -> emission cell, wavenumber, position,
//                 isotropic direction -> cell-by-cell walk with Beer-Lambert
//                 attenuation (Eq. I, first term), binary64 atomic deposits;
//                 persistent warps refilled by ballot.
//   k_reduce / k_final : deterministic two-pass binary64 sum of the absorbed
//                 power and the energy balance.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "rt_common.cuh"
#include "rt_walk.cuh"

namespace rt {

rt_status validate_spec(const rt_spectral *s);

namespace {

constexpr int kWalkThreads = 256;
constexpr int kReduceBlocks = 256;

__global__ void k_cell_prep(const float *__restrict__ T, const float *__restrict__ p,
                            const float *__restrict__ x, CellParams C, float4 *__restrict__ out,
                            uint32_t *status) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C.ncells) return;
  out[c] = cell_prep_one(T, p, x, c, C, status);
}

// Persistent walk: each warp owns a contiguous range of rays.  Lanes step their
// own rays; when half of the warp's lanes are idle (ballot), the idle lanes take
// the warp's next rays together, so ray set-up and stepping stay converged.
constexpr int kRefillIdleDefault = 16;
constexpr int kWalkUnroll = 8;  // steps per pass of the walk loop

// ---------------------------------------------------------------- grouping rays by wavenumber band
constexpr int kBandHist = 8192;  // bands counted in a shared-memory histogram (else global atomics)

// rays per band (counts zeroed before the launch)
__global__ void k_band_count(WalkParams W, int band_pts, long long n_bands, unsigned long long *__restrict__ counts) {
  __shared__ unsigned int hist[kBandHist];
  const bool local = n_bands <= kBandHist;
  if (local)
    for (int b = threadIdx.x; b < (int)n_bands; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  for (unsigned long long rr = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; rr < W.n_rays;
       rr += (unsigned long long)gridDim.x * blockDim.x) {
    const int b = ray_nu_index(W, rr) / band_pts;
    if (local) atomicAdd(&hist[b], 1u);
    else atomicAdd(&counts[b], 1ull);
  }
  __syncthreads();
  if (local)
    for (int b = threadIdx.x; b < (int)n_bands; b += blockDim.x)
      if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

// band_start and item_start (exclusive prefix sums over the bands; one block), the
// scatter cursors; counts == nullptr: one band holding all n_rays rays
__global__ void k_band_plan(const unsigned long long *__restrict__ counts, long long n_bands,
                            unsigned long long n_rays, long long chunk, long long *__restrict__ band_start,
                            long long *__restrict__ item_start, unsigned long long *__restrict__ cursor) {
  __shared__ long long sc[1024], si[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  // each thread sums a contiguous run of bands, then the runs are scanned
  const long long per = (n_bands + nt - 1) / nt;
  const long long b0 = min(n_bands, (long long)t * per), b1 = min(n_bands, b0 + per);
  long long c = 0, it = 0;
  for (long long b = b0; b < b1; ++b) {
    const long long k = counts ? (long long)counts[b] : (long long)n_rays;
    c += k;
    it += (k + chunk - 1) / chunk;
  }
  sc[t] = c;
  si[t] = it;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {  // inclusive scan of the runs (Hillis-Steele)
    const long long a = t >= o ? sc[t - o] : 0, bi = t >= o ? si[t - o] : 0;
    __syncthreads();
    sc[t] += a;
    si[t] += bi;
    __syncthreads();
  }
  long long pc = sc[t] - c, pi = si[t] - it;
  for (long long b = b0; b < b1; ++b) {
    const long long k = counts ? (long long)counts[b] : (long long)n_rays;
    band_start[b] = pc;
    item_start[b] = pi;
    if (cursor) cursor[b] = (unsigned long long)pc;
    pc += k;
    pi += (k + chunk - 1) / chunk;
  }
  if (t == nt - 1) {
    band_start[n_bands] = sc[t];
    item_start[n_bands] = si[t];
  }
}

// ray offsets into their band's run of order (order within a band: arrival order)
__global__ void k_band_scatter(WalkParams W, int band_pts, unsigned long long *__restrict__ cursor,
                               uint32_t *__restrict__ order) {
  for (unsigned long long rr = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; rr < W.n_rays;
       rr += (unsigned long long)gridDim.x * blockDim.x) {
    const int b = ray_nu_index(W, rr) / band_pts;
    order[atomicAdd(&cursor[b], 1ull)] = (uint32_t)rr;
  }
}

}  // namespace

int g_walk_blocks = 5;   // resident walk blocks per SM the launch is compiled for (4 or 5)
int g_walk_refill = 16;  // idle lanes that trigger a refill (12 or 16)
int g_walk_group = 0;    // rays grouped by wavenumber: 0 when >= 32 rays per wavenumber, 1 never, 2 always

namespace {

// [nT][n_nu] -> [n_nu][nT] through 32 x 33 shared tiles
__global__ void k_transpose(const float *__restrict__ in, int rows, long long cols, float *__restrict__ out) {
  __shared__ float t[32][33];
  const long long c0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i;
    const long long c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(long long)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const long long c = c0 + i;
    const int r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = t[threadIdx.x][i];
  }
}

// [nT][n_nu] -> node pairs out[j * (nT - 1) + k] = {in[k][j], in[k + 1][j]}: each block
// stages kPairRows + 1 rows of 32 wavenumbers and writes the pairs wavenumber by wavenumber.
constexpr int kPairRows = 64;
__global__ void k_pair_table(const float *__restrict__ in, int nT, long long n_nu, float2 *__restrict__ out) {
  __shared__ float t[kPairRows + 1][33];
  const long long j0 = (long long)blockIdx.x * 32;
  const int k0 = blockIdx.y * kPairRows;
  const int rows = min(kPairRows + 1, nT - k0);
  for (int idx = threadIdx.x; idx < rows * 32; idx += blockDim.x) {
    const int r = idx >> 5, c = idx & 31;
    if (j0 + c < n_nu) t[r][c] = in[(long long)(k0 + r) * n_nu + j0 + c];
  }
  __syncthreads();
  const int np = rows - 1;
  for (int idx = threadIdx.x; idx < np * 32; idx += blockDim.x) {
    const int c = idx / np, r = idx - c * np;
    if (j0 + c < n_nu) out[(j0 + c) * (long long)(nT - 1) + k0 + r] = make_float2(t[r][c], t[r + 1][c]);
  }
}

template <bool REC, int TAB, int MINB, int REFILL>
__global__ void __launch_bounds__(kWalkThreads, MINB)
k_walk(const float4 *__restrict__ cells, const float *__restrict__ tab, const uint32_t *__restrict__ order,
       WalkParams W, double *__restrict__ absorbed, double *__restrict__ scalars,
       unsigned long long *__restrict__ steps_out, uint32_t *status, RecordPtrs rec) {
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const unsigned long long wid = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long next = W.n_rays * wid / nwarps;
  const unsigned long long last = W.n_rays * (wid + 1) / nwarps;
  const bool record = REC;
  __shared__ int4 s_axes[3];  // per axis {n, cell stride, h bits}
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    s_axes[a] = make_int4(W.n[a], a == 0 ? 1 : (a == 1 ? W.n[0] : W.n[0] * W.n[1]), __float_as_int(W.h[a]), 0);
  }
  __syncthreads();
  double em = 0.0, esc = 0.0;
  unsigned long long nsteps = 0;
  Ray R;
  float4 cd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // data of the ray's current cell
  const float2 *krow = nullptr;  // node-pair table: the ray's wavenumber row
  const float *krow1 = nullptr;  // wavenumber-major table: the ray's row
  bool active = false;
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (next < last && (idle == 0xffffffffu || __popc(idle) >= REFILL)) {
      const unsigned rank = __popc(idle & ((1u << lane) - 1u));
      if (!active && next + rank < last) {
        // order: the rays grouped by wavenumber, so that a warp's lanes share a table row
        ray_init(W, cells, tab, order ? (unsigned long long)__ldg(order + next + rank) : next + rank, record, R,
                 &cd);
        if (TAB == 2) krow = reinterpret_cast<const float2 *>(tab) + (long long)R.j * (W.nT - 1);
        if (TAB == 1) krow1 = tab + (long long)R.j * W.nT;
        active = true;
      }
      next += __popc(idle);
    }
    const unsigned am = __ballot_sync(0xffffffffu, active);
    if (!am) break;
    if (!active) continue;
    bool done = false;
    if (__all_sync(am, R.trans == 0.0f && !W.tau_cut)) {
      // every active lane dark: kWalkUnroll DDA-only steps
#pragma unroll
      for (int u = 0; u < kWalkUnroll; ++u)
        if (!done) done = ray_step<REC, true, true, true>(W, 0.0f, absorbed, status, rec, R, true, NoPrefetch(), s_axes);
    } else {
    // kWalkUnroll steps per pass of the loop; each step loads the table value of
    // its cell and the next cell's data, both in flight while its arithmetic runs
#pragma unroll
    for (int u = 0; u < kWalkUnroll; ++u) {
      if (!done) {
        // a dark ray (transmission zero, no optical-depth cut) needs neither its cell's
        // kappa nor the next cell's data
        const bool lit = R.trans != 0.0f || W.tau_cut;
        const float kap = !lit ? 0.0f : (TAB == 2 ? cell_kappa_row(cd, krow) : (TAB == 1 ? cell_kappa_row1(cd, krow1, W.nT) : cell_kappa_l<TAB>(cd, tab, W.nT, W.n_nu, R.j)));
        float4 cdn = cd;
        done = ray_step<REC, true, true>(W, kap, absorbed, status, rec, R, true,
                                         [&](int c) { if (lit) cdn = __ldg(cells + c); }, s_axes);
        cd = cdn;
      }
    }
    }
    if (done) {
      const float out = R.w * R.trans;
      em += (double)R.w;
      esc += (double)out;
      nsteps += (unsigned long long)R.nv;
      if (REC && R.row >= 0) {
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

rt_status walk_setup(const rt_grid *grid, const rt_spectral *spec, uint64_t ray_begin,
                     uint64_t n_rays, uint64_t n_total, uint64_t seed, uint32_t enclosure,
                     int32_t flags, const rt_tally_buf *tally, const rt_record *record,
                     WalkParams *W, RecordPtrs *rp) {
  rt_status v = validate_grid(grid);
  if (v != RT_OK) return v;
  v = validate_spec(spec);
  if (v != RT_OK) return v;
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
  const long long nc = (long long)grid->nx * grid->ny * grid->nz;
  W->n[0] = grid->nx; W->n[1] = grid->ny; W->n[2] = grid->nz;
  const double h[3] = {grid->hx, grid->hy, grid->hz};
  double V = 1.0;
  for (int a = 0; a < 3; ++a) {
    W->fin[a] = std::isfinite(h[a]) ? 1 : 0;
    W->h[a] = (float)h[a];
    if (W->fin[a]) V *= h[a];
  }
  W->ncells = nc;
  W->n_nu = spec->n_nu;
  W->nT = spec->nT;
  W->mode = mode;
  W->tau_cut = (flags & RT_TAU_CUT) ? 1 : 0;
  W->step_cap = grid->nx + grid->ny + grid->nz + 4;
  W->ray_begin = ray_begin;
  W->n_rays = n_rays;
  W->seed_lo = (uint32_t)seed;
  W->seed_hi = (uint32_t)(seed >> 32);
  W->enclosure = enclosure;
  W->nu_major = 0;
  W->nu_min = (float)spec->nu_min;
  W->dnu = (float)spec->dnu;
  const double pi = 3.14159265358979323846;
  W->w_scale = (float)(4.0 * pi * V * 100.0 * (100.0 * spec->dnu) * (double)nc *
                       (double)spec->n_nu / (double)n_total);
  const double hP = 6.62607015e-34, cL = 299792458.0, kB = 1.380649e-23;
  W->two_hc2 = (float)(2.0 * hP * cL * cL);
  W->c2_m = (float)(hP * cL / kB);
  *rp = RecordPtrs{nullptr, nullptr, nullptr, nullptr, nullptr};
  W->rec_n = 0;
  W->rec_max = 0;
  if (record && record->n_rays > 0) {
    *rp = RecordPtrs{record->cells, record->ds, record->n_visits, record->weight, record->escaped};
    W->rec_n = record->n_rays;
    W->rec_max = record->max_visits;
  }
  return RT_OK;
}

rt_status launch_transpose(const float *tab, int nT, long long n_nu, float *tabt, cudaStream_t st) {
  dim3 tg((unsigned)((n_nu + 31) / 32), (unsigned)((nT + 31) / 32));
  k_transpose<<<tg, dim3(32, 8), 0, st>>>(tab, nT, n_nu, tabt);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

int walk_table_layout(int nT, long long n_nu) {
  return (nT >= 2 && (size_t)n_nu * (size_t)(nT - 1) * 8 <= kPairTableBytes) ? 2 : 1;
}

size_t walk_table_bytes(int layout, int nT, long long n_nu) {
  return layout == 2 ? (size_t)n_nu * (size_t)(nT - 1) * 8 : (size_t)n_nu * (size_t)nT * 4;
}

rt_status launch_walk_table(int layout, const float *tab, int nT, long long n_nu, float *out, cudaStream_t st) {
  if (layout != 2) return launch_transpose(tab, nT, n_nu, out, st);
  dim3 g((unsigned)((n_nu + 31) / 32), (unsigned)((nT - 1 + kPairRows - 1) / kPairRows));
  k_pair_table<<<g, 256, 0, st>>>(tab, nT, n_nu, reinterpret_cast<float2 *>(out));
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

CellParams cell_params(const rt_spectral *spec, long long ncells, int has_px) {
  CellParams C;
  C.ncells = ncells;
  C.Tmin = (float)spec->T_min;
  C.dT = spec->nT >= 2 ? (float)((spec->T_max - spec->T_min) / (double)(spec->nT - 1)) : 1.0f;
  C.den = (float)(spec->p_ref_atm * spec->x_ref);
  C.pref = (float)spec->p_ref_atm;
  C.xref = (float)spec->x_ref;
  C.nT = spec->nT;
  C.has_px = has_px;
  return C;
}

rt_status cell_prep(const rt_grid *grid, const rt_spectral *spec, float4 *cells, uint32_t *status,
                    cudaStream_t st) {
  const long long nc = (long long)grid->nx * grid->ny * grid->nz;
  const CellParams C = cell_params(spec, nc, (grid->p_atm || grid->x) ? 1 : 0);
  k_cell_prep<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(grid->T, grid->p_atm, grid->x, C, cells,
                                                           status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status band_plan(const WalkParams &W, int band_pts, long long n_bands, long long chunk,
                    unsigned long long *counts, long long *band_start, long long *item_start, uint32_t *order,
                    int sms, cudaStream_t st) {
  if (n_bands > 1) {
    RT_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)n_bands * sizeof(unsigned long long), st));
    const unsigned gb = (unsigned)std::min<unsigned long long>((W.n_rays + 255) / 256, 8ull * (unsigned)sms);
    k_band_count<<<gb, 256, 0, st>>>(W, band_pts, n_bands, counts);
    RT_CUDA_TRY(cudaGetLastError());
    // the counts are read by the plan, then the same words serve as the scatter cursors
    k_band_plan<<<1, 1024, 0, st>>>(counts, n_bands, W.n_rays, chunk, band_start, item_start, counts);
    RT_CUDA_TRY(cudaGetLastError());
    if (order) {
      k_band_scatter<<<gb, 256, 0, st>>>(W, band_pts, counts, order);
      RT_CUDA_TRY(cudaGetLastError());
    }
  } else {
    k_band_plan<<<1, 1024, 0, st>>>(nullptr, 1, W.n_rays, chunk, band_start, item_start, nullptr);
    RT_CUDA_TRY(cudaGetLastError());
  }
  return RT_OK;
}

rt_status trace_impl(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                     uint64_t ray_begin, uint64_t n_rays, uint64_t n_total, uint64_t seed,
                     uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                     const rt_record *record, cudaStream_t st) {
  if (!kappa) return fail(RT_E_INVAL, "kappa is NULL");
  WalkParams W;
  RecordPtrs rp;
  rt_status v = walk_setup(grid, spec, ray_begin, n_rays, n_total, seed, enclosure, flags, tally,
                           record, &W, &rp);
  if (v != RT_OK) return v;
  if (n_rays == 0) return RT_OK;
  Scratch scr;
  const int layout = walk_table_layout(spec->nT, spec->n_nu);
  const size_t cbytes = ((size_t)W.ncells * sizeof(float4) + 255) & ~size_t(255);
  const size_t tbytes = (walk_table_bytes(layout, spec->nT, spec->n_nu) + 255) & ~size_t(255);
  // rays grouped by wavenumber (one band per wavenumber): counts, band and item starts, order
  const bool group = n_rays <= 0xFFFFFFFFull &&
                     (g_walk_group == 2 || (g_walk_group == 0 && n_rays >= 32ull * (unsigned long long)spec->n_nu));
  const long long nb = spec->n_nu;
  const size_t pbytes = group ? (((size_t)nb * 8 * 3 + 64 + 255) & ~size_t(255)) : 0;
  const size_t obytes = group ? (size_t)n_rays * sizeof(uint32_t) : 0;
  v = scr.alloc(cbytes + tbytes + pbytes + obytes, st);
  if (v != RT_OK) return v;
  float4 *cells = scr.as<float4>();
  float *tabw = reinterpret_cast<float *>(scr.as<char>() + cbytes);
  v = cell_prep(grid, spec, cells, tally->status, st);
  if (v != RT_OK) return v;
  v = launch_walk_table(layout, kappa, spec->nT, spec->n_nu, tabw, st);
  if (v != RT_OK) return v;
  W.nu_major = layout;
  int dev = 0, sms = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint32_t *order = nullptr;
  if (group) {
    char *pb = scr.as<char>() + cbytes + tbytes;
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(pb);
    long long *band_start = reinterpret_cast<long long *>(counts + nb);
    long long *item_start = band_start + (nb + 1);
    order = reinterpret_cast<uint32_t *>(pb + pbytes);
    v = band_plan(W, 1, nb, 1LL << 40, counts, band_start, item_start, order, sms, st);
    if (v != RT_OK) return v;
  }
  const bool rec = rp.cells != nullptr;
  // visit recording (a test path) uses one configuration; the tuned shape otherwise
  auto pick = [&](auto tab) {
    constexpr int L = decltype(tab)::value;
    if (rec) return k_walk<true, L, 5, kRefillIdleDefault>;
    if (g_walk_blocks == 4) return g_walk_refill == 12 ? k_walk<false, L, 4, 12> : k_walk<false, L, 4, 16>;
    return g_walk_refill == 12 ? k_walk<false, L, 5, 12> : k_walk<false, L, 5, 16>;
  };
  auto kern = layout == 2 ? pick(std::integral_constant<int, 2>()) : pick(std::integral_constant<int, 1>());
  int per_sm = 0;
  RT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkThreads, 0));
  if (per_sm < 1) per_sm = 1;
  // persistent warps, each with a contiguous ray range of at least 64 rays
  unsigned long long want = (n_rays + 64ull * (kWalkThreads / 32) - 1) / (64ull * (kWalkThreads / 32));
  const unsigned long long cap = (unsigned long long)sms * (unsigned long long)per_sm;
  const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  kern<<<blocks, kWalkThreads, 0, st>>>(cells, tabw, order, W, tally->absorbed, tally->scalars, tally->steps,
                                        tally->status, rp);
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
