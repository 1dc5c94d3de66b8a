// Many independent enclosures (grids of uneven size with their own fields, ray
// counts and tallies) traced in one persistent launch.  A plan holds, in device
// memory, each enclosure's walk parameters and the prefix sums of its work
// items (chunks of rays); the walk kernel's warps pull items from one atomic
// counter, so enclosures of every size keep all SMs busy.  Enclosure e draws
// its rays with Philox counter word 3 = e, exactly as rt_trace with
// enclosure = e, so the batched tallies equal per-enclosure traces.
//   k_cell_prep_batch : cell brackets of all enclosures (concatenated cells).
//   k_walk_batch      : persistent work-queue walk.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "rt_common.cuh"
#include "rt_walk.cuh"

namespace rt {

namespace {

struct EnclDev {
  WalkParams W;
  const float *T, *p, *x;
  double *absorbed, *scalars;
  unsigned long long *steps;
  uint32_t *status;
  long long cell_off;
  long long item_off;
  int has_px;
};

__device__ __forceinline__ int find_segment(const long long *off, int n, long long v) {
  int a = 0, b = n;  // last e with off[e] <= v
  while (b - a > 1) {
    const int m = (a + b) >> 1;
    if (off[m] <= v) a = m; else b = m;
  }
  return a;
}

__global__ void k_cell_prep_batch(const EnclDev *__restrict__ E, const long long *__restrict__ cell_off,
                                  int n_encl, long long total, CellParams C, float4 *__restrict__ cells) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int e = find_segment(cell_off, n_encl, g);
  const EnclDev &D = E[e];
  CellParams Ce = C;
  Ce.has_px = D.has_px;
  cells[g] = cell_prep_one(D.T, D.p, D.x, g - D.cell_off, Ce, D.status);
}

constexpr int kRefillIdleBatch = 16;
constexpr int kBatchUnroll = 4;

template <int TAB>
__global__ void __launch_bounds__(256, 4)
k_walk_batch(const EnclDev *__restrict__ E, const long long *__restrict__ item_off, int n_encl,
             long long n_items, int rays_per_item, const float4 *__restrict__ cells_all,
             const float *__restrict__ tab, unsigned long long *__restrict__ counter) {
  // the current item's enclosure (walk parameters and tally pointers), one slot
  // per warp, read like the constant bank
  __shared__ __align__(16) EnclDev s_e[8];
  __shared__ int4 s_axes[8][3];  // per warp slot: per axis {n, cell stride, h bits}
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const RecordPtrs rec{nullptr, nullptr, nullptr, nullptr, nullptr};
  const EnclDev &D = s_e[warp];
  const WalkParams &W = D.W;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((long long)it >= n_items) break;
    const int e = find_segment(item_off, n_encl, (long long)it);
    {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(E + e);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&s_e[warp]);
      for (int w = lane; w < (int)(sizeof(EnclDev) / 4); w += 32) dst[w] = src[w];
      __syncwarp();
      if (lane < 3)
        s_axes[warp][lane] = make_int4(W.n[lane], lane == 0 ? 1 : (lane == 1 ? W.n[0] : W.n[0] * W.n[1]),
                                       __float_as_int(W.h[lane]), 0);
      __syncwarp();
    }
    const float4 *cells = cells_all + D.cell_off;
    unsigned long long next = ((long long)it - D.item_off) * (unsigned long long)rays_per_item;
    const unsigned long long last = min(next + (unsigned long long)rays_per_item, W.n_rays);
    double em = 0.0, esc = 0.0;
    unsigned long long nsteps = 0;
    Ray R;
    float4 cd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // data of the ray's current cell
    const float2 *krow = nullptr;  // node-pair table: the ray's wavenumber row
    const float *krow1 = nullptr;  // wavenumber-major table: the ray's row
    bool active = false;
    for (;;) {
      const unsigned idle = __ballot_sync(0xffffffffu, !active);
      if (next < last && (idle == 0xffffffffu || __popc(idle) >= kRefillIdleBatch)) {
        const unsigned rank = __popc(idle & ((1u << lane) - 1u));
        if (!active && next + rank < last) {
          ray_init(W, cells, tab, next + rank, false, R, &cd);
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
        // every active lane dark: DDA-only steps
#pragma unroll
        for (int u = 0; u < kBatchUnroll; ++u)
          if (!done)
            done = ray_step<false, false, true, true>(W, 0.0f, D.absorbed, D.status, rec, R, true, NoPrefetch(),
                                                      s_axes[warp]);
      } else {
#pragma unroll
      for (int u = 0; u < kBatchUnroll; ++u) {  // steps per pass of the loop
        if (!done) {
          // a dark ray (transmission zero, no optical-depth cut) needs neither its cell's
          // kappa nor the next cell's data
          const bool lit = R.trans != 0.0f || W.tau_cut;
          const float kap = !lit ? 0.0f : (TAB == 2 ? cell_kappa_row(cd, krow) : (TAB == 1 ? cell_kappa_row1(cd, krow1, W.nT) : cell_kappa_l<TAB>(cd, tab, W.nT, W.n_nu, R.j)));
          float4 cdn = cd;
          done = ray_step<false, false, true>(W, kap, D.absorbed, D.status, rec, R, true,
                                              [&](int c) { if (lit) cdn = __ldg(cells + c); }, s_axes[warp]);
          cd = cdn;
        }
      }
      }
      if (done) {
        em += (double)R.w;
        esc += (double)(R.w * R.trans);
        nsteps += (unsigned long long)R.nv;
        active = false;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      em += __shfl_down_sync(0xffffffffu, em, o);
      esc += __shfl_down_sync(0xffffffffu, esc, o);
      nsteps += __shfl_down_sync(0xffffffffu, nsteps, o);
    }
    if (lane == 0) {
      if (em != 0.0) atomicAdd(D.scalars + 0, em);
      if (esc != 0.0) atomicAdd(D.scalars + 2, esc);
      if (nsteps) atomicAdd(D.steps, nsteps);
    }
    __syncwarp();  // the slot is rewritten by the next item
  }
}

}  // namespace

}  // namespace rt

struct rt_batch {
  int n_encl = 0;
  long long n_items = 0, total_cells = 0;
  int rays_per_item = 0, threads = 0;
  rt::CellParams C{};
  rt::EnclDev *d_encl = nullptr;
  long long *d_item_off = nullptr, *d_cell_off = nullptr;
  unsigned long long *d_counter = nullptr;
  float4 *d_cells = nullptr;
  float *d_tabt = nullptr;  // the walk's copy of the table (wavenumber-major or node pairs)
  int layout = 1;
  int nT = 0;
  long long n_nu = 0;
  void *mem = nullptr;
  cudaStream_t alloc_stream = nullptr;
  bool async_alloc = false;
  unsigned blocks = 0;
};

namespace rt {

static rt_status batch_build(int32_t n_encl, const rt_enclosure *encl, const rt_spectral *spec,
                             uint64_t seed, int32_t flags, const rt_batch_opts *opts, bool async,
                             cudaStream_t st, rt_batch **out) {
  if (!out) return fail(RT_E_INVAL, "rt_batch_create: out is NULL");
  *out = nullptr;
  if (n_encl < 1 || !encl) return fail(RT_E_INVAL, "rt_batch_create: need n_encl >= 1 enclosures");
  if ((flags & 0xF) != RT_SRC_EMIT) return fail(RT_E_INVAL, "rt_batch_create: only RT_SRC_EMIT");
  int rays_per_item = (opts && opts->rays_per_item > 0) ? opts->rays_per_item : 4096;
  int threads = (opts && opts->threads > 0) ? opts->threads : 256;
  if (threads % 32 != 0 || threads > 256) return fail(RT_E_INVAL, "rt_batch_create: threads must be a multiple of 32, <= 256");
  if (rays_per_item < 32) return fail(RT_E_INVAL, "rt_batch_create: rays_per_item must be >= 32");
  std::vector<EnclDev> H((size_t)n_encl);
  std::vector<long long> item_off((size_t)n_encl + 1), cell_off((size_t)n_encl + 1);
  long long items = 0, cells = 0;
  for (int e = 0; e < n_encl; ++e) {
    RecordPtrs rp;
    rt_status v = walk_setup(&encl[e].grid, spec, 0, encl[e].n_rays, encl[e].n_rays > 0 ? encl[e].n_rays : 1,
                             seed, (uint32_t)e, flags, &encl[e].tally, nullptr, &H[e].W, &rp);
    if (v != RT_OK) {
      char msg[384];
      snprintf(msg, sizeof(msg), "%s", rt_last_error());
      return fail(v, "enclosure %d: %s", e, msg);
    }
    H[e].W.nu_major = walk_table_layout(spec->nT, spec->n_nu);
    H[e].T = encl[e].grid.T;
    H[e].p = encl[e].grid.p_atm;
    H[e].x = encl[e].grid.x;
    H[e].has_px = (encl[e].grid.p_atm || encl[e].grid.x) ? 1 : 0;
    H[e].absorbed = encl[e].tally.absorbed;
    H[e].scalars = encl[e].tally.scalars;
    H[e].steps = encl[e].tally.steps;
    H[e].status = encl[e].tally.status;
    H[e].cell_off = cells;
    H[e].item_off = items;
    cell_off[e] = cells;
    item_off[e] = items;
    cells += H[e].W.ncells;
    items += (long long)((encl[e].n_rays + (uint64_t)rays_per_item - 1) / (uint64_t)rays_per_item);
  }
  cell_off[n_encl] = cells;
  item_off[n_encl] = items;
  const size_t b_encl = sizeof(EnclDev) * (size_t)n_encl;
  const size_t o_item = (b_encl + 255) & ~size_t(255);
  const size_t o_cell = (o_item + 8 * ((size_t)n_encl + 1) + 255) & ~size_t(255);
  const size_t o_cnt = (o_cell + 8 * ((size_t)n_encl + 1) + 255) & ~size_t(255);
  const size_t o_cells = o_cnt + 256;
  const size_t o_tabt = (o_cells + sizeof(float4) * (size_t)cells + 255) & ~size_t(255);
  const int layout = walk_table_layout(spec->nT, spec->n_nu);
  const size_t total = o_tabt + walk_table_bytes(layout, spec->nT, spec->n_nu);
  rt_batch *B = new rt_batch();
  cudaError_t ce = async ? cudaMallocAsync(&B->mem, total, st) : cudaMalloc(&B->mem, total);
  if (ce != cudaSuccess) {
    delete B;
    return cuda_fail(ce, "rt_batch_create: device tables");
  }
  B->async_alloc = async;
  B->alloc_stream = st;
  char *base = (char *)B->mem;
  B->d_encl = (EnclDev *)base;
  B->d_item_off = (long long *)(base + o_item);
  B->d_cell_off = (long long *)(base + o_cell);
  B->d_counter = (unsigned long long *)(base + o_cnt);
  B->d_cells = (float4 *)(base + o_cells);
  B->d_tabt = (float *)(base + o_tabt);
  B->nT = spec->nT;
  B->n_nu = spec->n_nu;
  B->layout = layout;
  B->n_encl = n_encl;
  B->n_items = items;
  B->total_cells = cells;
  B->rays_per_item = rays_per_item;
  B->threads = threads;
  B->C = cell_params(spec, 0, 0);
  cudaError_t e1 = cudaMemcpyAsync(B->d_encl, H.data(), b_encl, cudaMemcpyHostToDevice, st);
  cudaError_t e2 = cudaMemcpyAsync(B->d_item_off, item_off.data(), 8 * ((size_t)n_encl + 1), cudaMemcpyHostToDevice, st);
  cudaError_t e3 = cudaMemcpyAsync(B->d_cell_off, cell_off.data(), 8 * ((size_t)n_encl + 1), cudaMemcpyHostToDevice, st);
  cudaError_t e4 = async ? cudaSuccess : cudaStreamSynchronize(st);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
    if (async) cudaFreeAsync(B->mem, st); else cudaFree(B->mem);
    delete B;
    return cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4)),
                     "rt_batch_create: upload");
  }
  int dev = 0, sms = 0, per_sm = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, layout == 2 ? k_walk_batch<2> : k_walk_batch<1>, threads, 0));
  if (per_sm < 1) per_sm = 1;
  B->blocks = (unsigned)(sms * per_sm);
  *out = B;
  return RT_OK;
}

static rt_status batch_run(rt_batch *B, const float *kappa, cudaStream_t st) {
  if (!B || !kappa) return fail(RT_E_INVAL, "rt_batch_trace: NULL plan or kappa");
  rt_status v = RT_OK;
  RT_CUDA_TRY(cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned long long), st));
  if (B->total_cells > 0) {
    k_cell_prep_batch<<<(unsigned)((B->total_cells + 255) / 256), 256, 0, st>>>(
        B->d_encl, B->d_cell_off, B->n_encl, B->total_cells, B->C, B->d_cells);
    RT_CUDA_TRY(cudaGetLastError());
  }
  v = launch_walk_table(B->layout, kappa, B->nT, B->n_nu, B->d_tabt, st);
  if (v != RT_OK) return v;
  auto kern = B->layout == 2 ? k_walk_batch<2> : k_walk_batch<1>;
  kern<<<B->blocks, B->threads, 0, st>>>(B->d_encl, B->d_item_off, B->n_encl, B->n_items,
                                         B->rays_per_item, B->d_cells, B->d_tabt, B->d_counter);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

extern "C" {

rt_status rt_batch_create(int32_t n_encl, const rt_enclosure *encl, const rt_spectral *spec,
                          uint64_t seed, int32_t flags, const rt_batch_opts *opts, rt_batch **out) {
  return rt::batch_build(n_encl, encl, spec, seed, flags, opts, false, nullptr, out);
}

rt_status rt_batch_trace(rt_batch *plan, const float *kappa, void *stream) {
  return rt::batch_run(plan, kappa, (cudaStream_t)stream);
}

rt_status rt_batch_destroy(rt_batch *plan) {
  if (!plan) return RT_OK;
  cudaError_t e = plan->async_alloc ? cudaFreeAsync(plan->mem, plan->alloc_stream) : cudaFree(plan->mem);
  delete plan;
  if (e != cudaSuccess) return rt::cuda_fail(e, "rt_batch_destroy");
  return RT_OK;
}

rt_status rt_trace_batch(int32_t n_encl, const rt_enclosure *encl, const float *kappa,
                         const rt_spectral *spec, uint64_t seed, int32_t flags,
                         const rt_batch_opts *opts, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  rt_batch *B = nullptr;
  rt_status v = rt::batch_build(n_encl, encl, spec, seed, flags, opts, true, st, &B);
  if (v != RT_OK) return v;
  v = rt::batch_run(B, kappa, st);
  rt_status d = rt_batch_destroy(B);
  return v != RT_OK ? v : d;
}

}  // extern "C"
