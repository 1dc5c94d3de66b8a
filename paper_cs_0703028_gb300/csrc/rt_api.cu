// Host-side plumbing of the C ABI: thread-local error messages, stream-ordered
// scratch, status words, Weideman coefficients.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rt_common.cuh"

namespace rt {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

rt_status fail(rt_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

rt_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();  // clear a sticky launch error of this thread, if any
  return (e == cudaErrorMemoryAllocation) ? RT_E_NOMEM : RT_E_CUDA;
}

static void configure_pool_once() {
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
    uint64_t keep = UINT64_MAX;  // keep freed scratch in the pool between calls
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  });
}

rt_status Scratch::alloc(size_t bytes, cudaStream_t stream) {
  configure_pool_once();
  s = stream;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    p = nullptr;
    return cuda_fail(e, "cudaMallocAsync(scratch)");
  }
  return RT_OK;
}

// Weideman (1994): with t = L tan(theta/2), expand
//   psi(theta) = exp(-t^2) (L^2 + t^2) = sum_n a_n exp(i n theta);
// then w(z) = 2 sum_{n>=0} a_{n+1} Z^n / (L - iz)^2 + (1/sqrt(pi)) / (L - iz),
// Z = (L + iz)/(L - iz), L = (N / sqrt 2)^(1/2).  The a_n are the trapezoidal
// Fourier coefficients on 2M = 4N equispaced angles (psi = 0 at theta = pi).
void weideman_coefficients(WeidCoef *out) {
  const int N = kWeidN, M = 2 * N;
  const double L = std::sqrt(N / std::sqrt(2.0));
  const double pi = 3.14159265358979323846;
  double psi[2 * M];
  double th[2 * M];
  for (int k = -M; k < M; ++k) {
    double theta = k * pi / M;
    th[k + M] = theta;
    if (k == -M) {
      psi[k + M] = 0.0;
    } else {
      double t = L * std::tan(theta / 2);
      psi[k + M] = std::exp(-t * t) * (L * L + t * t);
    }
  }
  out->L = (float)L;
  const double scale = 2.0 * std::sqrt(pi);
  for (int n = 1; n <= N; ++n) {
    double acc = 0.0;
    for (int k = 0; k < 2 * M; ++k) acc += psi[k] * std::cos(n * th[k]);
    out->a[n - 1] = (float)(scale * acc / (2 * M));
  }
}

}  // namespace rt

extern "C" {

const char *rt_version(void) { return "paper_cs_0703028_gb300 rt 0.1 (sm_103a)"; }

const char *rt_last_error(void) { return rt::g_err; }

size_t rt_kappa_table_elems(const rt_spectral *spec) {
  if (!spec || spec->nT < 1 || spec->n_nu < 1) return 0;
  return (size_t)spec->nT * (size_t)spec->n_nu;
}

}  // extern "C"

rt_status rt::status_from_bits(uint32_t bits) {
  if (bits & RT_DEV_NONFINITE) return rt::fail(RT_E_NONFINITE, "device: non-finite or non-positive input value");
  if (bits & RT_DEV_UNSORTED) return rt::fail(RT_E_UNSORTED, "device: line list not sorted by centre");
  if (bits & RT_DEV_STEPCAP) return rt::fail(RT_E_STEPCAP, "device: a ray exceeded its step cap");
  if (bits & RT_DEV_TIMEOUT) return rt::fail(RT_E_TIMEOUT, "device: a bounded wait ran out");
  if (bits & RT_DEV_COLUMN) return rt::fail(RT_E_INVAL, "device: index outside the table");
  return RT_OK;
}

extern "C" {

rt_status rt_status_read(const uint32_t *status, void *stream) {
  if (!status) return rt::fail(RT_E_INVAL, "rt_status_read: status is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t bits = 0;
  RT_CUDA_TRY(cudaMemcpyAsync(&bits, status, sizeof(bits), cudaMemcpyDeviceToHost, s));
  RT_CUDA_TRY(cudaStreamSynchronize(s));
  return rt::status_from_bits(bits);
}

rt_status rt_tally_zero(const rt_tally_buf *t, int64_t ncells, void *stream) {
  if (!t || !t->absorbed || !t->scalars || !t->steps || !t->status || ncells < 1)
    return rt::fail(RT_E_INVAL, "rt_tally_zero: bad tally buffer");
  cudaStream_t s = (cudaStream_t)stream;
  RT_CUDA_TRY(cudaMemsetAsync(t->absorbed, 0, sizeof(double) * (size_t)ncells, s));
  RT_CUDA_TRY(cudaMemsetAsync(t->scalars, 0, sizeof(double) * 4, s));
  RT_CUDA_TRY(cudaMemsetAsync(t->steps, 0, sizeof(unsigned long long), s));
  RT_CUDA_TRY(cudaMemsetAsync(t->status, 0, sizeof(uint32_t), s));
  return RT_OK;
}

}  // extern "C"
