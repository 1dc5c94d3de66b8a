// Measured ALU ceilings for the line sum's roofline: binary32 FMA and MUFU
// reciprocal throughput in lane operations per second, from kernels of
// independent chains that fill every SM (no memory traffic inside the loop; the
// reciprocal chain interleaves one add per reciprocal, on the FMA pipe).
#include <cmath>

#include "rt_common.cuh"
#include "rt_tc.cuh"

namespace rt {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent chains per thread
constexpr int kProbeIters = 16384;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float b, float c, float *out) {
  float a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[i]) : "f"(b), "f"(c));
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_rcp_probe(float *out) {
  float a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = 1.0f + (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it)
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i)  // the add keeps consecutive reciprocals from cancelling
      asm volatile("{\n rcp.approx.ftz.f32 %0, %0;\n add.rn.f32 %0, %0, 0f3A83126F;\n}" : "+f"(a[i]));
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The bounded-wait path the library's kernels take when a copy or a product never
// completes: one mbarrier that expects one arrival, waited on with the bounded
// try-wait loop of the tensor-core kernels (tc::mbar_wait) for `limit` iterations.
// With arrive = 0 nothing arrives, the wait gives up, and the status word receives
// RT_DEV_TIMEOUT, as a timed-out kernel reports it; with arrive = 1 thread 0 arrives
// first and the wait succeeds.
__global__ void k_wait_probe(uint32_t limit, int arrive, uint32_t *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(&bar)) : "memory");
  __syncthreads();
  const int ok = tc::mbar_wait(&bar, 0, limit) ? 1 : 0;
  if (!__syncthreads_and(ok) && threadIdx.x == 0) status_or(status, RT_DEV_TIMEOUT);
}

}  // namespace

rt_status wait_probe(uint32_t limit, int32_t arrive, uint32_t *status, cudaStream_t st) {
  if (!status) return fail(RT_E_INVAL, "rt_wait_probe: status is NULL");
  if (limit < 1 || limit > (1u << 24)) return fail(RT_E_INVAL, "rt_wait_probe: limit must be in [1, 2^24]");
  k_wait_probe<<<1, 32, 0, st>>>(limit, arrive ? 1 : 0, status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status alu_probe(double *out, cudaStream_t st) {
  if (!out) return fail(RT_E_INVAL, "rt_alu_probe: out is NULL");
  int dev = 0, sms = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = (unsigned)sms * 8u;  // 8 blocks of 256 threads per SM: full occupancy
  Scratch scr;
  rt_status v = scr.alloc((size_t)blocks * kProbeThreads * sizeof(float), st);
  if (v != RT_OK) return v;
  float *sink = scr.as<float>();
  cudaEvent_t e0, e1;
  RT_CUDA_TRY(cudaEventCreate(&e0));
  RT_CUDA_TRY(cudaEventCreate(&e1));
  const double ops = (double)blocks * kProbeThreads * kProbeChains * kProbeIters;
  for (int kind = 0; kind < 2; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, st);
      if (kind == 0)
        k_fma_probe<<<blocks, kProbeThreads, 0, st>>>(0.999f, 1e-3f, sink);
      else
        k_rcp_probe<<<blocks, kProbeThreads, 0, st>>>(sink);
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "rt_alu_probe");
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
    out[kind] = ops / (best * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

extern "C" rt_status rt_alu_probe(double *out, void *stream) {
  return rt::alu_probe(out, (cudaStream_t)stream);
}

extern "C" rt_status rt_wait_probe(uint32_t limit, int32_t arrive, uint32_t *status, void *stream) {
  return rt::wait_probe(limit, arrive, status, (cudaStream_t)stream);
}
