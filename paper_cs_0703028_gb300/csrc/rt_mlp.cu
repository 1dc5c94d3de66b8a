// Surrogate network for kappa: (log nu, T, p, x) -> log kappa, an MLP
// 4 -> 128 -> 128 -> 128 -> 128 -> 1 with SiLU, trained and evaluated in BF16
// on the fifth-generation tensor cores with FP32 accumulation in tensor memory.
//   k_mlp_prep : FP32 master weights -> BF16 tiles in the K-major core-matrix
//                layout (W2..W4 and their transposes), ready for bulk copies.
//   k_mlp_fwd  : per 128-row tile, layer 1 on the CUDA cores, layers 2..4 as
//                128x128x128 tcgen05 products with a bias + SiLU epilogue read
//                from tensor memory, linear head; for training also the
//                pre-activations, the output gradient and the loss.
//   k_mlp_bwd  : per 128-row tile, for each of layers 4..2 two tcgen05 products
//                (dW = dZ^T H, dH = dZ W), SiLU derivative epilogues, bias and
//                first-layer gradients, written to the tile's own FP32 partial.
//   k_grad_adam : the gradient, the tiles' partials summed in tile order, and
//                the Adam update of the FP32 masters (Kingma and Ba); within a
//                run of steps also the next step's BF16 tiles.
//   k_walk_mlp : the Monte-Carlo walk with the network in place of the table
//                (three 128-ray tiles per block; every layer, biases included,
//                on the tensor cores).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "rt_common.cuh"
#include "rt_tc.cuh"
#include "rt_walk.cuh"

namespace rt {
namespace {

constexpr int kH = 128;
constexpr double kPiD = 3.14159265358979323846;
constexpr int kNParam = 50305;
constexpr int oW1 = 0, oB1 = 512, oW2 = 640, oB2 = 17024, oW3 = 17152, oB3 = 33536, oW4 = 33664,
              oB4 = 50048, oW5 = 50176, oB5 = 50304;
constexpr int kGradStride = (kNParam + 15) & ~15;  // per-tile gradient partials, 64-byte rows
constexpr int kTileElems = kH * kH;           // 16384 bf16 = 32 KB
constexpr uint32_t kTileBytes = kTileElems * 2;
constexpr uint32_t kWaitLimit = 1u << 24;

struct Norm {
  float lo[4], hi[4], mean, scale;
};
static_assert(sizeof(Norm) == sizeof(rt_mlp_norm), "Norm must have the layout of rt_mlp_norm");

// Network `net` of an ensemble with per-network norms in device memory (norms),
// or the one network of a call that passed its norm by value (norms == nullptr).
__device__ __forceinline__ Norm net_norm(const Norm *__restrict__ norms, const Norm &single, int net) {
  return norms ? norms[net] : single;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigmoid_fast(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }

// Training pre-activations Z[layer][unit][sample] (n samples): the 32 lanes of a
// warp hold consecutive samples, so their accesses to one unit are coalesced.
__device__ __forceinline__ long long zidx(long long layer, int c, long long n, long long row) {
  return (layer * kH + c) * n + row;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// bf16 element (r, k) of a K-major 128x128 tile (in units of 2-byte elements)
__device__ __forceinline__ int tile_index(int r, int k) { return (int)(tc::kmajor_offset(r, k, kH) >> 1); }

__global__ void k_mlp_prep(const float *__restrict__ P, uint16_t *__restrict__ tiles, int n_mats) {
  const int m = blockIdx.y;  // 0..2: W2..W4 (rows = out), 3..5: transposes (rows = in)
  const long long net = blockIdx.z;
  P += net * kNParam;
  tiles += net * n_mats * kTileElems;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kTileElems) return;
  const int r = idx / kH, k = idx % kH;
  const int base = (m % 3 == 0) ? oW2 : (m % 3 == 1 ? oW3 : oW4);
  const float w = (m < 3) ? P[base + r * kH + k] : P[base + k * kH + r];
  tiles[m * kTileElems + tile_index(r, k)] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

__device__ __forceinline__ void normalise(const float *__restrict__ in, long long row, bool valid,
                                          const Norm &N, float (&u)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float v = valid ? in[row * 4 + i] : N.lo[i];
    u[i] = 2.0f * (v - N.lo[i]) / (N.hi[i] - N.lo[i]) - 1.0f;
  }
}

// FP32 parameters used on the CUDA cores (layer 1, biases, head), staged once
// per block so that each use is a shared-memory (float4) read.
struct SmallParams {
  float4 w1[kH];      // W1 rows
  float b1[kH];
  float b[3][kH];     // b2, b3, b4
  float w5[kH];
  float b5;
};

__device__ __forceinline__ void stage_small(SmallParams &S, const float *__restrict__ P) {
  for (int c = threadIdx.x; c < kH; c += blockDim.x) {
    S.w1[c] = make_float4(P[oW1 + 4 * c], P[oW1 + 4 * c + 1], P[oW1 + 4 * c + 2], P[oW1 + 4 * c + 3]);
    S.b1[c] = P[oB1 + c];
    S.b[0][c] = P[oB2 + c];
    S.b[1][c] = P[oB3 + c];
    S.b[2][c] = P[oB4 + c];
    S.w5[c] = P[oW5 + c];
  }
  if (threadIdx.x == 0) S.b5 = P[oB5];
}

__device__ __forceinline__ float layer1(const SmallParams &S, int c, const float (&u)[4]) {
  const float4 w = S.w1[c];
  return fmaf(w.w, u[3], fmaf(w.z, u[2], fmaf(w.y, u[1], fmaf(w.x, u[0], S.b1[c]))));
}

// Two weight buffers: W2 and W3 are copied at the start, W4 into the first buffer
// once the product with W2 has completed.  About 101 KB in all, so that two blocks
// share an SM.
struct FwdSmem {
  uint16_t W[2][kTileElems];  // layer l's weights (rows = out) in buffer l mod 2
  uint16_t A[kTileElems];     // current layer input, rows = samples
  SmallParams sp;
  uint64_t bar_w[2], bar_mma;
  uint32_t tmem;
  float red[4];
  float yh[kH];               // the head's partial sum over the second half of the units
};

// Two threads per sample row, as in the backward pass: thread t takes row t mod 128
// and half t / 128 of the units of every layer.
constexpr int kFwdThreads = 2 * kH;

// Networks of an ensemble along grid.y: network `net` reads its parameters, tiles,
// samples (n rows at net * in_stride) and activations at net times the per-network
// strides.
template <bool TRAIN>
__global__ void __launch_bounds__(kFwdThreads, 2)
k_mlp_fwd(const float *__restrict__ P, const uint16_t *__restrict__ tiles, long long tile_stride, Norm N1,
          const Norm *__restrict__ norms, const float *__restrict__ inputs, const float *__restrict__ targets,
          long long n, long long in_stride, float *__restrict__ Z, float *__restrict__ dy,
          float *__restrict__ loss, float loss_scale, float *__restrict__ out, uint32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  FwdSmem &S = *reinterpret_cast<FwdSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long net = blockIdx.y;
  const Norm N = net_norm(norms, N1, (int)net);
  P += net * kNParam;
  tiles += net * tile_stride;
  inputs += net * in_stride * 4;  // the network's n rows of samples (in_stride rows apart)
  if (TRAIN) {
    targets += net * in_stride;
    Z += net * 4 * kH * n;
    dy += net * n;
  } else {
    out += net * in_stride;
  }
  const int r = tid & (kH - 1);          // sample row within the tile
  const int cb = (tid >> 7) * (kH / 2);  // first unit of the thread's half
  const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;  // the warp's tensor-memory lanes
  const long long row = (long long)blockIdx.x * kH + r;
  const bool valid = row < n;

  if (tid == 0) {
    tc::mbar_init(&S.bar_w[0], 1);
    tc::mbar_init(&S.bar_w[1], 1);
    tc::mbar_init(&S.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(&S.tmem, kH);
  stage_small(S.sp, P);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem;
  bool w4_issued = false;  // thread 0: the copy of W4 is in flight or done
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      tc::mbar_arrive_expect_tx(&S.bar_w[b], kTileBytes);
      tc::bulk_g2s(&S.W[b][0], tiles + b * kTileElems, kTileBytes, &S.bar_w[b]);
    }
  }

  // layer 1 on the CUDA cores
  float u[4];
  normalise(inputs, row, valid, N, u);
#pragma unroll 1
  for (int c0 = cb; c0 < cb + kH / 2; c0 += 8) {
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + i;
      const float z = layer1(S.sp, c, u);
      if (TRAIN && valid) Z[zidx(0, c, n, row)] = z;
      h[i] = z * sigmoid_fast(z);
    }
    uint4 pk = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                          pack_bf16x2(h[6], h[7]));
    *reinterpret_cast<uint4 *>(&S.A[tile_index(r, c0)]) = pk;
  }
  int timeout = 0;
  int mma_pending = -1;  // parity of a product whose completion wait gave up

  float y = 0.0f;
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    timeout = tc::mbar_wait(&S.bar_w[l & 1], (uint32_t)(l >> 1), kWaitLimit) ? 0 : 1;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    if (__syncthreads_or(timeout)) {  // timeout block-uniform from here on
      timeout = 1;
      break;
    }
    if (tid == 0) {
      tc::fence_after_sync();
      tc::mma_128x128x128(tmem, S.A, S.W[l & 1]);
      tc::mma_commit(&S.bar_mma);
    }
    timeout = tc::mbar_wait(&S.bar_mma, (uint32_t)(l & 1), kWaitLimit) ? 0 : 1;
    if (__syncthreads_or(timeout)) {
      timeout = 1;
      mma_pending = l & 1;
      break;
    }
    tc::fence_after_sync();
    if (l == 0 && tid == 0) {  // W4 into the buffer the finished product read
      tc::mbar_arrive_expect_tx(&S.bar_w[0], kTileBytes);
      tc::bulk_g2s(&S.W[0][0], tiles + 2 * kTileElems, kTileBytes, &S.bar_w[0]);
      w4_issued = true;
    }
    const float *bias = S.sp.b[l];
#pragma unroll 1
    for (int c0 = cb; c0 < cb + kH / 2; c0 += 32) {
      float acc[32];
      tc::tmem_ld32(tmem + lanes + (uint32_t)c0, acc);
#pragma unroll
      for (int i = 0; i < 32; i += 8) {
        float h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = c0 + i + q;
          const float z = acc[i + q] + bias[c];
          if (TRAIN && valid) Z[zidx(l + 1, c, n, row)] = z;
          h[q] = z * sigmoid_fast(z);
          if (l == 2) y = fmaf(S.sp.w5[c], h[q], y);
        }
        if (l < 2) {
          uint4 pk = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                                pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
          *reinterpret_cast<uint4 *>(&S.A[tile_index(r, c0 + i)]) = pk;
        }
      }
    }
  }
  if (timeout) {
    if (tid == 0) {
      status_or(status, RT_DEV_TIMEOUT);
      // a weight copy or a product may still be in flight: let it land (bounded)
      // before the block releases its shared and tensor memory
      tc::mbar_wait(&S.bar_w[0], 0, kWaitLimit);
      tc::mbar_wait(&S.bar_w[1], 0, kWaitLimit);
      if (w4_issued) tc::mbar_wait(&S.bar_w[0], 1, kWaitLimit);
      if (mma_pending >= 0) tc::mbar_wait(&S.bar_mma, (uint32_t)mma_pending, kWaitLimit);
    }
  }
  if (!timeout && cb != 0) S.yh[r] = y;
  __syncthreads();
  if (!timeout && cb == 0) {
    y += S.yh[r];
    y += S.sp.b5;
    if (TRAIN) {
      const float ts = valid ? (targets[row] - N.mean) / N.scale : 0.0f;
      const float res = valid ? (y - ts) : 0.0f;
      if (valid) dy[row] = res / (float)n;
      float l2 = 0.5f * res * res / (float)n * loss_scale;
      for (int o = 16; o > 0; o >>= 1) l2 += __shfl_down_sync(0xffffffffu, l2, o);
      if (lane == 0) S.red[warp] = l2;
    } else if (valid) {
      out[row] = N.mean + N.scale * y;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (TRAIN && tid == 0 && !timeout) atomicAdd(loss, S.red[0] + S.red[1] + S.red[2] + S.red[3]);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kH);
  }
}

// dZ and H are written one row per sample (16-byte stores of 8 units) and serve
// both products: dZ K-major as the A operand of dH = dZ W, and dZ, H read MN-major
// (as their transposes) for dW = dZ^T H.  Column sums over the tile's samples (bias
// and first-layer gradients) are reduced by warp shuffles into per-row-quarter
// partials; about 110 KB in all, so that two blocks share an SM.
struct BwdSmem {
  uint16_t dZ[kTileElems];   // rows = samples, k = out
  uint16_t H[kTileElems];    // rows = samples, k = in
  uint16_t Wt[kTileElems];   // current layer's transposed weights, rows = in
  float colred[5][4][kH];    // [bias, dW1 k = 0..3][row quarter][unit] partial sums
  float dyred[4];            // per row quarter: sum of dy
  uint64_t bar_w, bar_mma;
  uint32_t tmem;
};

__device__ __forceinline__ void put_bf16(uint16_t *tile, int r, int k, float v) {
  tile[tile_index(r, k)] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// elements (r, k0 .. k0 + 7) of a K-major tile (k0 a multiple of 8): one 16-byte store
__device__ __forceinline__ void put_bf16x8(uint16_t *tile, int r, int k0, const float *v) {
  *reinterpret_cast<uint4 *>(&tile[tile_index(r, k0)]) =
      make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                 pack_bf16x2(v[6], v[7]));
}

// v: this lane's values of 16 consecutive columns (its row).  Returns, in every
// lane, the sum over the warp's 32 rows of column (lane & 15): four halving
// exchange steps leave each lane one column summed over its 16-lane half, the last
// step adds the two halves.  A fixed tree, so the sum is deterministic.  v is clobbered.
__device__ __forceinline__ float warp_column_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 8, h = 8; o >= 1; o >>= 1, h >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = upper ? v[i] : v[i + h];
      const float keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Two threads per sample row: thread t takes row t mod 128 (its warp reads that
// row's tensor-memory lane) and half t / 128 of the 128 units, in chunks of 16.
constexpr int kBwdThreads = 2 * kH;
constexpr int kBwdChunk = 16;

__global__ void __launch_bounds__(kBwdThreads, 2)
k_mlp_bwd(const float *__restrict__ P, const uint16_t *__restrict__ tiles, long long tile_stride, Norm N1,
          const Norm *__restrict__ norms, const float *__restrict__ inputs, long long n, long long in_stride,
          const float *__restrict__ Z, const float *__restrict__ dy, float *__restrict__ Gpart,
          uint32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  BwdSmem &S = *reinterpret_cast<BwdSmem *>(smem_raw);
  const long long net = blockIdx.y;  // network of an ensemble (strides as in k_mlp_fwd)
  const Norm N = net_norm(norms, N1, (int)net);
  P += net * kNParam;
  tiles += net * tile_stride;
  inputs += net * in_stride * 4;
  Z += net * 4 * kH * n;
  dy += net * n;
  // this tile's gradient partial (every parameter written exactly once; summed over
  // the tiles in a fixed order by k_grad_adam)
  float *G = Gpart + (net * gridDim.x + blockIdx.x) * kGradStride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & (kH - 1);          // sample row within the tile
  const int q4 = warp & 3;               // row quarter = the warp's tensor-memory lanes
  const int cb = (tid >> 7) * (kH / 2);  // first unit of the thread's half
  const uint32_t lanes = (uint32_t)(q4 * 32) << 16;
  const long long row = (long long)blockIdx.x * kH + r;
  const bool valid = row < n;

  if (tid == 0) {
    tc::mbar_init(&S.bar_w, 1);
    tc::mbar_init(&S.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(&S.tmem, 2 * kH);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem;
  if (tid == 0) {  // W4^T first
    tc::mbar_arrive_expect_tx(&S.bar_w, kTileBytes);
    tc::bulk_g2s(S.Wt, tiles + 5 * kTileElems, kTileBytes, &S.bar_w);
  }
  float u[4];
  normalise(inputs, row, valid, N, u);
  const float dyv = valid ? dy[row] : 0.0f;
  if (tid < kH) {  // db5 = sum_s dy, per row quarter
    float d = dyv;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) S.dyred[q4] = d;
  }

  // head: dw5 = sum_s dy h4
#pragma unroll 1
  for (int c0 = cb; c0 < cb + kH / 2; c0 += kBwdChunk) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z4 = valid ? Z[zidx(3, c0 + i, n, row)] : 0.0f;
      v[i] = dyv * z4 * sigmoid_fast(z4);
    }
    const float cs = warp_column_sum16(v, lane);
    if (lane < 16) S.colred[0][q4][c0 + lane] = cs;
  }
  __syncthreads();
  if (tid < kH) G[oW5 + tid] = S.colred[0][0][tid] + S.colred[0][1][tid] + S.colred[0][2][tid] + S.colred[0][3][tid];
  if (tid == 0) G[oB5] = S.dyred[0] + S.dyred[1] + S.dyred[2] + S.dyred[3];
  __syncthreads();
  // dz4 = dy w5 silu'(z4) -> dZ and db4; h3 -> H (for dW4)
#pragma unroll 1
  for (int c0 = cb; c0 < cb + kH / 2; c0 += kBwdChunk) {
    float dz[16], h[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float z4 = valid ? Z[zidx(3, c0 + i, n, row)] : 0.0f;
      const float z3 = valid ? Z[zidx(2, c0 + i, n, row)] : 0.0f;
      const float s4 = sigmoid_fast(z4);
      dz[i] = dyv * __ldg(P + oW5 + c0 + i) * (s4 * (1.0f + z4 * (1.0f - s4)));
      h[i] = z3 * sigmoid_fast(z3);
    }
    put_bf16x8(S.dZ, r, c0, dz);
    put_bf16x8(S.dZ, r, c0 + 8, dz + 8);
    put_bf16x8(S.H, r, c0, h);
    put_bf16x8(S.H, r, c0 + 8, h + 8);
    const float cs = warp_column_sum16(dz, lane);
    if (lane < 16) S.colred[0][q4][c0 + lane] = cs;
  }
  __syncthreads();
  if (tid < kH) G[oB4 + tid] = S.colred[0][0][tid] + S.colred[0][1][tid] + S.colred[0][2][tid] + S.colred[0][3][tid];

  int timeout = 0;
  bool aborted = false;
  uint32_t wphase = 0;
  int w_pending = -1, mma_pending = -1;  // parities of a copy / products whose wait gave up
#pragma unroll 1
  for (int l = 4; l >= 2; --l) {
    // W_l (rows = out) maps h_{l-1} -> z_l
    if (!tc::mbar_wait(&S.bar_w, wphase, kWaitLimit)) timeout = 1;
    wphase ^= 1u;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    if (__syncthreads_or(timeout)) {
      w_pending = (int)(wphase ^ 1u);
      aborted = true;
      break;
    }
    if (tid == 0) {
      tc::fence_after_sync();
      tc::mma_128x128x128_mn(tmem, S.dZ, S.H);       // dW_l[out][in] = dZ^T H
      tc::mma_128x128x128(tmem + kH, S.dZ, S.Wt);    // dH_{l-1}[sample][in]
      tc::mma_commit(&S.bar_mma);
    }
    timeout = tc::mbar_wait(&S.bar_mma, (uint32_t)((4 - l) & 1), kWaitLimit) ? 0 : 1;
    if (__syncthreads_or(timeout)) {
      mma_pending = (4 - l) & 1;
      aborted = true;
      break;
    }
    tc::fence_after_sync();
    if (tid == 0 && l > 2) {  // next transposed weights into the now free buffer
      tc::mbar_arrive_expect_tx(&S.bar_w, kTileBytes);
      tc::bulk_g2s(S.Wt, tiles + (l == 4 ? 4 : 3) * kTileElems, kTileBytes, &S.bar_w);
    }
    float *gW = G + (l == 4 ? oW4 : (l == 3 ? oW3 : oW2));
    const long long zl = (long long)(l - 2);  // block of z_{l-1}
#pragma unroll 1
    for (int c0 = cb; c0 < cb + kH / 2; c0 += kBwdChunk) {
      // this chunk's pre-activations first, so that their loads overlap the
      // tensor-memory reads below
      float z[16], zp[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        z[i] = valid ? Z[zidx(zl, c0 + i, n, row)] : 0.0f;
        zp[i] = (valid && l > 2) ? Z[zidx(zl - 1, c0 + i, n, row)] : 0.0f;
      }
      float acc[16];
      tc::tmem_ld16(tmem + lanes + (uint32_t)c0, acc);
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        *reinterpret_cast<float4 *>(gW + r * kH + c0 + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
      tc::tmem_ld16(tmem + lanes + (uint32_t)(kH + c0), acc);
      float dz[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float s = sigmoid_fast(z[i]);
        dz[i] = acc[i] * (s * (1.0f + z[i] * (1.0f - s)));
      }
      if (l > 2) {
        float h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = zp[i] * sigmoid_fast(zp[i]);
        put_bf16x8(S.dZ, r, c0, dz);
        put_bf16x8(S.dZ, r, c0 + 8, dz + 8);
        put_bf16x8(S.H, r, c0, h);
        put_bf16x8(S.H, r, c0 + 8, h + 8);
      }
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = dz[i];
      float cs = warp_column_sum16(v, lane);
      if (lane < 16) S.colred[0][q4][c0 + lane] = cs;
      if (l == 2) {  // first layer: dW1[c][k] = sum_s dz1[s][c] u[s][k]
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = dz[i] * u[k];
          cs = warp_column_sum16(v, lane);
          if (lane < 16) S.colred[1 + k][q4][c0 + lane] = cs;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    const int ob = (l == 4 ? oB3 : (l == 3 ? oB2 : oB1));
    if (tid < kH) G[ob + tid] = S.colred[0][0][tid] + S.colred[0][1][tid] + S.colred[0][2][tid] + S.colred[0][3][tid];
    if (l == 2 && tid < kH) {
      float g[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        g[k] = S.colred[1 + k][0][tid] + S.colred[1 + k][1][tid] + S.colred[1 + k][2][tid] + S.colred[1 + k][3][tid];
      *reinterpret_cast<float4 *>(G + oW1 + tid * 4) = make_float4(g[0], g[1], g[2], g[3]);
    }
  }
  if (aborted && tid == 0) {  // some thread's wait gave up; let what is still in flight land (bounded)
    status_or(status, RT_DEV_TIMEOUT);
    if (w_pending >= 0) tc::mbar_wait(&S.bar_w, (uint32_t)w_pending, kWaitLimit);
    if (mma_pending >= 0) tc::mbar_wait(&S.bar_mma, (uint32_t)mma_pending, kWaitLimit);
  }
  if (aborted) {  // block-uniform: the partial holds no gradient of this tile
    __syncthreads();  // the other threads' partial writes are done before the zeros
    for (int i = tid; i < kNParam; i += kBwdThreads) G[i] = 0.0f;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kH);
  }
}

// gradient = sum of the tiles' partials, in tile order (deterministic), and
// unless `adam` is 0 the Adam update of the FP32 masters with it (Kingma and Ba);
// with `tiles` given, an updated weight of W2..W4 is also written to its two BF16
// tile positions (the layout k_mlp_prep writes), ready for the next step.  The
// gradient itself is stored only when grad is not NULL (within a run of steps,
// only the last step's).  Each thread takes PER parameters kAdamThreads apart,
// all their loads issued before the first update (PER = 4 for an ensemble of at
// least kAdamWide networks, else 1, so that a single network still fills the GPU).
constexpr int kAdamThreads = 256, kAdamWide = 64;

__device__ __forceinline__ void adam_tile_write(uint16_t *__restrict__ tiles, int i, float w) {
  const int mat = (i >= oW2 && i < oW2 + kTileElems) ? 0
                  : (i >= oW3 && i < oW3 + kTileElems) ? 1
                  : (i >= oW4 && i < oW4 + kTileElems) ? 2 : -1;
  if (mat >= 0) {
    const int e = i - (mat == 0 ? oW2 : (mat == 1 ? oW3 : oW4));
    const int r = e / kH, k = e % kH;  // row (output unit), column (input unit)
    const uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(w));
    tiles[mat * kTileElems + tile_index(r, k)] = h;
    tiles[(mat + 3) * kTileElems + tile_index(k, r)] = h;
  }
}

template <int PER>
__global__ void __launch_bounds__(kAdamThreads)
k_grad_adam(const float *__restrict__ part, int nparts, float *__restrict__ grad, int adam,
            float *__restrict__ P, float *__restrict__ m, float *__restrict__ v, float lr, float b1, float b2,
            float eps, float c1, float c2, uint16_t *__restrict__ tiles) {
  const int i0 = blockIdx.x * (kAdamThreads * PER) + threadIdx.x;
  const long long net = blockIdx.y;  // network of an ensemble: its partials, parameters, moments, tiles
  part += net * nparts * kGradStride;
  if (grad) grad += net * kNParam;
  P += net * kNParam;
  if (adam) {
    m += net * kNParam;
    v += net * kNParam;
  }
  if (tiles) tiles += net * 6 * kTileElems;
  if (PER == 1) {  // one parameter per thread (few networks, many tile partials each)
    const int i = i0;
    if (i >= kNParam) return;
    float gi = 0.0f;
    for (int t = 0; t < nparts; ++t) gi += part[(long long)t * kGradStride + i];
    if (grad) grad[i] = gi;
    if (!adam) return;
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float pi = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    P[i] = pi;
    if (tiles) adam_tile_write(tiles, i, pi);
    return;
  }
  // out-of-range slots read the last parameter (a valid address, no branch in the
  // loads) and store nothing
  int ix[PER];
  float g[PER], pv[PER], mv[PER], vv[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    ix[q] = min(i0 + q * kAdamThreads, kNParam - 1);
    g[q] = part[ix[q]];
    if (adam) {
      pv[q] = P[ix[q]];
      mv[q] = m[ix[q]];
      vv[q] = v[ix[q]];
    }
  }
#pragma unroll 4
  for (int t = 1; t < nparts; ++t) {
#pragma unroll
    for (int q = 0; q < PER; ++q) g[q] += part[(long long)t * kGradStride + ix[q]];
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = i0 + q * kAdamThreads;
    if (i >= kNParam) continue;
    if (grad) grad[i] = g[q];
    if (!adam) continue;
    const float mi = fmaf(b1, mv[q], (1.0f - b1) * g[q]);
    const float vi = fmaf(b2, vv[q], (1.0f - b2) * g[q] * g[q]);
    m[i] = mi;
    v[i] = vi;
    const float pi = pv[q] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    P[i] = pi;
    if (tiles) adam_tile_write(tiles, i, pi);
  }
}

// Self-test of the tensor-core path: D = A B^T for 128 x 128 x 128, A and B
// given as FP32 row-major [128][128] (rounded to bf16); with MN, D = A^T B with
// both tiles read MN-major (the backward pass's weight-gradient product).  The MN
// form keeps each tile 64 KB apart from the next member, so that a product reading
// past its 32 KB tile stays inside the block's shared memory.
template <bool MN>
__global__ void __launch_bounds__(128)
k_tc_selftest(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ D,
              uint32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int kGap = MN ? 2 * kTileElems : kTileElems;
  uint16_t *sA = reinterpret_cast<uint16_t *>(smem_raw);
  uint16_t *sB = sA + kGap;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + kGap);
  uint32_t *holder = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(holder, kH);
  for (int k = 0; k < kH; ++k) {
    put_bf16(sA, tid, k, A[tid * kH + k]);
    put_bf16(sB, tid, k, B[tid * kH + k]);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *holder;
  if (tid == 0) {
    if (MN) tc::mma_128x128x128_mn(tmem, sA, sB);
    else tc::mma_128x128x128(tmem, sA, sB);
    tc::mma_commit(bar);
  }
  const int ok = tc::mbar_wait(bar, 0, kWaitLimit) ? 1 : 0;
  if (!ok && tid == 0) tc::mbar_wait(bar, 0, kWaitLimit);  // bounded: let the product land
  if (__syncthreads_and(ok)) {
    tc::fence_after_sync();
    for (int c0 = 0; c0 < kH; c0 += 32) {
      float acc[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
      for (int i = 0; i < 32; ++i) D[tid * kH + c0 + i] = acc[i];
    }
  } else if (tid == 0) {
    status_or(status, RT_DEV_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kH);
  }
}

// ---------------------------------------------------------------- surrogate walk
constexpr int kWalkTiles = 3;                   // 128-ray tiles sharing the resident weights
constexpr int kWalkMlpThreads = 128 * kWalkTiles;
constexpr int kWalkTmemCols = 512;              // power of two >= kWalkTiles * kH

// Layer 1 (K = 4) on the tensor cores as one K = 16 product: each input u_i and
// weight w_i split into BF16 high and low parts, u w ~ u_hi w_hi + u_hi w_lo + u_lo w_hi
// (the dropped u_lo w_lo is below 2^-16 of the term), and the bias as b_hi + b_lo
// against two constant-one columns: the products are exact in the FP32
// accumulator, so z keeps about 16 significant bits.
constexpr int kL1K = 16;
constexpr int kL1Elems = kH * kL1K;

// column k of the layer-1 operands: 3i + {0, 1, 2} for input i, 12 and 13 the bias
__device__ __forceinline__ int l1_index(int r, int k) { return (int)(tc::kmajor_offset(r, k, kL1K) >> 1); }

struct WalkSmall {  // the head; every hidden layer's bias is in its tensor-core product
  float w5[kH];
  float b5;
};

struct WalkMlpSmem {
  uint16_t W[3][kTileElems];           // W2..W4 (rows = out)
  uint16_t A[kWalkTiles][kTileElems];  // layer inputs of the tiles
  uint16_t A1[kWalkTiles][kL1Elems];   // layer-1 inputs (hi/lo split, K = 16)
  uint16_t B1[kL1Elems];               // layer-1 weights and bias (hi/lo split, rows = out)
  uint16_t Bb[3][kL1Elems];            // biases of layers 2..4 against A1's constant-one columns
  WalkSmall sp;
  uint64_t bar_w, bar_mma[kWalkTiles];
  unsigned long long next, end;        // the current work item's claim cursor and end
  int band;                            // the current work item's band (-1: no item left)
  uint32_t tmem;
};

// Work of a surrogate walk over a spectral-band ensemble: the rays grouped by the
// band of their wavenumber index (order[band_start[b] ..] are band b's ray offsets;
// nullptr: one band, rays in order), cut into work items of at most `chunk` rays
// that never straddle a band (band b's items are item_start[b] .. item_start[b+1]).
struct BandPlan {
  const uint32_t *order;
  const long long *band_start, *item_start;
  unsigned long long *item_next;  // work-item counter, zero at launch
  long long chunk;
  int n_bands;
};
static_assert(sizeof(WalkMlpSmem) <= 227 * 1024, "surrogate walk shared memory exceeds 227 KB per block");

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// the walk's parameters in shared memory: layer-1 operand B, biases and head
__device__ __forceinline__ void stage_walk(WalkMlpSmem &S, const float *__restrict__ P) {
  for (int e = threadIdx.x; e < kL1Elems; e += blockDim.x) {
    const int n = e / kL1K, k = e % kL1K;
    uint16_t bits = 0;
    if (k < 12) {
      const float w = P[oW1 + 4 * n + k / 3];
      const uint16_t hi = bf16_bits(w);
      bits = (k % 3 == 1) ? bf16_bits(w - bf16_value(hi)) : hi;
    } else if (k < 14) {
      const float b = P[oB1 + n];
      const uint16_t hi = bf16_bits(b);
      bits = (k == 13) ? bf16_bits(b - bf16_value(hi)) : hi;
    }
    S.B1[l1_index(n, k)] = bits;
  }
  // layers 2..4: K = 16 operands with b_hi, b_lo in rows 12, 13 (A1's 1.0 columns), zeros elsewhere
  for (int e = threadIdx.x; e < 3 * kL1Elems; e += blockDim.x) {
    const int l = e / kL1Elems, n = (e % kL1Elems) / kL1K, k = e % kL1K;
    uint16_t bits = 0;
    if (k == 12 || k == 13) {
      const float b = P[(l == 0 ? oB2 : (l == 1 ? oB3 : oB4)) + n];
      const uint16_t hi = bf16_bits(b);
      bits = (k == 13) ? bf16_bits(b - bf16_value(hi)) : hi;
    }
    S.Bb[l][l1_index(n, k)] = bits;
  }
  for (int c = threadIdx.x; c < kH; c += blockDim.x) S.sp.w5[c] = P[oW5 + c];
  if (threadIdx.x == 0) S.sp.b5 = P[oB5];
}

// The 128 threads of one tile (4 warps, named barrier 1 + tile) synchronise
// among themselves only, so the tiles of a block drift apart and one tile's
// epilogue runs while another tile's products occupy the tensor cores.
__device__ __forceinline__ void tile_sync(int tile) {
  asm volatile("barrier.cta.sync %0, 128;" ::"r"(1 + tile) : "memory");
}
__device__ __forceinline__ bool tile_or(int tile, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
      " barrier.cta.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r) : "r"((uint32_t)v), "r"(1 + tile) : "memory");
  return r != 0;
}

// Network output (log kappa) for this thread's query, the 128 threads of its tile
// together.  Returns false if a bounded tensor-core wait ran out.
__device__ __forceinline__ bool mlp_eval_tile(WalkMlpSmem &S, uint32_t tmem, const Norm &N,
                                              const float (&raw)[4], uint32_t &phase, float &logk) {
  const int tid = threadIdx.x, tile = tid >> 7, r = tid & 127, warp = tid >> 5;
  {  // this row of the layer-1 operand A: {u_hi, u_hi, u_lo} per input, then 1, 1, 0, 0
    uint16_t e[kL1K];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float u = 2.0f * (raw[i] - N.lo[i]) / (N.hi[i] - N.lo[i]) - 1.0f;
      const uint16_t hi = bf16_bits(u);
      e[3 * i] = hi;
      e[3 * i + 1] = hi;
      e[3 * i + 2] = bf16_bits(u - bf16_value(hi));
    }
    e[12] = e[13] = 0x3F80u;  // 1.0
    e[14] = e[15] = 0u;
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = (uint32_t)e[2 * i] | ((uint32_t)e[2 * i + 1] << 16);
    *reinterpret_cast<uint4 *>(&S.A1[tile][l1_index(r, 0)]) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(&S.A1[tile][l1_index(r, 8)]) = make_uint4(w[4], w[5], w[6], w[7]);
  }
  float y = 0.0f;
  const uint32_t tcol = tmem + (uint32_t)(tile * kH);
  // l = 0: layer 1 (K = 16); l = 1..3: W2..W4 (K = 128)
#pragma unroll 1
  for (int l = 0; l < 4; ++l) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    tile_sync(tile);
    if (r == 0) {
      tc::fence_after_sync();
      const uint64_t a1 = tc::smem_desc(tc::smem_addr(S.A1[tile]), 128u, 256u);
      if (l == 0) {
        tc::mma_bf16(tcol, a1, tc::smem_desc(tc::smem_addr(S.B1), 128u, 256u), tc::idesc_bf16_f32(128, 128), 0u);
      } else {
        tc::mma_128x128x128(tcol, S.A[tile], S.W[l - 1]);
        tc::mma_bf16(tcol, a1, tc::smem_desc(tc::smem_addr(S.Bb[l - 1]), 128u, 256u),
                     tc::idesc_bf16_f32(128, 128), 1u);  // + bias
      }
      tc::mma_commit(&S.bar_mma[tile]);
    }
    const int timeout = tc::mbar_wait(&S.bar_mma[tile], phase, kWaitLimit) ? 0 : 1;
    phase ^= 1u;
    if (tile_or(tile, timeout)) {
      // the product may still be in flight: let it land (bounded) before the tile stops
      if (r == 0) tc::mbar_wait(&S.bar_mma[tile], phase ^ 1u, kWaitLimit);
      return false;
    }
    tc::fence_after_sync();
#pragma unroll 1
    for (int c0 = 0; c0 < kH; c0 += 32) {
      float z[32];  // pre-activations, biases included
      tc::tmem_ld32(tcol + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, z);
      if (l < 3) {  // next layer's BF16 input: binary32 SiLU (as in training), rounded to BF16
#pragma unroll
        for (int i = 0; i < 32; i += 8)
          *reinterpret_cast<uint4 *>(&S.A[tile][tile_index(r, c0 + i)]) =
              make_uint4(pack_bf16x2(z[i] * sigmoid_fast(z[i]), z[i + 1] * sigmoid_fast(z[i + 1])),
                         pack_bf16x2(z[i + 2] * sigmoid_fast(z[i + 2]), z[i + 3] * sigmoid_fast(z[i + 3])),
                         pack_bf16x2(z[i + 4] * sigmoid_fast(z[i + 4]), z[i + 5] * sigmoid_fast(z[i + 5])),
                         pack_bf16x2(z[i + 6] * sigmoid_fast(z[i + 6]), z[i + 7] * sigmoid_fast(z[i + 7])));
      } else {  // last hidden layer: binary32 SiLU into the head
#pragma unroll
        for (int q = 0; q < 32; ++q) y = fmaf(S.sp.w5[c0 + q], z[q] * sigmoid_fast(z[q]), y);
      }
    }
  }
  // this tile's accumulators are read before its next products overwrite them
  tc::fence_before_sync();
  logk = N.mean + N.scale * (y + S.sp.b5);
  return true;
}

__global__ void __launch_bounds__(kWalkMlpThreads, 1)
k_walk_mlp(const float *__restrict__ P, const uint16_t *__restrict__ tiles, Norm N1,
           const Norm *__restrict__ norms, BandPlan B, const float *__restrict__ T,
           const float *__restrict__ Pf, const float *__restrict__ Xf, float p_ref, float x_ref, WalkParams W,
           double *__restrict__ absorbed, double *__restrict__ scalars,
           unsigned long long *__restrict__ steps_out, unsigned long long *__restrict__ evals_out,
           uint32_t *status, RecordPtrs rec) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WalkMlpSmem &S = *reinterpret_cast<WalkMlpSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&S.bar_w, 1);
    for (int t = 0; t < kWalkTiles; ++t) tc::mbar_init(&S.bar_mma[t], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(&S.tmem, kWalkTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem;
  const bool record = rec.cells != nullptr;
  double em = 0.0, esc = 0.0;
  unsigned long long nsteps = 0;
  uint32_t phase = 0;   // this tile's product barrier phase
  uint32_t wphase = 0;  // the weight copies' barrier phase
  int cur_band = -1, timeout = 0;
  bool weights_late = false;
  const int tile = tid >> 7;
  unsigned long long n_evals = 0;  // this tile's network evaluations (counted by its thread 0)
  Norm N = N1;
#pragma unroll 1
  for (;;) {  // work items: one band's network, at most B.chunk of its rays
    if (tid == 0) {
      const long long it = (long long)atomicAdd(B.item_next, 1ull);
      int band = -1;
      long long b0 = 0, b1 = 0;
      if (it < B.item_start[B.n_bands]) {
        int lo = 0, hi = B.n_bands - 1;  // the last band whose first item is <= it
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (B.item_start[mid] <= it) lo = mid; else hi = mid - 1;
        }
        band = lo;
        b0 = B.band_start[band] + (it - B.item_start[band]) * B.chunk;
        b1 = min(b0 + B.chunk, B.band_start[band + 1]);
      }
      S.band = band;
      S.next = (unsigned long long)b0;
      S.end = (unsigned long long)b1;
    }
    __syncthreads();
    const int band = S.band;
    if (band < 0) break;
    if (band != cur_band) {  // this band's network: small parameters staged, hidden layers copied
      stage_walk(S, P + (long long)band * kNParam);
      tc::fence_smem_to_async();  // B1, Bb are read by the tensor cores of every tile
      if (tid == 0) {
        tc::mbar_arrive_expect_tx(&S.bar_w, 3 * kTileBytes);
        tc::bulk_g2s(&S.W[0][0], tiles + (long long)band * 3 * kTileElems, 3 * kTileBytes, &S.bar_w);
      }
      const int late = tc::mbar_wait(&S.bar_w, wphase, kWaitLimit) ? 0 : 1;
      wphase ^= 1u;
      tc::fence_before_sync();
      if (__syncthreads_or(late)) {
        weights_late = true;
        timeout = 1;
        break;
      }
      tc::fence_after_sync();
      N = net_norm(norms, N1, band);
      cur_band = band;
    }
    Ray R;
    bool active = false;
#pragma unroll 1
    for (;;) {  // the item's rays: a lane whose ray is done claims the next one
      if (!active) {
        const unsigned long long claim = atomicAdd(&S.next, 1ull);
        if (claim < S.end) {
          ray_init(W, nullptr, nullptr, B.order ? (unsigned long long)B.order[claim] : claim, record, R);
          active = true;
        }
      }
      if (!tile_or(tile, active)) break;  // this tile has no ray of the item left
      float raw[4] = {N.lo[0], N.lo[1], N.lo[2], N.lo[3]};
      float Tc = 1.0f;
      if (active) {
        Tc = T[R.cell];
        raw[0] = __logf(fmaf((float)R.j, W.dnu, W.nu_min));
        raw[1] = Tc;
        raw[2] = Pf ? Pf[R.cell] : p_ref;
        raw[3] = Xf ? Xf[R.cell] : x_ref;
      }
      float logk = 0.0f;
      if (!mlp_eval_tile(S, tmem, N, raw, phase, logk)) {
        timeout = 1;
        break;
      }
      n_evals += (tid & 127) == 0 ? 1 : 0;
      if (active) {
        const float kap = __expf(logk);
        if (R.w < 0.0f) R.w = emission_weight(W, R.j, Tc, kap);
        bool fin = ray_step(W, kap, absorbed, status, rec, R);
        // a dark ray (transmission zero, no optical-depth cut) needs no more kappa: it
        // takes its remaining steps at once, DDA only, and frees its lane for a new ray
        if (!fin && R.trans == 0.0f && !W.tau_cut)
          while (!(fin = ray_step<true, true, false, true>(W, 0.0f, absorbed, status, rec, R))) {
          }
        if (fin) {
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
    }
    // every tile is done with this item (and with the band's weights) before the next
    if (__syncthreads_or(timeout)) {  // any tile's wait gave up: the block stops, flag uniform
      timeout = 1;
      break;
    }
  }
  if (timeout && tid == 0) status_or(status, RT_DEV_TIMEOUT);
  if (weights_late && tid == 0) tc::mbar_wait(&S.bar_w, wphase ^ 1u, kWaitLimit);  // bounded: let the copy land
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
  if (evals_out && n_evals) atomicAdd(evals_out, n_evals);  // nonzero only in a tile's thread 0
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kWalkTmemCols);
  }
}

// Training samples drawn from line-by-line tables kappa[kp][kT][j] (x_ref mole
// fraction): Philox counter (i, 0, 0, 0x6d6c70) under the seed picks the
// wavenumber, temperature node, pressure node and a mole fraction in
// [x_lo, x_hi]; the target is log(kappa x / x_ref) (kappa is linear in x).
__global__ void k_mlp_samples(const float *__restrict__ tables, int np, int nT, long long n_nu,
                              const float *__restrict__ p_nodes, float T_min, float dT, float nu_min,
                              float dnu, float x_lo, float x_hi, float x_ref, uint32_t seed_lo,
                              uint32_t seed_hi, long long n, float *__restrict__ inputs,
                              float *__restrict__ targets) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32x4 v = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)((unsigned long long)i >> 32), 0u, 0x6d6c70u},
                                seed_lo, seed_hi);
  const long long j = (long long)(((unsigned long long)v.x * (unsigned long long)n_nu) >> 32);
  const int kT = (int)(((unsigned long long)v.y * (unsigned long long)nT) >> 32);
  const int kp = (int)(((unsigned long long)v.z * (unsigned long long)np) >> 32);
  const float x = x_lo + (x_hi - x_lo) * ((float)(v.w >> 8) * 0x1p-24f);
  const float kap = tables[((long long)kp * nT + kT) * n_nu + j];
  inputs[i * 4 + 0] = __logf(fmaf((float)j, dnu, nu_min));
  inputs[i * 4 + 1] = fmaf((float)kT, dT, T_min);
  inputs[i * 4 + 2] = p_nodes[kp];
  inputs[i * 4 + 3] = x;
  targets[i] = logf(fmaxf(kap * (x / x_ref), 1e-30f));
}

// Training samples of a spectral-band ensemble: band b (grid.y) draws its n samples
// from its own wavenumbers j in [b band_pts, min((b + 1) band_pts, n_nu)): Philox
// counter (i, i >> 32, b + 1, 0x6d6c70) under the seed picks j in the band, the T
// node, the pressure node and x as k_mlp_samples does; rows b n + i.  A sample whose
// low byte of word 3 is below em_256 (of 256) instead draws j with probability
// proportional to kappa I_b(nu_j, T_k) over the band at its (p, T) node (the
// emission the walk samples), by a scan of the band's cumulative weights.
__global__ void k_mlp_samples_bands(const float *__restrict__ tables, int np, int nT, long long n_nu,
                                    const float *__restrict__ p_nodes, float T_min, float dT, float nu_min,
                                    float dnu, float x_lo, float x_hi, float x_ref, uint32_t seed_lo,
                                    uint32_t seed_hi, int band_pts, int em_256, float c2_cm, long long n,
                                    float *__restrict__ inputs, float *__restrict__ targets) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long b = blockIdx.y;
  if (i >= n) return;
  const u32x4 v = philox4x32_10(u32x4{(uint32_t)i, (uint32_t)((unsigned long long)i >> 32), (uint32_t)(b + 1),
                                      0x6d6c70u}, seed_lo, seed_hi);
  const long long j0 = b * band_pts;
  const long long width = min((long long)band_pts, n_nu - j0);
  const int kT = (int)(((unsigned long long)v.y * (unsigned long long)nT) >> 32);
  const int kp = (int)(((unsigned long long)v.z * (unsigned long long)np) >> 32);
  const float x = x_lo + (x_hi - x_lo) * ((float)(v.w >> 8) * 0x1p-24f);
  const float *row = tables + ((long long)kp * nT + kT) * n_nu;
  long long j = j0 + (long long)(((unsigned long long)v.x * (unsigned long long)width) >> 32);
  if ((int)(v.w & 255u) < em_256) {
    const float Tk = fmaf((float)kT, dT, T_min);
    auto weight = [&](long long q) {  // kappa nu^3 / (exp(c2 nu / T) - 1), the Planck constants dropped
      const float nu = fmaf((float)q, dnu, nu_min);
      return row[q] * nu * nu * nu / expm1f(c2_cm * nu / Tk);
    };
    float tot = 0.0f;
    for (long long q = j0; q < j0 + width; ++q) tot += weight(q);
    const float target = tot * ((float)(v.x >> 8) * 0x1p-24f);
    float acc = 0.0f;
    j = j0 + width - 1;
    for (long long q = j0; q < j0 + width; ++q) {
      acc += weight(q);
      if (acc > target) {
        j = q;
        break;
      }
    }
  }
  const float kap = row[j];
  const long long o = b * n + i;
  inputs[o * 4 + 0] = __logf(fmaf((float)j, dnu, nu_min));
  inputs[o * 4 + 1] = fmaf((float)kT, dT, T_min);
  inputs[o * 4 + 2] = p_nodes[kp];
  inputs[o * 4 + 3] = x;
  targets[o] = logf(fmaxf(kap * (x / x_ref), 1e-30f));
}

}  // namespace

rt_status validate_spec(const rt_spectral *s);

namespace {

rt_status set_smem(const void *fn, size_t bytes) {
  RT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return RT_OK;
}

rt_status validate_norm(const rt_mlp_norm *nm) {
  if (!nm) return fail(RT_E_INVAL, "norm is NULL");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(nm->in_lo[i]) || !std::isfinite(nm->in_hi[i]) || !(nm->in_hi[i] > nm->in_lo[i]))
      return fail(RT_E_INVAL, "norm: input range %d must be finite with hi > lo", i);
  if (!std::isfinite(nm->out_mean) || !std::isfinite(nm->out_scale) || !(nm->out_scale > 0))
    return fail(RT_E_INVAL, "norm: out_mean, out_scale must be finite, scale > 0");
  return RT_OK;
}

Norm to_norm(const rt_mlp_norm *nm) {
  Norm N;
  for (int i = 0; i < 4; ++i) {
    N.lo[i] = nm->in_lo[i];
    N.hi[i] = nm->in_hi[i];
  }
  N.mean = nm->out_mean;
  N.scale = nm->out_scale;
  return N;
}

}  // namespace

// BF16 tiles of n_nets networks: the first n_mats of W2..W4, W2^T..W4^T per network
rt_status mlp_prep_tiles(const float *params, uint16_t *tiles, int n_nets, int n_mats, cudaStream_t st) {
  k_mlp_prep<<<dim3(kTileElems / 256, n_mats, n_nets), 256, 0, st>>>(params, tiles, n_mats);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

// scratch of one training step of n samples for each of n_nets networks: BF16 weight
// tiles, pre-activations, output gradients, per-tile gradient partials
size_t train_scratch_bytes(int64_t n, int n_nets) {
  const size_t grid = (size_t)((n + kH - 1) / kH);
  const size_t nn = (size_t)n_nets;
  return nn * (6 * (size_t)kTileBytes + (size_t)4 * (size_t)n * kH * sizeof(float) + (size_t)n * sizeof(float) +
               grid * kGradStride * sizeof(float)) + 64;
}

rt_status validate_train(float *params, float *m, float *v, float *grad, const float *inputs,
                         const float *targets, int64_t n, int n_nets, const rt_mlp_norm *nm, bool norm_on_device,
                         int32_t flags, float *loss) {
  if (!params || !grad || !inputs || !targets || !loss)
    return fail(RT_E_INVAL, "rt_mlp_train_step: NULL buffer");
  if (!(flags & RT_MLP_GRAD_ONLY) && (!m || !v)) return fail(RT_E_INVAL, "rt_mlp_train_step: NULL Adam state");
  if (n < 1 || n > (1LL << 26)) return fail(RT_E_INVAL, "rt_mlp_train_step: n out of range");
  if (n_nets < 1 || n_nets > 65535) return fail(RT_E_INVAL, "rt_mlp_train_steps_nets: n_nets must be in [1, 65535]");
  if ((double)n * (double)n_nets > (double)(1LL << 30))
    return fail(RT_E_INVAL, "rt_mlp_train_steps_nets: n * n_nets must not exceed 2^30 samples per step");
  if (!nm) return fail(RT_E_INVAL, "norm is NULL");
  if (!norm_on_device) {
    rt_status s = validate_norm(nm);
    if (s != RT_OK) return s;
  }
  static std::once_flag once;
  static rt_status attr = RT_OK;
  std::call_once(once, [] {
    attr = set_smem((const void *)k_mlp_fwd<true>, sizeof(FwdSmem));
    if (attr == RT_OK) attr = set_smem((const void *)k_mlp_bwd, sizeof(BwdSmem));
    if (attr == RT_OK) {  // two backward blocks per SM: the largest shared-memory split
      const cudaError_t e = cudaFuncSetAttribute((const void *)k_mlp_bwd,
                                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) attr = fail(RT_E_CUDA, "k_mlp_bwd carveout: %s", cudaGetErrorString(e));
    }
  });
  return attr;
}

// one step on validated arguments, scratch of train_scratch_bytes(n, n_nets) bytes;
// `chained`: the scratch's BF16 tiles already hold the parameters and the loss slot
// is zero (a run of steps), and the Adam kernel refreshes the tiles for the next
// step.  n_nets networks (norms: device [n_nets], or N1 by value for one network)
// each take n samples of inputs / targets at row net * in_stride.  `write_grad`:
// the step stores its gradient into grad (always with RT_MLP_GRAD_ONLY).
rt_status mlp_train_core(float *params, float *m, float *v, float *grad, const float *inputs,
                         const float *targets, int64_t n, int64_t in_stride, int n_nets, const Norm &N1,
                         const Norm *norms, float lr, int32_t step, int32_t flags, float *loss, uint32_t *status,
                         char *scr, bool chained, bool write_grad, cudaStream_t st) {
  const unsigned grid = (unsigned)((n + kH - 1) / kH);
  const size_t nn = (size_t)n_nets;
  uint16_t *tiles = reinterpret_cast<uint16_t *>(scr);
  float *Z = reinterpret_cast<float *>(scr + nn * 6 * (size_t)kTileBytes);
  float *dy = Z + nn * 4 * (size_t)n * kH;
  float *gpart = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(dy + nn * (size_t)n) + 63) & ~uintptr_t(63));  // 64-byte aligned rows
  if (!chained) {
    RT_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    rt_status s = mlp_prep_tiles(params, tiles, n_nets, 6, st);
    if (s != RT_OK) return s;
  }
  const long long ts = 6LL * kTileElems;
  k_mlp_fwd<true><<<dim3(grid, n_nets), kFwdThreads, sizeof(FwdSmem), st>>>(
      params, tiles, ts, N1, norms, inputs, targets, n, in_stride, Z, dy, loss, 1.0f / (float)n_nets, nullptr,
      status);
  RT_CUDA_TRY(cudaGetLastError());
  k_mlp_bwd<<<dim3(grid, n_nets), kBwdThreads, sizeof(BwdSmem), st>>>(params, tiles, ts, N1, norms, inputs, n,
                                                                      in_stride, Z, dy, gpart, status);
  RT_CUDA_TRY(cudaGetLastError());
  const bool adam = !(flags & RT_MLP_GRAD_ONLY);
  const float c1 = adam ? (float)(1.0 - std::pow(0.9, step)) : 1.0f;
  const float c2 = adam ? (float)(1.0 - std::pow(0.999, step)) : 1.0f;
  float *g_out = write_grad ? grad : nullptr;
  uint16_t *t_out = chained ? tiles : nullptr;
  if (n_nets >= kAdamWide) {
    constexpr int per_block = kAdamThreads * 4;
    k_grad_adam<4><<<dim3((kNParam + per_block - 1) / per_block, n_nets), kAdamThreads, 0, st>>>(
        gpart, (int)grid, g_out, adam ? 1 : 0, params, m, v, lr, 0.9f, 0.999f, 1e-8f, c1, c2, t_out);
  } else {
    k_grad_adam<1><<<dim3((kNParam + kAdamThreads - 1) / kAdamThreads, n_nets), kAdamThreads, 0, st>>>(
        gpart, (int)grid, g_out, adam ? 1 : 0, params, m, v, lr, 0.9f, 0.999f, 1e-8f, c1, c2, t_out);
  }
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status mlp_train_impl(float *params, float *m, float *v, float *grad, const float *inputs,
                         const float *targets, int64_t n, const rt_mlp_norm *nm, float lr, int32_t step,
                         int32_t flags, float *loss, uint32_t *status, cudaStream_t st) {
  rt_status s = validate_train(params, m, v, grad, inputs, targets, n, 1, nm, false, flags, loss);
  if (s != RT_OK) return s;
  if (!(flags & RT_MLP_GRAD_ONLY) && (step < 1 || !std::isfinite(lr) || lr < 0))
    return fail(RT_E_INVAL, "rt_mlp_train_step: step >= 1 and finite lr >= 0 required");
  Scratch scr;
  s = scr.alloc(train_scratch_bytes(n, 1), st);
  if (s != RT_OK) return s;
  return mlp_train_core(params, m, v, grad, inputs, targets, n, n, 1, to_norm(nm), nullptr, lr, step, flags,
                        loss, status, scr.as<char>(), false, true, st);
}

// n_steps steps of n_nets networks (one network: nm is a host norm; an ensemble: nm
// is a device array of n_nets norms), inputs / targets [n_nets][n] rows
rt_status mlp_train_steps_impl(float *params, float *m, float *v, float *grad, const float *inputs,
                              const float *targets, int64_t n, int64_t batch, int n_nets, const rt_mlp_norm *nm,
                              bool norm_on_device, double lr0, double lr1, int32_t step_first, int32_t n_steps,
                              int32_t total_steps, float *losses, uint32_t *status, cudaStream_t st) {
  if (!inputs || !targets) return fail(RT_E_INVAL, "rt_mlp_train_steps: NULL buffer");
  if (batch < 1 || batch > n) return fail(RT_E_INVAL, "rt_mlp_train_steps: batch must be in [1, n]");
  if (step_first < 1 || n_steps < 0 || total_steps < 1 ||
      (int64_t)step_first - 1 + n_steps > (int64_t)total_steps)
    return fail(RT_E_INVAL, "rt_mlp_train_steps: need step_first >= 1, n_steps >= 0, "
                            "step_first - 1 + n_steps <= total_steps");
  if (!std::isfinite(lr0) || !std::isfinite(lr1) || lr0 < 0 || lr1 < 0)
    return fail(RT_E_INVAL, "rt_mlp_train_steps: finite learning rates >= 0 required");
  if (n_nets < 1) return fail(RT_E_INVAL, "rt_mlp_train_steps_nets: n_nets must be >= 1");
  if (n_steps == 0) return RT_OK;
  // one scratch for all steps: the step's buffers, then a loss slot if none is given
  const size_t sb = (train_scratch_bytes(batch, n_nets) + 255) & ~size_t(255);
  Scratch scr;
  rt_status r = scr.alloc(sb + 256, st);
  if (r != RT_OK) return r;
  float *loss1 = reinterpret_cast<float *>(scr.as<char>() + sb);
  r = validate_train(params, m, v, grad, inputs, targets, batch, n_nets, nm, norm_on_device, 0,
                     losses ? losses : loss1);
  if (r != RT_OK) return r;
  const Norm N1 = norm_on_device ? Norm{} : to_norm(nm);
  const Norm *norms = norm_on_device ? reinterpret_cast<const Norm *>(nm) : nullptr;
  // the steps after the first take their BF16 tiles from the previous step's Adam
  // kernel, and a given loss buffer is zeroed once for all steps
  if (losses) RT_CUDA_TRY(cudaMemsetAsync(losses, 0, (size_t)n_steps * sizeof(float), st));
  r = mlp_prep_tiles(params, scr.as<uint16_t>(), n_nets, 6, st);
  if (r != RT_OK) return r;
  const int64_t nb = n / batch;
  const double span = (double)std::max(1, total_steps - 1);
  for (int32_t i = 0; i < n_steps; ++i) {
    const int64_t s = (int64_t)step_first - 1 + i;
    const int64_t b = s % nb;
    const double lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + std::cos(kPiD * (double)s / span));
    if (!losses) RT_CUDA_TRY(cudaMemsetAsync(loss1, 0, sizeof(float), st));
    // every network's batch b: rows b * batch .. of its own n rows
    r = mlp_train_core(params, m, v, grad, inputs + 4 * b * batch, targets + b * batch, batch, n, n_nets, N1,
                       norms, (float)lr, (int32_t)(s + 1), 0, losses ? losses + i : loss1, status, scr.as<char>(),
                       true, i == n_steps - 1, st);
    if (r != RT_OK) return r;
  }
  return RT_OK;
}

rt_status mlp_forward_impl(int n_nets, const float *params, const rt_mlp_norm *nm, bool norm_on_device,
                           const float *inputs, int64_t n, float *out, uint32_t *status, cudaStream_t st) {
  if (n < 0) return fail(RT_E_INVAL, "rt_mlp_forward: n < 0");
  if (n_nets < 1 || n_nets > 65535) return fail(RT_E_INVAL, "rt_mlp_forward_nets: n_nets must be in [1, 65535]");
  if (n == 0) return RT_OK;  // no sample: the buffers are not read and may be NULL
  if (!params || !inputs || !out || !nm) return fail(RT_E_INVAL, "rt_mlp_forward: NULL buffer");
  if (!norm_on_device) {
    rt_status s = validate_norm(nm);
    if (s != RT_OK) return s;
  }
  static std::once_flag once;
  static rt_status attr = RT_OK;
  std::call_once(once, [] { attr = set_smem((const void *)k_mlp_fwd<false>, sizeof(FwdSmem)); });
  if (attr != RT_OK) return attr;
  Scratch scr;
  rt_status s = scr.alloc((size_t)n_nets * 3 * (size_t)kTileBytes, st);
  if (s != RT_OK) return s;
  s = mlp_prep_tiles(params, scr.as<uint16_t>(), n_nets, 3, st);
  if (s != RT_OK) return s;
  const unsigned grid = (unsigned)((n + kH - 1) / kH);
  const Norm N1 = norm_on_device ? Norm{} : to_norm(nm);
  const Norm *norms = norm_on_device ? reinterpret_cast<const Norm *>(nm) : nullptr;
  k_mlp_fwd<false><<<dim3(grid, n_nets), kFwdThreads, sizeof(FwdSmem), st>>>(
      params, scr.as<uint16_t>(), 3LL * kTileElems, N1, norms, inputs, nullptr, n, n, nullptr, nullptr, nullptr,
      1.0f, out, status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status tc_selftest_impl(const float *A, const float *B, float *D, bool mn, uint32_t *status,
                           cudaStream_t st) {
  if (!A || !B || !D) return fail(RT_E_INVAL, "rt_tc_selftest: NULL buffer");
  const size_t bytes = (mn ? 4 : 2) * (size_t)kTileBytes + 64;
  static std::once_flag once;
  static rt_status attr = RT_OK;
  std::call_once(once, [] {
    attr = set_smem((const void *)k_tc_selftest<false>, 2 * (size_t)kTileBytes + 64);
    if (attr == RT_OK) attr = set_smem((const void *)k_tc_selftest<true>, 4 * (size_t)kTileBytes + 64);
  });
  if (attr != RT_OK) return attr;
  if (mn) k_tc_selftest<true><<<1, kH, bytes, st>>>(A, B, D, status);
  else k_tc_selftest<false><<<1, kH, bytes, st>>>(A, B, D, status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

// The surrogate walk over n_bands networks (band b serves j in [b band_pts, ..)):
// params device [n_bands][RT_MLP_NPARAM], norms device [n_bands] (or N1 by value
// for a single network with band_pts >= n_nu).
rt_status trace_mlp_core(const rt_grid *grid, int band_pts, const float *params, const Norm &N1,
                         const Norm *norms, const rt_spectral *spec, uint64_t ray_begin, uint64_t n_rays,
                         uint64_t n_total, uint64_t seed, uint32_t enclosure, int32_t flags,
                         const rt_tally_buf *tally, const rt_record *record, cudaStream_t st) {
  WalkParams W;
  RecordPtrs rp;
  const bool count_evals = (flags & RT_COUNT_EVALS) != 0;
  flags &= ~RT_COUNT_EVALS;
  rt_status v = walk_setup(grid, spec, ray_begin, n_rays, n_total, seed, enclosure, flags, tally, record, &W, &rp);
  if (v != RT_OK) return v;
  if ((flags & 0xF) != RT_SRC_EMIT) return fail(RT_E_INVAL, "rt_trace_mlp: only RT_SRC_EMIT");
  if (band_pts < 1) return fail(RT_E_INVAL, "rt_trace_mlp_bands: band_pts must be >= 1");
  const long long nb_ll = (spec->n_nu + band_pts - 1) / band_pts;
  if (nb_ll > 65535) return fail(RT_E_INVAL, "rt_trace_mlp_bands: at most 65535 bands (n_nu / band_pts)");
  const int n_bands = (int)nb_ll;
  if (n_bands > 1 && n_rays > 0xFFFFFFFFull)
    return fail(RT_E_INVAL, "rt_trace_mlp_bands: at most 2^32 - 1 rays per call with several bands");
  if (n_rays == 0) return RT_OK;
  static std::once_flag once;
  static rt_status attr = RT_OK;
  std::call_once(once, [] { attr = set_smem((const void *)k_walk_mlp, sizeof(WalkMlpSmem)); });
  if (attr != RT_OK) return attr;
  int dev = 0, sms = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  RT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned long long want = (n_rays + 8ull * kWalkMlpThreads - 1) / (8ull * kWalkMlpThreads);
  const unsigned blocks = (unsigned)(want < (unsigned long long)sms ? (want > 0 ? want : 1) : sms);
  // work items of about 1/8 of a block's share of the rays (at least 1024), so that
  // the blocks finish together
  const long long chunk = std::max(1024LL, (long long)(n_rays / (8ull * blocks)));
  // scratch: the bands' BF16 hidden-layer tiles, the plan, the band-grouped ray order
  const size_t tiles_b = (size_t)n_bands * 3 * kTileBytes;
  const size_t plan_b = (((size_t)n_bands * 8 * 3 + 16 * 3 + 255) / 256) * 256;
  const size_t order_b = n_bands > 1 ? (size_t)n_rays * sizeof(uint32_t) : 0;
  Scratch scr;
  v = scr.alloc(tiles_b + plan_b + order_b, st);
  if (v != RT_OK) return v;
  char *base = scr.as<char>();
  uint16_t *tiles = reinterpret_cast<uint16_t *>(base);
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(base + tiles_b);  // then cursors
  long long *band_start = reinterpret_cast<long long *>(counts + n_bands);
  long long *item_start = band_start + (n_bands + 1);
  unsigned long long *item_next = reinterpret_cast<unsigned long long *>(item_start + (n_bands + 1));
  uint32_t *order = n_bands > 1 ? reinterpret_cast<uint32_t *>(base + tiles_b + plan_b) : nullptr;
  v = mlp_prep_tiles(params, tiles, n_bands, 3, st);
  if (v != RT_OK) return v;
  RT_CUDA_TRY(cudaMemsetAsync(item_next, 0, sizeof(unsigned long long), st));
  v = band_plan(W, band_pts, n_bands, chunk, counts, band_start, item_start, order, sms, st);
  if (v != RT_OK) return v;
  BandPlan B{order, band_start, item_start, item_next, chunk, n_bands};
  k_walk_mlp<<<blocks, kWalkMlpThreads, sizeof(WalkMlpSmem), st>>>(
      params, tiles, N1, norms, B, grid->T, grid->p_atm, grid->x, (float)spec->p_ref_atm, (float)spec->x_ref, W,
      tally->absorbed, tally->scalars, tally->steps, count_evals ? tally->steps + 1 : nullptr, tally->status, rp);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status trace_mlp_impl(const rt_grid *grid, const float *params, const rt_mlp_norm *nm,
                         const rt_spectral *spec, uint64_t ray_begin, uint64_t n_rays, uint64_t n_total,
                         uint64_t seed, uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                         const rt_record *record, cudaStream_t st) {
  if (!params) return fail(RT_E_INVAL, "rt_trace_mlp: params is NULL");
  rt_status v = validate_norm(nm);
  if (v != RT_OK) return v;
  if (!spec) return fail(RT_E_INVAL, "rt_trace_mlp: spec is NULL");
  const long long pts = std::max<long long>(1, std::min<long long>(spec->n_nu, 0x7FFFFFFF));
  return trace_mlp_core(grid, (int)pts, params, to_norm(nm), nullptr, spec, ray_begin, n_rays, n_total, seed,
                        enclosure, flags, tally, record, st);
}

rt_status trace_mlp_bands_impl(const rt_grid *grid, int32_t band_pts, const float *params,
                               const rt_mlp_norm *norms, const rt_spectral *spec, uint64_t ray_begin,
                               uint64_t n_rays, uint64_t n_total, uint64_t seed, uint32_t enclosure, int32_t flags,
                               const rt_tally_buf *tally, const rt_record *record, cudaStream_t st) {
  if (!params || !norms) return fail(RT_E_INVAL, "rt_trace_mlp_bands: params or norms is NULL");
  if (!spec) return fail(RT_E_INVAL, "rt_trace_mlp_bands: spec is NULL");
  return trace_mlp_core(grid, band_pts, params, Norm{}, reinterpret_cast<const Norm *>(norms), spec, ray_begin,
                        n_rays, n_total, seed, enclosure, flags, tally, record, st);
}

rt_status mlp_samples_impl(const float *tables, int32_t np, const float *p_nodes, const rt_spectral *spec,
                           float x_lo, float x_hi, uint64_t seed, int64_t n, float *inputs,
                           float *targets, cudaStream_t st) {
  rt_status v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!tables || !p_nodes || !inputs || !targets || np < 1 || n < 0)
    return fail(RT_E_INVAL, "rt_mlp_make_samples: bad arguments");
  if (!(x_lo > 0) || !(x_hi >= x_lo)) return fail(RT_E_INVAL, "rt_mlp_make_samples: need 0 < x_lo <= x_hi");
  if (n == 0) return RT_OK;
  const float dT = spec->nT > 1 ? (float)((spec->T_max - spec->T_min) / (spec->nT - 1)) : 0.0f;
  k_mlp_samples<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      tables, np, spec->nT, spec->n_nu, p_nodes, (float)spec->T_min, dT, (float)spec->nu_min,
      (float)spec->dnu, x_lo, x_hi, (float)spec->x_ref, (uint32_t)seed, (uint32_t)(seed >> 32), n, inputs,
      targets);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

rt_status mlp_samples_bands_impl(const float *tables, int32_t np, const float *p_nodes, const rt_spectral *spec,
                                 int32_t band_pts, float x_lo, float x_hi, float emission_mix, uint64_t seed,
                                 int64_t n, float *inputs, float *targets, cudaStream_t st) {
  rt_status v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!tables || !p_nodes || !inputs || !targets || np < 1 || n < 0 || band_pts < 1)
    return fail(RT_E_INVAL, "rt_mlp_make_samples_bands: bad arguments");
  if (!(x_lo > 0) || !(x_hi >= x_lo)) return fail(RT_E_INVAL, "rt_mlp_make_samples_bands: need 0 < x_lo <= x_hi");
  if (!(emission_mix >= 0.0f && emission_mix <= 1.0f))
    return fail(RT_E_INVAL, "rt_mlp_make_samples_bands: emission_mix must be in [0, 1]");
  const long long n_bands = (spec->n_nu + band_pts - 1) / band_pts;
  if (n_bands > 65535) return fail(RT_E_INVAL, "rt_mlp_make_samples_bands: at most 65535 bands");
  if (n == 0) return RT_OK;
  const float dT = spec->nT > 1 ? (float)((spec->T_max - spec->T_min) / (spec->nT - 1)) : 0.0f;
  k_mlp_samples_bands<<<dim3((unsigned)((n + 255) / 256), (unsigned)n_bands), 256, 0, st>>>(
      tables, np, spec->nT, spec->n_nu, p_nodes, (float)spec->T_min, dT, (float)spec->nu_min, (float)spec->dnu,
      x_lo, x_hi, (float)spec->x_ref, (uint32_t)seed, (uint32_t)(seed >> 32), band_pts,
      (int)std::lround(emission_mix * 256.0f), (float)(100.0 * 6.62607015e-34 * 299792458.0 / 1.380649e-23), n,
      inputs, targets);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace rt

extern "C" {

rt_status rt_trace_mlp_bands(const rt_grid *grid, int32_t band_pts, const float *params,
                             const rt_mlp_norm *norms, const rt_spectral *spec, uint64_t ray_begin,
                             uint64_t n_rays, uint64_t n_rays_total, uint64_t seed, uint32_t enclosure,
                             int32_t flags, const rt_tally_buf *tally, const rt_record *record, void *stream) {
  return rt::trace_mlp_bands_impl(grid, band_pts, params, norms, spec, ray_begin, n_rays, n_rays_total, seed,
                                  enclosure, flags, tally, record, (cudaStream_t)stream);
}

rt_status rt_mlp_make_samples_bands(const float *tables, int32_t n_p, const float *p_nodes,
                                    const rt_spectral *spec, int32_t band_pts, float x_lo, float x_hi,
                                    float emission_mix, uint64_t seed, int64_t n_per_band, float *inputs,
                                    float *targets, void *stream) {
  return rt::mlp_samples_bands_impl(tables, n_p, p_nodes, spec, band_pts, x_lo, x_hi, emission_mix, seed,
                                    n_per_band, inputs, targets, (cudaStream_t)stream);
}

rt_status rt_trace_mlp(const rt_grid *grid, const float *params, const rt_mlp_norm *norm,
                       const rt_spectral *spec, uint64_t ray_begin, uint64_t n_rays,
                       uint64_t n_rays_total, uint64_t seed, uint32_t enclosure, int32_t flags,
                       const rt_tally_buf *tally, const rt_record *record, void *stream) {
  return rt::trace_mlp_impl(grid, params, norm, spec, ray_begin, n_rays, n_rays_total, seed, enclosure,
                            flags, tally, record, (cudaStream_t)stream);
}

rt_status rt_mlp_make_samples(const float *tables, int32_t n_p, const float *p_nodes,
                              const rt_spectral *spec, float x_lo, float x_hi, uint64_t seed,
                              int64_t n, float *inputs, float *targets, void *stream) {
  return rt::mlp_samples_impl(tables, n_p, p_nodes, spec, x_lo, x_hi, seed, n, inputs, targets,
                              (cudaStream_t)stream);
}


rt_status rt_mlp_train_step(float *params, float *adam_m, float *adam_v, float *grad,
                            const float *inputs, const float *targets, int64_t n,
                            const rt_mlp_norm *norm, float lr, int32_t step, int32_t flags,
                            float *loss, uint32_t *status, void *stream) {
  return rt::mlp_train_impl(params, adam_m, adam_v, grad, inputs, targets, n, norm, lr, step, flags,
                            loss, status, (cudaStream_t)stream);
}

rt_status rt_mlp_train_steps(float *params, float *adam_m, float *adam_v, float *grad,
                             const float *inputs, const float *targets, int64_t n, int64_t batch,
                             const rt_mlp_norm *norm, double lr0, double lr1, int32_t step_first,
                             int32_t n_steps, int32_t total_steps, float *losses, uint32_t *status,
                             void *stream) {
  return rt::mlp_train_steps_impl(params, adam_m, adam_v, grad, inputs, targets, n, batch, 1, norm, false, lr0,
                                  lr1, step_first, n_steps, total_steps, losses, status, (cudaStream_t)stream);
}

rt_status rt_mlp_train_steps_nets(int32_t n_nets, float *params, float *adam_m, float *adam_v, float *grad,
                                  const float *inputs, const float *targets, int64_t n, int64_t batch,
                                  const rt_mlp_norm *norms, double lr0, double lr1, int32_t step_first,
                                  int32_t n_steps, int32_t total_steps, float *losses, uint32_t *status,
                                  void *stream) {
  return rt::mlp_train_steps_impl(params, adam_m, adam_v, grad, inputs, targets, n, batch, n_nets, norms, true,
                                  lr0, lr1, step_first, n_steps, total_steps, losses, status,
                                  (cudaStream_t)stream);
}

rt_status rt_mlp_forward(const float *params, const rt_mlp_norm *norm, const float *inputs,
                         int64_t n, float *out, uint32_t *status, void *stream) {
  return rt::mlp_forward_impl(1, params, norm, false, inputs, n, out, status, (cudaStream_t)stream);
}

rt_status rt_mlp_forward_nets(int32_t n_nets, const float *params, const rt_mlp_norm *norms, const float *inputs,
                              int64_t n, float *out, uint32_t *status, void *stream) {
  return rt::mlp_forward_impl(n_nets, params, norms, true, inputs, n, out, status, (cudaStream_t)stream);
}

rt_status rt_tc_selftest(const float *A, const float *B, float *D, uint32_t *status, void *stream) {
  return rt::tc_selftest_impl(A, B, D, false, status, (cudaStream_t)stream);
}

rt_status rt_tc_selftest_mn(const float *A, const float *B, float *D, uint32_t *status, void *stream) {
  return rt::tc_selftest_impl(A, B, D, true, status, (cudaStream_t)stream);
}

}  // extern "C"
