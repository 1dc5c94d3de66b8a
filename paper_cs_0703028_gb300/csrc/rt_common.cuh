// Shared device helpers of the GB300 radiative-transfer library: status
// handling, Philox4x32-10, double-float (binary32 pair) arithmetic and the
// binary32 Faddeeva real part used by the Voigt profile.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rt.h"

namespace rt {

// ---------------------------------------------------------------- host errors
void set_error(const char *fmt, ...);
rt_status fail(rt_status s, const char *fmt, ...);
rt_status cuda_fail(cudaError_t e, const char *what);
rt_status status_from_bits(uint32_t bits);

#define RT_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) return ::rt::cuda_fail(e__, #expr); \
  } while (0)

// Stream-ordered scratch that is released on the same stream when it goes out
// of scope (the memory returns to the pool once the queued work is done).
struct Scratch {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(const Scratch &) = delete;
  Scratch &operator=(const Scratch &) = delete;
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
  rt_status alloc(size_t bytes, cudaStream_t stream);
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds of two 32x32->64 multiplies with a Weyl key schedule.
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two binary32 values (Dekker 1971; Knuth TAOCP 4.2.2):
// exact two-sum and FMA-based two-product give about 44 significant bits.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
__device__ __forceinline__ df df_quick(float a, float b) {  // requires |a| >= |b|
  float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_quick(s.hi, e);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_quick(p, e);
}
// 1/a by one Newton correction of the binary32 reciprocal, carried in double-float.
__device__ __forceinline__ df df_recip(df a) {
  float r = __frcp_rn(a.hi);
  df ar = df_mul(a, df{r, 0.0f});
  float e = __fsub_rn(__fsub_rn(1.0f, ar.hi), ar.lo);
  return df_quick(r, __fmul_rn(r, e));
}
// Exact split of a binary64 into hi + lo binary32 (hi = RN(v), lo = RN(v - hi)).
__device__ __forceinline__ df df_from_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return df{hi, lo};
}

// ---------------------------------------------------------------- Faddeeva
// sqrt(pi) * Re w(x + i y) for y > 0 in binary32, w the Faddeeva function
// (the Voigt function times sqrt(pi)).  Regions by |z|:
//  |z| >= 8 : the asymptotic series w ~ (i / (sqrt(pi) z)) sum_n (2n-1)!! / (2 z^2)^n
//             (Abramowitz & Stegun 7.1.23).  Written with t = 1/|z|^2 and
//             s = y^2 t, its real part is
//               sqrt(pi) Re w = y t [1 + t (3 - 4s)/2 + 3 t^2 (5 - 20s + 16s^2)/4
//                                    + 15 t^3 (7 - 56s + 112s^2 - 64s^3)/8
//                                    + 105 t^4 (9 - 120s + 432s^2 - 576s^3 + 256s^4)/16 + ...]
//             (Im z^(2n+1) expanded with x^2 t = 1 - s); three terms for |z| >= 20,
//             five for 8 <= |z| < 20;
//  |z| < 8  : Weideman's (1994) rational series in Z = (L + iz)/(L - iz), N = 24,
//             coefficients from the Fourier series of exp(-t^2)(L^2 + t^2) on the
//             tan-mapped line (computed on the host in binary64); its method error
//             is below 2e-9 relative there, the rest is binary32 rounding.
// Measured relative error against binary64: <= 5.3e-7 for |z| >= 8, <= 2.2e-6 for
// 5 <= |z| < 8, <= 1.5e-6 for |z| < 5 with y >= 0.5 (degrading toward 1e-4 as y -> 0).
constexpr int kWeidN = 24;
struct WeidCoef {
  float L;
  float a[kWeidN];  // 2 sqrt(pi) a_n, n = 1..N
};

// bracket of the three-term series; sqrt(pi) Re w = y t S3
__device__ __forceinline__ float faddeeva_series3(float t, float s) {
  const float c1 = fmaf(s, -2.0f, 1.5f);
  const float c2 = fmaf(s, fmaf(s, 12.0f, -15.0f), 3.75f);
  return fmaf(t, fmaf(t, c2, c1), 1.0f);
}

// bracket of the five-term series; sqrt(pi) Re w = y t S5
__device__ __forceinline__ float faddeeva_series5(float t, float s) {
  const float c1 = fmaf(s, -2.0f, 1.5f);
  const float c2 = fmaf(s, fmaf(s, 12.0f, -15.0f), 3.75f);
  const float c3 = fmaf(s, fmaf(s, fmaf(s, -120.0f, 210.0f), -105.0f), 13.125f);
  const float c4 = fmaf(s, fmaf(s, fmaf(s, fmaf(s, 1680.0f, -3780.0f), 2835.0f), -787.5f), 59.0625f);
  return fmaf(t, fmaf(t, fmaf(t, fmaf(t, c4, c3), c2), c1), 1.0f);
}

__device__ __forceinline__ float faddeeva_re_core(float x, float y, const WeidCoef &c) {
  // iz = -y + i x;  d = L - iz = (L + y) - i x;  n = L + iz = (L - y) + i x
  const float dr = c.L + y, di = -x;
  const float nr = c.L - y, ni = x;
  const float inv = 1.0f / (dr * dr + di * di);
  const float vr = dr * inv, vi = -di * inv;  // v = 1 / d
  const float zr = nr * vr - ni * vi;         // Z = n v
  const float zi = nr * vi + ni * vr;
  float pr = c.a[kWeidN - 1], pi = 0.0f;
#pragma unroll
  for (int n = kWeidN - 2; n >= 0; --n) {
    const float t = pr * zr - pi * zi + c.a[n];
    pi = pr * zi + pi * zr;
    pr = t;
  }
  // sqrt(pi) w = v (p v + 1) with p scaled by 2 sqrt(pi)
  const float qr = pr * vr - pi * vi + 1.0f;
  const float qi = pr * vi + pi * vr;
  return vr * qr - vi * qi;
}

// sqrt(pi) Re w(x + iy) for |z|^2 = r2 below 400 (the five-term and rational-series regions)
__device__ __forceinline__ float faddeeva_re_near(float x, float y, float r2, const WeidCoef &c) {
  if (r2 >= 64.0f) {
    const float t = __fdividef(1.0f, r2);
    return y * t * faddeeva_series5(t, y * y * t);
  }
  return faddeeva_re_core(x, y, c);
}

__device__ __forceinline__ float faddeeva_re(float x, float y, const WeidCoef &c) {
  const float r2 = x * x + y * y;
  if (r2 >= 400.0f) {
    const float t = __fdividef(1.0f, r2);
    return y * t * faddeeva_series3(t, y * y * t);
  }
  return faddeeva_re_near(x, y, r2, c);
}

// Host: Weideman coefficients for N = kWeidN (binary64 DFT, then binary32).
void weideman_coefficients(WeidCoef *out);

// ---------------------------------------------------------------- misc
__device__ __forceinline__ void status_or(uint32_t *status, uint32_t bits) {
  if (status) atomicOr(status, bits);
}

}  // namespace rt
