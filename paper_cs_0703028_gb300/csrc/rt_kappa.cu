// Absorption-coefficient table on a temperature grid: Eqs. (S) and (tau) of
// Section 3, for one absorbing gas, with Lorentz or Voigt line shapes and a
// wing cutoff.  Five kernels:
//   k_line_geometry : per line, the binary64 grid decisions (cutoff window
//                     [j_lo, j_hi], nearest grid index j_c and offset) and the
//                     profile-evaluation count; validates device-resident lists.
//   k_prefactor     : per (T node, line), Eq. (S) times the number density and
//                     the width parameters, in binary32 with double-float
//                     arithmetic for the Boltzmann exponent; for Voigt lines
//                     also the far-wing polynomial coefficients.
//   k_tile_lines    : per 256-point wavenumber tile, the range of lines whose
//                     windows reach it, split into segments by kind: far lines
//                     (degree-1 or degree-2 far-wing series, masked where the
//                     window ends inside the tile), covering lines with the
//                     degree-4 series, and the general path (near-centre zone).
//   k_kappa         : per (tile, up to 8 T nodes), the line sum.  The tile's
//                     lines are staged in shared memory by bulk asynchronous
//                     copies (cp.async.bulk + mbarrier), double buffered; each
//                     lane owns 8 consecutive points (two float4 stores) and
//                     Kahan-sums over lines in ascending nu0.
//   k_kappa_ppl     : with a fixed number of points per line, one thread per
//                     point and eight T nodes over the few lines whose windows hold it.
#include <cmath>
#include <mutex>
#include <type_traits>

#include "rt_common.cuh"

namespace rt {
namespace {

constexpr int kPtsPerThread = 8;
constexpr int kTilePts = 32 * kPtsPerThread;  // 256 wavenumbers per block, one warp per T node
constexpr int kMaxTPerBlock = 8;              // warps (T nodes) per block
constexpr int kChunk = 96;                    // lines per staged chunk
constexpr int kGroup = 8;                     // fast-path lines summed before one compensated add
constexpr unsigned kWaitLimit = 1u << 22;     // bounded mbarrier waits

// CODATA 2018 (SI); derived quantities are formed on the host in binary64.
constexpr double kH = 6.62607015e-34, kC = 299792458.0, kKB = 1.380649e-23;
constexpr double kAmu = 1.66053906660e-27, kAtm = 101325.0;
constexpr double kPi = 3.14159265358979323846;

struct GeomParams {
  double nu_min, dnu, cutoff;
  long long n_nu, n_lines;
  int nT, check, ppl;
};

struct PrefParams {
  double T_min, T_max, T_ref;  // exact inputs, split into double-float in the kernel
  df c2;                       // second radiation constant h c / k_B, cm K
  float u_coef;                // x_ref p_ref atm / k_B * 1e-6  [cm^-3 K]
  float p_ref, n_T, q_exp;
  float doppler;               // sqrt(2 ln2 k_B / (m amu)) / c  [K^-1/2]
  float inv_dnu, dnu;
  long long n_lines;
  int nT, profile;
};

__device__ __forceinline__ double grid_nu(double nu_min, long long j, double dnu) {
  return __dadd_rn(nu_min, __dmul_rn((double)j, dnu));
}

__global__ void k_line_geometry(const double *__restrict__ nu0, const double *__restrict__ S,
                                const double *__restrict__ g, const double *__restrict__ E,
                                GeomParams P, int4 *__restrict__ R,
                                unsigned long long *evals, uint32_t *status) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (l < P.n_lines) {
    const double v = nu0[l];
    if (P.check) {
      const double s = S[l], gg = g[l], e = E[l];
      if (!isfinite(v) || !isfinite(s) || !(s > 0.0) || !isfinite(gg) || !(gg > 0.0) ||
          !isfinite(e) || !(e >= 0.0))
        status_or(status, RT_DEV_NONFINITE);
      if (l > 0 && !(nu0[l - 1] <= v)) status_or(status, RT_DEV_UNSORTED);
    }
    // nearest grid index: the origin of the line's local coordinate
    double fc = (v - P.nu_min) / P.dnu;
    fc = fmin(fmax(isfinite(fc) ? fc : 0.0, -536870912.0), 536870912.0);
    const long long jc = llrint(fc);
    const double dc = __dsub_rn(grid_nu(P.nu_min, jc, P.dnu), v);  // nu_jc - nu0
    const float dg = __double2float_rn(dc / P.dnu);                 // grid units
    // inclusive cutoff window: -cutoff <= nu_j - nu0 <= cutoff, in binary64
    double flo = floor((v - P.cutoff - P.nu_min) / P.dnu) - 1.0;
    double fhi = ceil((v + P.cutoff - P.nu_min) / P.dnu) + 1.0;
    flo = fmin(fmax(isfinite(flo) ? flo : 0.0, -1.0), (double)P.n_nu + 1.0);
    fhi = fmin(fmax(isfinite(fhi) ? fhi : 0.0, -2.0), (double)P.n_nu + 1.0);
    long long lo = (long long)flo, hi = (long long)fhi;
    if (P.ppl > 0) {  // fixed points per line around the centre
      double jf = floor((v - P.nu_min) / P.dnu);
      jf = fmin(fmax(isfinite(jf) ? jf : 0.0, -536870912.0), 536870912.0);
      lo = (long long)jf - P.ppl / 2 + 1;
      hi = (long long)jf + P.ppl / 2;
    }
    if (lo < 0) lo = 0;
    if (hi > P.n_nu - 1) hi = P.n_nu - 1;
    if (P.ppl <= 0) {
#pragma unroll 1
      for (int it = 0; it < 6 && lo < P.n_nu; ++it)
        if (__dsub_rn(grid_nu(P.nu_min, lo, P.dnu), v) < -P.cutoff) ++lo;
#pragma unroll 1
      for (int it = 0; it < 6 && hi >= 0; ++it)
        if (__dsub_rn(grid_nu(P.nu_min, hi, P.dnu), v) > P.cutoff) --hi;
    }
    R[l] = make_int4((int)lo, (int)hi, (int)jc, __float_as_int(dg));
    if (hi >= lo) cnt = (unsigned long long)(hi - lo + 1) * (unsigned long long)P.nT;
  }
  if (evals) {
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(evals, cnt);
  }
}

// Eq. (S) times the number density, and the profile's coefficients, for line l
// at T node k.  Voigt: P = {c0, s dnu, y^2, c2}, P2 = {c3, c4, half-widths of |z| < 20 and < 10}
// with the far-wing series c0 t + c1 t^2 + c2 t^3 + c3 t^4 + c4 t^5 (c1 = 1.5 c0).
// Writes the line's far-zone distances in grid units (float bits): beyond far[0]
// the t^4 and t^5 terms are below 2^-24 of the value (27 y^2 t^3 <= 2^-24 with
// t <= 1/x^2), so a degree-2 series is within one binary32 rounding of the full
// one; beyond far[1] (>= far[0]) also (3.75 + 2 y^2) t^2 <= 2^-25, so the degree-1
// series drops at most 1.25 * 2^-24 of the value.
// The quantities of T node k that every line shares.
struct PrefNode {
  df Tk, iT, iTref;
  float tr, qratio, wratio, sqrtT;
};

__device__ __forceinline__ PrefNode pref_node(const PrefParams &Q, int k) {
  // T_k = T_min + k (T_max - T_min) / (nT - 1) and 1/T_k in double-float
  PrefNode N;
  df Tk = df_from_double(Q.T_min);
  if (Q.nT > 1) {
    const df span = df_add(df_from_double(Q.T_max), df_neg(Tk));
    const df step = df_mul(span, df_recip(df{(float)(Q.nT - 1), 0.0f}));
    Tk = df_add(Tk, df_mul(step, df{(float)k, 0.0f}));
  }
  N.Tk = Tk;
  N.iT = df_recip(Tk);
  const df Tref = df_from_double(Q.T_ref);
  N.iTref = df_recip(Tref);
  N.tr = Tref.hi * N.iT.hi;  // T_ref / T
  N.qratio = powf(N.tr, Q.q_exp);
  N.wratio = powf(N.tr, Q.n_T);
  N.sqrtT = sqrtf(Tk.hi);
  return N;
}

__device__ __forceinline__ void prefactor_one(const double *__restrict__ nu0, const double *__restrict__ S,
                                                  const double *__restrict__ g, const double *__restrict__ E,
                                                  const PrefParams &Q, const PrefNode &N,
                                                  float4 *__restrict__ Pout, float4 *__restrict__ P2out,
                                                  long long l, int k, unsigned (&far)[2]) {
  const df iT = N.iT, iTref = N.iTref;
  const float iTf = iT.hi;
  // Eq. (S): Q ratio, Boltzmann ratio (exponent in double-float), stimulated emission
  const float qratio = N.qratio;
  const df arg = df_mul(df_mul(Q.c2, df_from_double(E[l])), df_add(iTref, df_neg(iT)));
  const float boltz = expf(arg.hi) * (1.0f + arg.lo);
  const float nu0f = __double2float_rn(nu0[l]);
  const float c2nu = Q.c2.hi * nu0f;
  const float stim = expm1f(-c2nu * iTf) / expm1f(-c2nu * iTref.hi);
  const float S_T = __double2float_rn(S[l]) * qratio * boltz * stim;
  const float A = (Q.u_coef * iTf) * S_T;  // u(T) S(T), cm^-1 per unit profile
  const float gam = __double2float_rn(g[l]) * Q.p_ref * N.wratio;
  float4 out;
  far[0] = far[1] = 0;
  if (Q.profile == RT_PROFILE_LORENTZ) {
    const float gg = gam * Q.inv_dnu;  // half-width in grid units
    out = make_float4(A * gg * (float)(1.0 / kPi) * Q.inv_dnu, gg * gg, 0.0f, 0.0f);
  } else {
    const float alpha = nu0f * N.sqrtT * Q.doppler;  // Doppler HWHM, cm^-1
    const float s = 0.83255461f / alpha;                  // sqrt(ln 2) / alpha
    const float y = s * gam;
    const float sd = s * Q.dnu;
    // half-width (grid units) of the region |z| < 20 where the far-wing series does not hold
    const float y2 = y * y;
    const float u_near = sqrtf(fmaxf(400.0f - y2, 0.0f)) / sd;
    // far wing: c0 t (1 + 1.5 t + (3.75 - 2 y^2) t^2 - 15 y^2 t^3 + 12 y^4 t^4), t = 1/|z|^2
    const float c0 = A * s * (float)(1.0 / kPi) * y;
    out = make_float4(c0, sd, y2, __fmaf_rn(-2.0f, y2, 3.75f) * c0);
    // half-width (grid units) of |z| < 10, inside which the general path takes the near form
    const float u_core = sqrtf(fmaxf(100.0f - y2, 0.0f)) / sd;
    P2out[(long long)k * Q.n_lines + l] = make_float4(-15.0f * y2 * c0, 12.0f * y2 * y2 * c0, u_near, u_core);
    // (27 y^2 / 2^-24)^(1/6) = 27.66 y^(1/3) and (2^25 (3.75 + 2 y^2))^(1/4), with 5 %
    // margin, in grid units
    const float d2 = 29.1f * cbrtf(y) / sd;
    const float d1 = fmaxf(1.05f * sqrtf(sqrtf(33554432.0f * (3.75f + 2.0f * y2))) / sd, d2);
    far[0] = (d2 >= 0.0f && d2 < 1e9f) ? __float_as_uint(d2) : __float_as_uint(1e9f);
    far[1] = (d1 >= 0.0f && d1 < 1e9f) ? __float_as_uint(d1) : __float_as_uint(1e9f);
  }
  Pout[(long long)k * Q.n_lines + l] = out;
}

__global__ void k_prefactor(const double *__restrict__ nu0, const double *__restrict__ S,
                            const double *__restrict__ g, const double *__restrict__ E,
                            PrefParams Q, float4 *__restrict__ Pout, float4 *__restrict__ P2out,
                            unsigned *__restrict__ far_bits) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  __shared__ PrefNode s_node;  // T node k's shared quantities, formed once per block
  if (threadIdx.x == 0) s_node = pref_node(Q, k);
  __syncthreads();
  const PrefNode N = s_node;
  unsigned fb[2] = {0, 0};  // this line's far-zone distances (grid units, float bits)
  if (l < Q.n_lines) prefactor_one(nu0, S, g, E, Q, N, Pout, P2out, l, k, fb);
  // block maxima, one atomic each per block (non-negative floats order like their bits)
  __shared__ unsigned s_max[2][32];
  for (int d = 0; d < 2; ++d) {
    const unsigned m = __reduce_max_sync(0xffffffffu, fb[d]);
    if ((threadIdx.x & 31) == 0) s_max[d][threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    unsigned m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_max[threadIdx.x][w]);
    if (m) atomicMax(far_bits + threadIdx.x, m);
  }
}


// ---- bulk asynchronous copies global -> shared, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ long long lower_bound_hi(const int4 *R, long long n, int j) {
  long long a = 0, b = n;  // first l with R[l].y >= j
  while (a < b) {
    long long m = (a + b) >> 1;
    if (R[m].y < j) a = m + 1; else b = m;
  }
  return a;
}
__device__ __forceinline__ long long lower_bound_lo(const int4 *R, long long n, int j) {
  long long a = 0, b = n;  // first l with R[l].x >= j
  while (a < b) {
    long long m = (a + b) >> 1;
    if (R[m].x < j) a = m + 1; else b = m;
  }
  return a;
}

// Kinds of line ranges within a tile (see k_tile_lines).
enum SegKind : int {
  kSegGeneral = 0,   // window masking and near-centre test per line
  kSegFast = 1,      // covering, degree-4 far-wing series
  kSegFar2 = 2,      // covering, degree-2 series
  kSegFar1 = 3,      // covering, degree-1 series
  kSegFar2Masked = 4,
  kSegFar1Masked = 5,
};
constexpr int kMaxSegs = 12;
constexpr int kTileInts = 5;  // int4 per tile: {lb, ub, nseg, 0}, 12 ends, 16 kind bytes

// Per tile of kTilePts wavenumbers [jw0, jw0 + kTilePts): the lines [lb, ub)
// whose windows reach it, split into ranges by kind.  Windows and centres are
// monotone in the (sorted) line index, so every set below is an index range:
//   cover : j_lo <= jw0 and j_hi >= jw0 + kTilePts - 1 (no masking needed);
//   near  : j_c within W + 4 grid points of the tile, W bounding the near-centre
//           half-width of every line (lines outside it have no point |z| < 20);
//   far2 / far1 : j_c more than D2 / D1 grid points from the tile, D1 >= D2 >= W + 4
//           bounding every line's far-zone distances (degree-2 / degree-1 series).
// Covering lines are far1, far2, fast or (near) general; partially covering
// lines are far1-masked, far2-masked or general.
__global__ void k_tile_lines(const int4 *__restrict__ R, long long n, long long n_nu, int W,
                             const unsigned *__restrict__ far_bits, long long n_tiles,
                             int4 *__restrict__ out) {
  // one warp per tile: lanes 0..9 run the tile's ten binary searches side by side
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_tiles) return;  // warp-uniform
  const long long D2 = max((long long)W + 4, (long long)ceilf(fminf(__uint_as_float(far_bits[0]), 1e9f)) + 2);
  const long long D1 = max(D2, (long long)ceilf(fminf(__uint_as_float(far_bits[1]), 1e9f)) + 2);
  const long long jw0 = t * kTilePts, jw1 = jw0 + kTilePts - 1;
  const long long jend = min(jw0 + (long long)kTilePts, n_nu);
  // search i: the first line whose field (0: window start, 1: window end, 2: centre) >= key
  const int fld = (lane == 1 || lane == 3) ? 0 : ((lane == 0 || lane == 2) ? 1 : 2);
  const long long key = lane == 0 ? jw0 : lane == 1 ? jend : lane == 2 ? jw1 : lane == 3 ? jw0 + 1
                        : lane == 4 ? jw0 - D1 : lane == 5 ? jw0 - D2 : lane == 6 ? jw0 - W - 4
                        : lane == 7 ? jw1 + W + 5 : lane == 8 ? jw1 + D2 + 1 : jw1 + D1 + 1;
  long long a = 0, e = n;
  if (lane < 10) {
    while (a < e) {
      const long long m = (a + e) >> 1;
      const int4 r = __ldg(R + m);
      const long long v = fld == 0 ? r.x : (fld == 1 ? r.y : r.z);
      if (v < key) a = m + 1; else e = m;
    }
  }
  long long sr[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) sr[i] = __shfl_sync(0xffffffffu, a, i);
  if (lane != 0) return;
  const long long lb = sr[0];
  const long long ub = max(lb, sr[1]);
  auto cl = [&](long long v) { return min(max(v, lb), ub); };
  const long long ca = cl(sr[2]);   // cover = [ca, cb)
  const long long cb = cl(sr[3]);
  const long long f1a = cl(sr[4]);  // far1: l < f1a or l >= f1b
  const long long f2a = cl(sr[5]);  // far2: l < f2a or l >= f2b
  const long long na = cl(sr[6]);   // near: [na, nb)
  const long long nb = cl(sr[7]);
  const long long f2b = cl(sr[8]);
  const long long f1b = cl(sr[9]);
  auto kind = [&](long long l) -> int {
    const bool far1 = l < f1a || l >= f1b, far2 = l < f2a || l >= f2b;
    if (l < ca || l >= cb) return far1 ? kSegFar1Masked : (far2 ? kSegFar2Masked : kSegGeneral);
    if (far1) return kSegFar1;
    if (far2) return kSegFar2;
    if (l < na || l >= nb) return kSegFast;
    return kSegGeneral;
  };
  // the change points, sorted; one segment per maximal run of equal kind
  long long b[9] = {ca, cb, f1a, f2a, na, nb, f2b, f1b, ub};
  for (int i = 1; i < 8; ++i)
    for (int j = i; j > 0 && b[j - 1] > b[j]; --j) {
      const long long x = b[j - 1]; b[j - 1] = b[j]; b[j] = x;
    }
  int ends[kMaxSegs];
  unsigned char kinds[16] = {};
  int nseg = 0;
  long long start = lb;
  for (int i = 0; i < 9; ++i) {
    const long long e = b[i];
    if (e <= start) continue;
    const int kd = kind(start);
    if (nseg > 0 && kinds[nseg - 1] == kd) {
      ends[nseg - 1] = (int)e;
    } else {
      kinds[nseg] = (unsigned char)kd;
      ends[nseg++] = (int)e;
    }
    start = e;
  }
  for (int i = nseg; i < kMaxSegs; ++i) ends[i] = (int)ub;
  int4 *o = out + kTileInts * t;
  o[0] = make_int4((int)lb, (int)ub, nseg, 0);
  for (int i = 0; i < 3; ++i) o[1 + i] = make_int4(ends[4 * i], ends[4 * i + 1], ends[4 * i + 2], ends[4 * i + 3]);
  int kw[4];
  for (int i = 0; i < 4; ++i)
    kw[i] = kinds[4 * i] | (kinds[4 * i + 1] << 8) | (kinds[4 * i + 2] << 16) | (kinds[4 * i + 3] << 24);
  o[4] = make_int4(kw[0], kw[1], kw[2], kw[3]);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Paired binary32 arithmetic (one f32x2 instruction for two lanes' worth of
// work): each component is rounded exactly as the scalar __fmaf_rn /
// __fadd_rn, so the paired forms give the same bits as the scalar ones.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rcp2(float2 d) { return make_float2(rcp_approx(d.x), rcp_approx(d.y)); }

// compensated (Kahan) add of v into s with running compensation c, per component
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 v) {
  const float2 y = __fadd2_rn(v, neg2(c));
  const float2 t = __fadd2_rn(s, y);
  c = __fadd2_rn(__fadd2_rn(t, neg2(s)), neg2(y));
  s = t;
}

// Block = 256 consecutive wavenumbers x up to 8 temperature nodes (one warp per
// node, 8 consecutive points per lane).  All warps walk the same lines: the
// block's lines are staged chunk by chunk (geometry R once, coefficients P and,
// for Voigt, P2 per node) with bulk asynchronous copies on an mbarrier, double
// buffered.  A point's offset from a line centre, in grid units, is the exact
// integer j - j_c plus the binary32 sub-grid offset of the centre, so its
// rounding error is relative to the distance itself.
// Voigt far wing (|z| >= 20): with t = 1/|z|^2 the three-term series is the
// polynomial c0 t + c1 t^2 + c2 t^3 + c3 t^4 + c4 t^5 (coefficients from
// k_prefactor).  The binary32 arithmetic runs on pairs of a lane's points (f32x2
// instructions).  Fast-path lines (whole tile covered, no near-centre point, or
// far lines with masked window ends) add kGroup lines per compensated add; the
// general-path lines evaluate a four-term series, replace the points of their
// contiguous near-centre range by faddeeva_re_near (one point per lane, handed
// back through shared memory), mask the ends of their windows, and add in pairs.
// Lorentz: P = {A g / (pi dnu), g^2}.
template <int PROFILE>
__global__ void __launch_bounds__(32 * kMaxTPerBlock, 3)
k_kappa(const float4 *__restrict__ P, const float4 *__restrict__ P2, const int4 *__restrict__ R,
        const int4 *__restrict__ tiles, long long n_lines, long long n_nu, int nT, WeidCoef wc,
        int vec_ok, int accumulate, float *__restrict__ kappa, uint32_t *status) {
  constexpr bool kVoigt = PROFILE == RT_PROFILE_VOIGT;
  constexpr int kPSets = kVoigt ? 2 : 1;
  __shared__ __align__(16) int4 sR[2][kChunk];
  __shared__ __align__(16) float4 sP[2][kPSets][kMaxTPerBlock][kChunk];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ float s_res[kMaxTPerBlock][kTilePts];          // near-centre values by tile point

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tpb = blockDim.x >> 5;
  const int k0 = blockIdx.y * tpb;
  const int nk = min(tpb, nT - k0);          // T nodes of this block
  const int k = k0 + min(warp, nk - 1);      // surplus warps shadow the last node, store nothing
  const long long j0 = (long long)blockIdx.x * kTilePts;
  const long long jend = min(j0 + (long long)kTilePts, n_nu);
  const int jw0 = (int)j0, jw1 = jw0 + kTilePts - 1;
  const int jt = jw0 + lane * kPtsPerThread;
  // offset of point j from a line centre j_c with sub-grid offset dg: the exact
  // integer difference, then one rounding
  auto point_offset = [&](int j, int jc, int dg_bits) -> float {
    return __fadd_rn((float)(j - jc), __int_as_float(dg_bits));
  };

  __shared__ int s_end[kMaxSegs];
  __shared__ unsigned char s_kind[kMaxSegs];
  const int4 *tinfo = tiles + (long long)kTileInts * blockIdx.x;
  const int4 ta = __ldg(tinfo);
  const int lb = ta.x, ub = ta.y;
  if (threadIdx.x < kMaxSegs) {
    const int q = threadIdx.x & 3;
    const int4 e = __ldg(tinfo + 1 + (threadIdx.x >> 2));
    const int4 kw = __ldg(tinfo + 4);
    const int w = (threadIdx.x >> 2) == 0 ? kw.x : ((threadIdx.x >> 2) == 1 ? kw.y : kw.z);
    s_end[threadIdx.x] = q == 0 ? e.x : (q == 1 ? e.y : (q == 2 ? e.z : e.w));
    s_kind[threadIdx.x] = (unsigned char)((w >> (8 * q)) & 255);
  }
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nchunks = (ub - lb + kChunk - 1) / kChunk;

  auto issue = [&](int c) {
    const long long l0 = (long long)lb + (long long)c * kChunk;
    const uint32_t cnt = (uint32_t)min((long long)kChunk, (long long)ub - l0);
    const int b = c & 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bars[b], cnt * 16u * (uint32_t)(kPSets * nk + 1));
    bulk_g2s(&sR[b][0], R + l0, cnt * 16u, &bars[b]);
    for (int w = 0; w < nk; ++w) {
      bulk_g2s(&sP[b][0][w][0], P + (long long)(k0 + w) * n_lines + l0, cnt * 16u, &bars[b]);
      if (kVoigt) bulk_g2s(&sP[b][kPSets - 1][w][0], P2 + (long long)(k0 + w) * n_lines + l0, cnt * 16u, &bars[b]);
    }
  };

  // compensated sums for the lane's points, as pairs (2h, 2h + 1)
  constexpr int kPairs = kPtsPerThread / 2;
  float2 acc[kPairs], cmp[kPairs];
#pragma unroll
  for (int h = 0; h < kPairs; ++h) acc[h] = cmp[h] = make_float2(0.0f, 0.0f);
  if (threadIdx.x == 0) {
    if (nchunks > 0) issue(0);
    if (nchunks > 1) issue(1);
  }
  const int wsel = min(warp, nk - 1);
  int seg = 0;  // current segment, carried across chunks
  bool aborted = false;
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    const uint32_t parity = (uint32_t)((c >> 1) & 1);
    unsigned spins = 0;
    int timed_out = 0;
    while (!mbar_try_wait(&bars[b], parity)) {
      if (++spins > kWaitLimit) {
        timed_out = 1;
        break;
      }
    }
    if (__syncthreads_or(timed_out)) {  // the block leaves together
      if (threadIdx.x == 0) {
        status_or(status, RT_DEV_TIMEOUT);
        // The copies of this chunk and of the next one (issued one chunk ahead) may
        // still be writing into this block's shared memory: wait for them, again with
        // a bound, so that no copy lands after the block has released it.
        for (int d = c; d < min(c + 2, nchunks); ++d) {
          unsigned n = 0;
          while (!mbar_try_wait(&bars[d & 1], (uint32_t)((d >> 1) & 1)) && ++n <= kWaitLimit) {
          }
        }
      }
      aborted = true;
      break;
    }
    const int l0 = lb + c * kChunk;
    const int cnt = min(kChunk, ub - l0);

    // fast paths: g[q] += value of line i at the lane's points (or = when first).
    // DEG 4: full far-wing series; DEG 2: far lines (t^3 and t^4 terms negligible);
    // MASK: zero outside the line's window.
    auto fast_line = [&](auto deg, auto mask, int i, float2 (&g)[kPairs], bool first) {
      constexpr int DEG = decltype(deg)::value;
      constexpr bool MASK = decltype(mask)::value;
      const int4 r = sR[b][i];
      const float4 p = sP[b][0][wsel][i];
      const float ul = point_offset(jt, r.z, r.w);
      if (!kVoigt) {
        const float2 u0 = dup2(ul), g2 = dup2(p.y), a2 = dup2(p.x);
#pragma unroll
        for (int h = 0; h < kPairs; ++h) {
          const float2 u = __fadd2_rn(u0, make_float2((float)(2 * h), (float)(2 * h + 1)));
          float2 rr = rcp2(__ffma2_rn(u, u, g2));
          if (MASK) {
            if (jt + 2 * h < r.x || jt + 2 * h > r.y) rr.x = 0.0f;
            if (jt + 2 * h + 1 < r.x || jt + 2 * h + 1 > r.y) rr.y = 0.0f;
          }
          g[h] = first ? __fmul2_rn(a2, rr) : __ffma2_rn(a2, rr, g[h]);
        }
      } else {
        const float2 c0 = dup2(p.x), c1 = dup2(1.5f * p.x), sd = dup2(p.y), y2 = dup2(p.z);
        const float2 xt = dup2(p.y * ul);
        float4 p2 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (DEG == 4) p2 = sP[b][kPSets - 1][wsel][i];
#pragma unroll
        for (int h = 0; h < kPairs; ++h) {
          const float2 x = __ffma2_rn(sd, make_float2((float)(2 * h), (float)(2 * h + 1)), xt);
          const float2 t = rcp2(__ffma2_rn(x, x, y2));
          float2 v;
          if (DEG == 4)
            v = __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, dup2(p2.y), dup2(p2.x)), dup2(p.w)), c1), c0);
          else if (DEG == 2)
            v = __ffma2_rn(t, __ffma2_rn(t, dup2(p.w), c1), c0);
          else
            v = __ffma2_rn(t, c1, c0);
          if (MASK) {
            if (jt + 2 * h < r.x || jt + 2 * h > r.y) v.x = 0.0f;
            if (jt + 2 * h + 1 < r.x || jt + 2 * h + 1 > r.y) v.y = 0.0f;
          }
          g[h] = first ? __fmul2_rn(t, v) : __ffma2_rn(t, v, g[h]);
        }
      }
    };
    auto run_fast = [&](auto deg, auto mask, int i, int i1) {
#pragma unroll 1
      for (; i + kGroup <= i1; i += kGroup) {
        float2 g[kPairs];
        fast_line(deg, mask, i, g, true);
#pragma unroll
        for (int e = 1; e < kGroup; ++e) fast_line(deg, mask, i + e, g, false);
#pragma unroll
        for (int h = 0; h < kPairs; ++h) kahan_add2(acc[h], cmp[h], g[h]);
      }
      if (i < i1) {
        float2 g[kPairs];
        fast_line(deg, mask, i, g, true);
#pragma unroll 1
        for (int e = i + 1; e < i1; ++e) fast_line(deg, mask, e, g, false);
#pragma unroll
        for (int h = 0; h < kPairs; ++h) kahan_add2(acc[h], cmp[h], g[h]);
      }
    };

    // general path: the value of line i at the lane's points, with masking
    // outside the window and near-centre points
    auto line_vals = [&](int i, float2 (&v)[kPairs]) {
        const int4 r = sR[b][i];
        const float4 p = sP[b][0][wsel][i];
        const float ul = point_offset(jt, r.z, r.w);
        if (!kVoigt) {
          const float2 u0 = dup2(ul), g2 = dup2(p.y), a2 = dup2(p.x);
#pragma unroll
          for (int h = 0; h < kPairs; ++h) {
            const float2 u = __fadd2_rn(u0, make_float2((float)(2 * h), (float)(2 * h + 1)));
            v[h] = __fmul2_rn(a2, rcp2(__ffma2_rn(u, u, g2)));
          }
        } else {
          const float4 p2 = sP[b][kPSets - 1][wsel][i];
          const float y2 = p.z;
          const float2 y22 = dup2(y2), sd = dup2(p.y), xt = dup2(p.y * ul);
          // four-term series, valid for |z| >= 10: the degree-4 polynomial plus the
          // fourth term 15 t^3 (7 - 56 s + 112 s^2 - 64 s^3) / 8, s = y^2 t, in t
          const float q1 = y2 * p.x, q2 = q1 * y2;
          const float2 c3 = dup2(__fmaf_rn(13.125f, p.x, p2.x)), c4 = dup2(__fmaf_rn(-105.0f, q1, p2.y));
          const float2 c5 = dup2(210.0f * q2), c6 = dup2(-120.0f * q2 * y2);
          const float2 c0 = dup2(p.x), c1 = dup2(1.5f * p.x), c2 = dup2(p.w);
#pragma unroll
          for (int h = 0; h < kPairs; ++h) {
            const float2 x = __ffma2_rn(sd, make_float2((float)(2 * h), (float)(2 * h + 1)), xt);
            const float2 t = rcp2(__ffma2_rn(x, x, y22));
            const float2 w = __ffma2_rn(
                t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, __ffma2_rn(t, c6, c5), c4), c3), c2), c1),
                c0);
            v[h] = __fmul2_rn(t, w);
          }
          // warp-uniform: the tile's offsets [fu, fu + kTilePts) meet the region |z| < 10,
          // |u| < u_core in grid units; its points are the contiguous tile indices [ea, eb]
          // (one point of margin each side: the near form holds at any |z|), evaluated
          // one per lane and handed to their owners through shared memory
          const float fu = (float)(jw0 - r.z) + __int_as_float(r.w);
          if (fu < p2.w + 1.0f && fu + (float)kTilePts > -p2.w - 1.0f) {
            const int ea = (int)fmaxf(floorf(-p2.w - 1.0f - fu), 0.0f);
            const int eb = (int)fminf(ceilf(p2.w + 1.0f - fu), (float)(kTilePts - 1));
            float *res = s_res[warp];
            const float y = sqrtf(y2);
            const float coef = __fdividef(p.x, y);
            for (int e = ea + lane; e <= eb; e += 32) {
              const float xe = p.y * point_offset(jw0 + e, r.z, r.w);
              res[e] = coef * faddeeva_re_near(xe, y, __fmaf_rn(xe, xe, y2), wc);
            }
            __syncwarp();
            const int p0 = lane * kPtsPerThread;
            if (p0 + kPtsPerThread > ea && p0 <= eb) {
#pragma unroll
              for (int h = 0; h < kPairs; ++h) {
                if (p0 + 2 * h >= ea && p0 + 2 * h <= eb) v[h].x = res[p0 + 2 * h];
                if (p0 + 2 * h + 1 >= ea && p0 + 2 * h + 1 <= eb) v[h].y = res[p0 + 2 * h + 1];
              }
            }
            __syncwarp();
          }
        }
        if (r.x > jw0 || r.y < jw1) {  // warp-uniform: the window ends inside this block's points
#pragma unroll
          for (int h = 0; h < kPairs; ++h) {
            if (jt + 2 * h < r.x || jt + 2 * h > r.y) v[h].x = 0.0f;
            if (jt + 2 * h + 1 < r.x || jt + 2 * h + 1 > r.y) v[h].y = 0.0f;
          }
        }
    };
    // lines enter the compensated sum in pairs: the sum of two positive line
    // values is rounded once (relative error <= 2^-24 of the pair)
    auto run_general = [&](int i, int i1) {
#pragma unroll 1
      for (; i + 1 < i1; i += 2) {
        float2 va[kPairs], vb[kPairs];
        line_vals(i, va);
        line_vals(i + 1, vb);
#pragma unroll
        for (int h = 0; h < kPairs; ++h) kahan_add2(acc[h], cmp[h], __fadd2_rn(va[h], vb[h]));
      }
      if (i < i1) {
        float2 va[kPairs];
        line_vals(i, va);
#pragma unroll
        for (int h = 0; h < kPairs; ++h) kahan_add2(acc[h], cmp[h], va[h]);
      }
    };

    // the chunk [l0, l0 + cnt) split at the tile's segment ends (block-uniform)
    int i = 0;
#pragma unroll 1
    while (i < cnt) {
      const int l = l0 + i;
      while (s_end[seg] <= l) ++seg;  // the last segment ends at ub > l
      const int i1 = min(cnt, s_end[seg] - l0);
      const int kd = s_kind[seg];
      if (kd == kSegFar1)
        run_fast(std::integral_constant<int, 1>(), std::false_type(), i, i1);
      else if (kd == kSegFar2)
        run_fast(std::integral_constant<int, 2>(), std::false_type(), i, i1);
      else if (kd == kSegFast)
        run_fast(std::integral_constant<int, 4>(), std::false_type(), i, i1);
      else if (kd == kSegFar1Masked)
        run_fast(std::integral_constant<int, 1>(), std::true_type(), i, i1);
      else if (kd == kSegFar2Masked)
        run_fast(std::integral_constant<int, 2>(), std::true_type(), i, i1);
      else
        run_general(i, i1);
      i = i1;
    }
    __syncthreads();  // every warp is done with buffer b
    if (threadIdx.x == 0 && c + 2 < nchunks) issue(c + 2);
  }
  if (aborted || warp >= nk) return;

  float *row = kappa + (long long)k * n_nu;
  float out[kPtsPerThread];
#pragma unroll
  for (int h = 0; h < kPairs; ++h) {
    out[2 * h] = __fsub_rn(acc[h].x, cmp[h].x);
    out[2 * h + 1] = __fsub_rn(acc[h].y, cmp[h].y);
  }
  if ((long long)jt + kPtsPerThread <= jend && vec_ok) {
#pragma unroll
    for (int q4 = 0; q4 < kPtsPerThread; q4 += 4) {
      float4 *dst = reinterpret_cast<float4 *>(row + jt + q4);
      if (accumulate) {
        const float4 o = *dst;
        out[q4] += o.x; out[q4 + 1] += o.y; out[q4 + 2] += o.z; out[q4 + 3] += o.w;
      }
      *dst = make_float4(out[q4], out[q4 + 1], out[q4 + 2], out[q4 + 3]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < kPtsPerThread; ++q)
      if ((long long)jt + q < jend) row[jt + q] = accumulate ? row[jt + q] + out[q] : out[q];
  }
}

// Fixed points per line (each line on the few grid points around its centre):
// one thread per point j, looping over kPplNodes T nodes; the lines whose windows
// hold j are a contiguous index range (windows are monotone in the sorted line
// index), found once per thread by binary search within the block's range, and
// summed in ascending nu0 with compensation at each node.  Every point is near its
// lines' centres, so each value is the near-centre form (faddeeva_re_near) rather
// than a far-wing series.
constexpr int kPplNodes = 8;

template <int PROFILE>
__global__ void __launch_bounds__(kTilePts)
k_kappa_ppl(const float4 *__restrict__ P, const int4 *__restrict__ R, long long n_lines, long long n_nu,
            int nT, WeidCoef wc, int accumulate, float *__restrict__ kappa) {
  __shared__ long long s_range[2];
  const long long jw0 = (long long)blockIdx.x * kTilePts;
  const long long jend = min(jw0 + (long long)kTilePts, n_nu);
  const int k0 = blockIdx.y * kPplNodes, k1 = min(k0 + kPplNodes, nT);
  if (threadIdx.x == 0) s_range[0] = lower_bound_hi(R, n_lines, (int)jw0);
  if (threadIdx.x == 1) s_range[1] = lower_bound_lo(R, n_lines, (int)jend);
  __syncthreads();
  const long long j = jw0 + threadIdx.x;
  if (j >= n_nu) return;
  // lines [a, b) of the block's range with hi >= j and lo <= j
  long long a = s_range[0], hi_end = max(s_range[0], s_range[1]);
  while (a < hi_end) {
    const long long m = (a + hi_end) >> 1;
    if (__ldg(&R[m].y) < (int)j) a = m + 1; else hi_end = m;
  }
  long long b = a, b_end = max(s_range[0], s_range[1]);
  while (b < b_end) {
    const long long m = (b + b_end) >> 1;
    if (__ldg(&R[m].x) <= (int)j) b = m + 1; else b_end = m;
  }
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const float4 *Pk = P + (long long)k * n_lines;
    float acc = 0.0f, cmp = 0.0f;
    for (long long l = a; l < b; ++l) {
      const int4 r = __ldg(R + l);
      const float4 p = __ldg(Pk + l);
      const float u = __fadd_rn((float)((int)j - r.z), __int_as_float(r.w));
      float v;
      if (PROFILE == RT_PROFILE_LORENTZ) {
        v = p.x * rcp_approx(__fmaf_rn(u, u, p.y));
      } else {
        const float x = p.y * u;
        const float y = sqrtf(p.z);
        v = __fdividef(p.x, y) * faddeeva_re_near(x, y, __fmaf_rn(x, x, p.z), wc);
      }
      const float yk = __fsub_rn(v, cmp);
      const float t = __fadd_rn(acc, yk);
      cmp = __fsub_rn(__fsub_rn(t, acc), yk);
      acc = t;
    }
    float *dst = kappa + (long long)k * n_nu + j;
    const float out = __fsub_rn(acc, cmp);
    *dst = accumulate ? *dst + out : out;
  }
}

// ---- adaptive points per line
// Each line's window at each T node: |nu_j - nu0| <= w = min(cutoff, sqrt(A gamma /
// (pi kappa_min))) with A = u(T_k) S(T_k) and gamma the Lorentz half-width at T_k, in
// binary64 in the order the float64 reading states it (number density x p atm / (k_B T)
// 1e-6, Eq. (S) as S_ref (T_ref/T)^q Boltzmann ratio stimulated-emission ratio).
struct AdaptParams {
  double nu_min, dnu, cutoff, T_min, T_max, T_ref, c2, x_ref, p_ref, n_T, q_exp, kappa_min;
  long long n_nu, n_lines;
  int nT;
};

__global__ void k_adaptive_windows(const double *__restrict__ nu0, const double *__restrict__ S,
                                   const double *__restrict__ g, const double *__restrict__ E, AdaptParams P,
                                   int2 *__restrict__ AW, unsigned long long *evals) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  unsigned long long cnt = 0;
  if (l < P.n_lines) {
    const double T = P.nT > 1 ? P.T_min + (double)k * ((P.T_max - P.T_min) / (double)(P.nT - 1)) : P.T_min;
    const double v = nu0[l];
    const double q = pow(P.T_ref / T, P.q_exp);
    const double boltz = exp(-P.c2 * E[l] / T) / exp(-P.c2 * E[l] / P.T_ref);
    const double stim = (-expm1(-P.c2 * v / T)) / (-expm1(-P.c2 * v / P.T_ref));
    const double ST = S[l] * q * boltz * stim;
    const double A = P.x_ref * P.p_ref * kAtm / (kKB * T) * 1e-6 * ST;
    const double gam = g[l] * P.p_ref * pow(P.T_ref / T, P.n_T);
    double w = sqrt(A * gam / (kPi * P.kappa_min));
    if (!(w <= P.cutoff)) w = P.cutoff;
    double flo = floor((v - w - P.nu_min) / P.dnu) - 1.0;
    double fhi = ceil((v + w - P.nu_min) / P.dnu) + 1.0;
    flo = fmin(fmax(isfinite(flo) ? flo : 0.0, -1.0), (double)P.n_nu + 1.0);
    fhi = fmin(fmax(isfinite(fhi) ? fhi : 0.0, -2.0), (double)P.n_nu + 1.0);
    long long lo = (long long)flo, hi = (long long)fhi;
    if (lo < 0) lo = 0;
    if (hi > P.n_nu - 1) hi = P.n_nu - 1;
#pragma unroll 1
    for (int it = 0; it < 6 && lo < P.n_nu; ++it)
      if (__dsub_rn(grid_nu(P.nu_min, lo, P.dnu), v) < -w) ++lo;
#pragma unroll 1
    for (int it = 0; it < 6 && hi >= 0; ++it)
      if (__dsub_rn(grid_nu(P.nu_min, hi, P.dnu), v) > w) --hi;
    AW[(long long)k * P.n_lines + l] = make_int2((int)lo, (int)hi);
    if (hi >= lo) cnt = (unsigned long long)(hi - lo + 1);
  }
  if (evals) {
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(evals, cnt);
  }
}

// The line sum with adaptive windows: a block per (256-point tile, T node).  The lines
// whose cutoff windows touch the tile are a contiguous index range; the block takes it
// in chunks of 256 lines, keeps (ballot compaction, in ascending nu0) those whose
// adaptive window at this node meets the tile, and each point then sums the kept
// lines whose window holds it (Kahan, ascending nu0).  A kept line can be far from
// the point (strong lines keep the whole cutoff window), so values take the full-range
// form: the Lorentz reciprocal, or the Faddeeva function in all its regions.
template <int PROFILE>
__global__ void __launch_bounds__(kTilePts)
k_kappa_adaptive(const float4 *__restrict__ P, const int4 *__restrict__ R, const int2 *__restrict__ AW,
                 long long n_lines, long long n_nu, WeidCoef wc, int accumulate, float *__restrict__ kappa) {
  __shared__ long long s_range[2];
  __shared__ int2 s_win[kTilePts];     // kept lines' windows at this node
  __shared__ float4 s_par[kTilePts];   // their {centre index bits, centre offset, coefficient, g^2 or y}
  __shared__ float s_sd[kTilePts];     // Voigt: s dnu (grid units to x)
  __shared__ int s_warp[kTilePts / 32];
  const long long jw0 = (long long)blockIdx.x * kTilePts;
  const long long jend = min(jw0 + (long long)kTilePts, n_nu);
  const int k = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_range[0] = lower_bound_hi(R, n_lines, (int)jw0);
  if (threadIdx.x == 1) s_range[1] = lower_bound_lo(R, n_lines, (int)jend);
  __syncthreads();
  const long long a = s_range[0], b = max(s_range[0], s_range[1]);
  const long long j = jw0 + threadIdx.x;
  const float4 *Pk = P + (long long)k * n_lines;
  const int2 *Wk = AW + (long long)k * n_lines;
  float acc = 0.0f, cmp = 0.0f;
#pragma unroll 1
  for (long long c0 = a; c0 < b; c0 += kTilePts) {
    const long long l = c0 + threadIdx.x;
    int2 w = make_int2(1, 0);
    bool keep = false;
    if (l < b) {
      w = __ldg(Wk + l);
      keep = w.y >= w.x && w.y >= (int)jw0 && (long long)w.x < jend;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int off = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kTilePts / 32; ++q) {
      const int c = s_warp[q];
      off += q < warp ? c : 0;
      total += c;
    }
    if (keep) {  // the kept line's constants, formed once for all the tile's points
      const int pos = off + __popc(m & ((1u << lane) - 1u));
      const int4 r = __ldg(R + l);
      const float4 p = __ldg(Pk + l);
      s_win[pos] = w;
      if (PROFILE == RT_PROFILE_LORENTZ) {
        s_par[pos] = make_float4(__int_as_float(r.z), __int_as_float(r.w), p.x, p.y);
      } else {
        const float y = sqrtf(p.z);
        s_par[pos] = make_float4(__int_as_float(r.z), __int_as_float(r.w), __fdividef(p.x, y), y);
        s_sd[pos] = p.y;
      }
    }
    __syncthreads();
    if (j < jend) {
#pragma unroll 1
      for (int i = 0; i < total; ++i) {
        const int2 ww = s_win[i];
        if ((int)j < ww.x || (int)j > ww.y) continue;
        const float4 q = s_par[i];
        const float u = __fadd_rn((float)((int)j - __float_as_int(q.x)), q.y);
        float v;
        if (PROFILE == RT_PROFILE_LORENTZ) {
          v = q.z * rcp_approx(__fmaf_rn(u, u, q.w));
        } else {
          v = q.z * faddeeva_re(s_sd[i] * u, q.w, wc);
        }
        const float yk = __fsub_rn(v, cmp);
        const float t = __fadd_rn(acc, yk);
        cmp = __fsub_rn(__fsub_rn(t, acc), yk);
        acc = t;
      }
    }
    __syncthreads();  // the kept list is rewritten by the next chunk
  }
  if (j < jend) {
    float *dst = kappa + (long long)k * n_nu + j;
    const float out = __fsub_rn(acc, cmp);
    *dst = accumulate ? *dst + out : out;
  }
}

int g_kappa_tpb = kMaxTPerBlock;

rt_status launch_kappa(const float4 *P, const float4 *P2, const int4 *R, int4 *tiles,
                       const unsigned *far_bits, const int2 *AW, long long n, const rt_spectral *spec,
                       double nu_abs_max, double mass_amu, float *kappa, uint32_t *status,
                       cudaStream_t st) {
  static WeidCoef wc;
  static std::once_flag wc_once;
  std::call_once(wc_once, [] { weideman_coefficients(&wc); });
  const long long n_tiles_a = (spec->n_nu + kTilePts - 1) / kTilePts;
  if (AW) {  // adaptive points per line: the windows' gather kernel
    dim3 g((unsigned)n_tiles_a, (unsigned)spec->nT);
    if (spec->profile == RT_PROFILE_LORENTZ)
      k_kappa_adaptive<RT_PROFILE_LORENTZ><<<g, kTilePts, 0, st>>>(P, R, AW, n, spec->n_nu, wc,
                                                                   spec->accumulate ? 1 : 0, kappa);
    else
      k_kappa_adaptive<RT_PROFILE_VOIGT><<<g, kTilePts, 0, st>>>(P, R, AW, n, spec->n_nu, wc,
                                                                 spec->accumulate ? 1 : 0, kappa);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
  }
  // W bounds every line's near-centre half-width sqrt(400 - y^2) / (s dnu) <= 20 alpha /
  // (sqrt(ln 2) dnu), alpha the largest Doppler half-width of a line that reaches the grid
  int W = 0;
  if (spec->profile == RT_PROFILE_VOIGT) {
    const double alpha = nu_abs_max * std::sqrt(spec->T_max) *
                         std::sqrt(2.0 * std::log(2.0) * kKB / (mass_amu * kAmu)) / kC;
    const double w = 20.0 * alpha / (std::sqrt(std::log(2.0)) * spec->dnu) * 1.01 + 2.0;
    W = (!(w < (double)(1 << 28))) ? (1 << 28) : (int)std::ceil(w);
  }
  const long long n_tiles = (spec->n_nu + kTilePts - 1) / kTilePts;
  if (spec->points_per_line > 0) {  // fixed points per line: the gather kernel
    dim3 g((unsigned)n_tiles, (unsigned)((spec->nT + kPplNodes - 1) / kPplNodes));
    if (spec->profile == RT_PROFILE_LORENTZ)
      k_kappa_ppl<RT_PROFILE_LORENTZ><<<g, kTilePts, 0, st>>>(P, R, n, spec->n_nu, spec->nT, wc,
                                                              spec->accumulate ? 1 : 0, kappa);
    else
      k_kappa_ppl<RT_PROFILE_VOIGT><<<g, kTilePts, 0, st>>>(P, R, n, spec->n_nu, spec->nT, wc,
                                                            spec->accumulate ? 1 : 0, kappa);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
  }
  k_tile_lines<<<(unsigned)((n_tiles + 3) / 4), 128, 0, st>>>(R, n, spec->n_nu, W, far_bits, n_tiles,
                                                                tiles);  // a warp per tile
  RT_CUDA_TRY(cudaGetLastError());
  const int vec_ok = ((reinterpret_cast<uintptr_t>(kappa) & 15u) == 0 && spec->n_nu % 4 == 0) ? 1 : 0;
  int want = g_kappa_tpb;
  if (want < 1 || want > kMaxTPerBlock) want = kMaxTPerBlock;
  const int tpb = spec->nT < want ? spec->nT : want;
  dim3 gk((unsigned)n_tiles, (unsigned)((spec->nT + tpb - 1) / tpb));
  auto kernel = spec->profile == RT_PROFILE_LORENTZ ? k_kappa<RT_PROFILE_LORENTZ> : k_kappa<RT_PROFILE_VOIGT>;
  kernel<<<gk, 32 * tpb, 0, st>>>(P, P2, R, tiles, n, spec->n_nu, spec->nT, wc, vec_ok,
                                  spec->accumulate ? 1 : 0, kappa, status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

}  // namespace

rt_status validate_spec(const rt_spectral *s) {
  if (!s) return fail(RT_E_INVAL, "spec is NULL");
  if (!(s->n_nu >= 1) || s->n_nu > (1LL << 30))
    return fail(RT_E_INVAL, "spec.n_nu must be in [1, 2^30]");
  if (!std::isfinite(s->nu_min) || !std::isfinite(s->dnu) || !(s->dnu > 0))
    return fail(RT_E_INVAL, "spec.nu_min / dnu must be finite, dnu > 0");
  if (!std::isfinite(s->cutoff) || s->cutoff < 0 || s->cutoff / s->dnu > (double)(1 << 28))
    return fail(RT_E_INVAL, "spec.cutoff must be finite, >= 0 and < 2^28 dnu");
  if (s->profile != RT_PROFILE_LORENTZ && s->profile != RT_PROFILE_VOIGT)
    return fail(RT_E_INVAL, "spec.profile must be RT_PROFILE_LORENTZ or RT_PROFILE_VOIGT");
  if (s->nT < 1 || s->nT > 65535) return fail(RT_E_INVAL, "spec.nT must be in [1, 65535]");
  if (!std::isfinite(s->T_min) || !std::isfinite(s->T_max) || !(s->T_min > 0) ||
      s->T_max < s->T_min || (s->nT > 1 && !(s->T_max > s->T_min)))
    return fail(RT_E_INVAL, "spec temperatures must satisfy 0 < T_min <= T_max (< when nT > 1)");
  if (!std::isfinite(s->p_ref_atm) || !(s->p_ref_atm > 0) || !std::isfinite(s->x_ref) ||
      !(s->x_ref > 0))
    return fail(RT_E_INVAL, "spec.p_ref_atm and spec.x_ref must be finite and > 0");
  if (s->points_per_line < 0 || s->points_per_line > (1 << 20))
    return fail(RT_E_INVAL, "spec.points_per_line must be in [0, 2^20]");
  if (s->accumulate != 0 && s->accumulate != 1) return fail(RT_E_INVAL, "spec.accumulate must be 0 or 1");
  if (!std::isfinite(s->kappa_min) || s->kappa_min < 0)
    return fail(RT_E_INVAL, "spec.kappa_min must be finite and >= 0");
  if (s->kappa_min > 0 && s->points_per_line > 0)
    return fail(RT_E_INVAL, "spec.kappa_min (adaptive points) and points_per_line exclude each other");
  return RT_OK;
}

namespace {

rt_status validate_host_lines(const rt_lines *L, const rt_spectral *s) {
  const double lim = 536870912.0 * s->dnu;  // 2^29 grid steps
  for (int64_t l = 0; l < L->n; ++l) {
    const double v = L->nu0[l], S = L->S_ref[l], g = L->gamma_ref[l], E = L->E_lower[l];
    if (!std::isfinite(v) || !std::isfinite(S) || !(S > 0) || !std::isfinite(g) || !(g > 0) ||
        !std::isfinite(E) || !(E >= 0))
      return fail(RT_E_NONFINITE, "line %lld: non-finite or non-positive parameter", (long long)l);
    if (!(std::fabs(v - s->nu_min) <= lim))
      return fail(RT_E_INVAL, "line %lld: centre too far from the spectral grid", (long long)l);
    if (l > 0 && !(L->nu0[l - 1] <= v))
      return fail(RT_E_UNSORTED, "line %lld: centres not in ascending order", (long long)l);
  }
  return RT_OK;
}

}  // namespace

rt_status launch_line_geometry(const double *nu0, const double *S, const double *g, const double *E,
                               long long n, const rt_spectral *spec, int check, int4 *R,
                               unsigned long long *evals, uint32_t *status, cudaStream_t st) {
  if (n <= 0) return RT_OK;
  GeomParams G{spec->nu_min, spec->dnu, spec->cutoff, spec->n_nu, n, spec->nT, check,
               spec->points_per_line};
  k_line_geometry<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nu0, S, g, E, G, R, evals, status);
  RT_CUDA_TRY(cudaGetLastError());
  return RT_OK;
}

namespace {

// Scratch of one build: [line arrays if host-resident][R: n int4][P: nT n float4]
// [P2: nT n float4, Voigt][tile segments: 3 int4 per 256-point tile][far-zone bound]
struct KappaLayout {
  size_t off_R, off_P, off_P2, off_tiles, off_far, off_AW, total;
};

KappaLayout kappa_layout(const rt_lines *lines, const rt_spectral *spec) {
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t n = (size_t)lines->n;
  const size_t pn = (size_t)spec->nT * n * sizeof(float4);
  KappaLayout L;
  L.off_R = up(lines->memory == RT_MEM_HOST ? 4 * n * sizeof(double) : 0);
  L.off_P = up(L.off_R + n * sizeof(int4));
  L.off_P2 = up(L.off_P + pn);
  L.off_tiles = up(L.off_P2 + (spec->profile == RT_PROFILE_VOIGT ? pn : 0));
  const size_t n_tiles = (size_t)((spec->n_nu + kTilePts - 1) / kTilePts);
  L.off_far = up(L.off_tiles + n_tiles * kTileInts * sizeof(int4));
  L.off_AW = L.off_far + 256;  // adaptive windows: nT n int2
  L.total = L.off_AW + (spec->kappa_min > 0 ? up((size_t)spec->nT * n * sizeof(int2)) : 0);
  return L;
}

rt_status validate_build_args(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                              uint32_t *status, const char *who) {
  rt_status v = validate_spec(spec);
  if (v != RT_OK) return v;
  if (!lines || !kappa) return fail(RT_E_INVAL, "%s: lines or kappa is NULL", who);
  if (lines->n < 0 || lines->n > (1LL << 31) - 1) return fail(RT_E_INVAL, "lines.n out of range");
  if (lines->memory != RT_MEM_HOST && lines->memory != RT_MEM_DEVICE)
    return fail(RT_E_INVAL, "lines.memory must be RT_MEM_HOST or RT_MEM_DEVICE");
  if (!std::isfinite(lines->T_ref) || !(lines->T_ref > 0) || !std::isfinite(lines->n_T) ||
      !std::isfinite(lines->q_exp) || !std::isfinite(lines->mass_amu) || !(lines->mass_amu > 0))
    return fail(RT_E_INVAL, "lines: T_ref, n_T, q_exp, mass_amu must be finite (T_ref, mass > 0)");
  if (lines->n > 0 && (!lines->nu0 || !lines->S_ref || !lines->gamma_ref || !lines->E_lower))
    return fail(RT_E_INVAL, "lines: NULL array");
  if (lines->memory == RT_MEM_DEVICE && !status)
    return fail(RT_E_INVAL, "device-resident lines need a device status word");
  return RT_OK;
}

// Everything after validation, on scratch laid out by kappa_layout.
rt_status run_build(char *base, const KappaLayout &L, const rt_lines *lines, const rt_spectral *spec,
                    float *kappa, unsigned long long *evals_out, uint32_t *status, cudaStream_t st) {
  const long long n = lines->n;
  const double *d_nu0 = lines->nu0, *d_S = lines->S_ref, *d_g = lines->gamma_ref, *d_E = lines->E_lower;
  if (lines->memory == RT_MEM_HOST) {
    double *d = reinterpret_cast<double *>(base);
    RT_CUDA_TRY(cudaMemcpyAsync(d, lines->nu0, n * sizeof(double), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + n, lines->S_ref, n * sizeof(double), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + 2 * n, lines->gamma_ref, n * sizeof(double), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(d + 3 * n, lines->E_lower, n * sizeof(double), cudaMemcpyHostToDevice, st));
    d_nu0 = d; d_S = d + n; d_g = d + 2 * n; d_E = d + 3 * n;
  }
  int4 *R = reinterpret_cast<int4 *>(base + L.off_R);
  float4 *P = reinterpret_cast<float4 *>(base + L.off_P);
  float4 *P2 = reinterpret_cast<float4 *>(base + L.off_P2);
  int4 *tiles = reinterpret_cast<int4 *>(base + L.off_tiles);
  unsigned *far_bits = reinterpret_cast<unsigned *>(base + L.off_far);

  GeomParams G{spec->nu_min, spec->dnu, spec->cutoff, spec->n_nu, n, spec->nT,
               lines->memory == RT_MEM_DEVICE ? 1 : 0, spec->points_per_line};
  const int tb = 256;
  const bool adaptive = spec->kappa_min > 0;
  // with adaptive points the evaluations are counted per (node, line) window below
  k_line_geometry<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(d_nu0, d_S, d_g, d_E, G, R,
                                                                adaptive ? nullptr : evals_out, status);
  RT_CUDA_TRY(cudaGetLastError());
  int2 *AW = nullptr;
  if (adaptive) {
    AW = reinterpret_cast<int2 *>(base + L.off_AW);
    AdaptParams A{spec->nu_min, spec->dnu, spec->cutoff, spec->T_min, spec->T_max, lines->T_ref,
                  100.0 * (kH * kC / kKB), spec->x_ref, spec->p_ref_atm, lines->n_T, lines->q_exp,
                  spec->kappa_min, spec->n_nu, n, spec->nT};
    dim3 ga((unsigned)((n + tb - 1) / tb), (unsigned)spec->nT);
    k_adaptive_windows<<<ga, tb, 0, st>>>(d_nu0, d_S, d_g, d_E, A, AW, evals_out);
    RT_CUDA_TRY(cudaGetLastError());
  }

  PrefParams Q;
  Q.T_min = spec->T_min;
  Q.T_max = spec->T_max;
  Q.T_ref = lines->T_ref;
  const double c2 = 100.0 * kH * kC / kKB;
  Q.c2.hi = (float)c2;
  Q.c2.lo = (float)(c2 - (double)Q.c2.hi);
  Q.u_coef = (float)(spec->x_ref * spec->p_ref_atm * kAtm / kKB * 1e-6);
  Q.p_ref = (float)spec->p_ref_atm;
  Q.n_T = (float)lines->n_T;
  Q.q_exp = (float)lines->q_exp;
  Q.doppler = (float)(std::sqrt(2.0 * std::log(2.0) * kKB / (lines->mass_amu * kAmu)) / kC);
  Q.inv_dnu = (float)(1.0 / spec->dnu);
  Q.dnu = (float)spec->dnu;
  Q.n_lines = n;
  Q.nT = spec->nT;
  Q.profile = spec->profile;
  dim3 gp((unsigned)((n + tb - 1) / tb), (unsigned)spec->nT);
  RT_CUDA_TRY(cudaMemsetAsync(far_bits, 0, 2 * sizeof(unsigned), st));
  k_prefactor<<<gp, tb, 0, st>>>(d_nu0, d_S, d_g, d_E, Q, P, P2, far_bits);
  RT_CUDA_TRY(cudaGetLastError());

  // largest |nu0| of a line whose window (cutoff or fixed points) reaches the grid
  const double reach = spec->cutoff + (spec->points_per_line + 2.0) * spec->dnu;
  const double nu_abs_max =
      std::fmax(std::fabs(spec->nu_min - reach),
                std::fabs(spec->nu_min + (double)spec->n_nu * spec->dnu + reach));
  return launch_kappa(P, P2, R, tiles, far_bits, AW, n, spec, nu_abs_max, lines->mass_amu, kappa, status, st);
}

}  // namespace

rt_status build_kappa_impl(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                           unsigned long long *evals_out, uint32_t *status, cudaStream_t st) {
  rt_status v = validate_build_args(lines, spec, kappa, status, "rt_build_kappa");
  if (v != RT_OK) return v;
  if (lines->memory == RT_MEM_HOST && lines->n > 0) {
    v = validate_host_lines(lines, spec);
    if (v != RT_OK) return v;
  }
  const size_t table = (size_t)spec->nT * (size_t)spec->n_nu;
  if (lines->n == 0) {
    if (!spec->accumulate) RT_CUDA_TRY(cudaMemsetAsync(kappa, 0, table * sizeof(float), st));
    return RT_OK;
  }
  const KappaLayout L = kappa_layout(lines, spec);
  Scratch scr;
  v = scr.alloc(L.total, st);
  if (v != RT_OK) return v;
  return run_build(scr.as<char>(), L, lines, spec, kappa, evals_out, status, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch is this file-scope device array: every
// GPU that loads the library holds it until the process exits.  Host code must
// not hand the array's name to a kernel (in host code it is a host-side stand-in
// for the symbol); the device address is looked up once per device below.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static rt_status static_scratch_address(void **out) {
  static std::mutex mu;
  static void *addr[256] = {};
  int dev = 0;
  RT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(RT_E_INVAL, "rt_build_kappa_static: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
    addr[dev] = p;
  }
  *out = addr[dev];
  return RT_OK;
}

rt_status build_kappa_static_impl(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                                  unsigned long long *evals_out, uint32_t *status, cudaStream_t st) {
  rt_status v = validate_build_args(lines, spec, kappa, status, "rt_build_kappa_static");
  if (v != RT_OK) return v;
  // same scratch layout as rt_build_kappa, checked against the fixed array
  const KappaLayout L = kappa_layout(lines, spec);
  if (L.total > kStaticScratchBytes)
    return fail(RT_E_INVAL,
                "rt_build_kappa_static: needs %zu bytes of scratch (16 B per line and T node, 32 B "
                "for Voigt lines, 16 B per line, 80 B per 256 wavenumbers, plus 32 B per line for "
                "host-resident lines), the static array holds %zu",
                L.total, kStaticScratchBytes);
  if (lines->memory == RT_MEM_HOST && lines->n > 0) {
    v = validate_host_lines(lines, spec);
    if (v != RT_OK) return v;
  }
  const size_t table = (size_t)spec->nT * (size_t)spec->n_nu;
  if (lines->n == 0) {
    if (!spec->accumulate) RT_CUDA_TRY(cudaMemsetAsync(kappa, 0, table * sizeof(float), st));
    return RT_OK;
  }
  void *scratch = nullptr;
  v = static_scratch_address(&scratch);
  if (v != RT_OK) return v;
  return run_build(reinterpret_cast<char *>(scratch), L, lines, spec, kappa, evals_out, status, st);
}

}  // namespace rt

extern "C" rt_status rt_build_kappa(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                                    unsigned long long *evals_out, uint32_t *status, void *stream) {
  return rt::build_kappa_impl(lines, spec, kappa, evals_out, status, (cudaStream_t)stream);
}

extern "C" rt_status rt_build_kappa_static(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                                           unsigned long long *evals_out, uint32_t *status,
                                           void *stream) {
  return rt::build_kappa_static_impl(lines, spec, kappa, evals_out, status, (cudaStream_t)stream);
}

namespace rt {
extern int g_walk_blocks, g_walk_refill, g_walk_group;  // rt_trace.cu
}

extern "C" rt_status rt_set_tuning(const rt_tuning *t) {
  if (!t) return rt::fail(RT_E_INVAL, "rt_set_tuning: NULL");
  if (t->kappa_t_per_block < 0 || t->kappa_t_per_block > 8)
    return rt::fail(RT_E_INVAL, "rt_set_tuning: kappa_t_per_block must be in [0, 8]");
  if (t->walk_blocks_per_sm != 0 && t->walk_blocks_per_sm != 4 && t->walk_blocks_per_sm != 5)
    return rt::fail(RT_E_INVAL, "rt_set_tuning: walk_blocks_per_sm must be 0, 4 or 5");
  if (t->walk_refill_idle != 0 && t->walk_refill_idle != 12 && t->walk_refill_idle != 16)
    return rt::fail(RT_E_INVAL, "rt_set_tuning: walk_refill_idle must be 0, 12 or 16");
  if (t->walk_group < 0 || t->walk_group > 2) return rt::fail(RT_E_INVAL, "rt_set_tuning: walk_group must be 0, 1 or 2");
  rt::g_kappa_tpb = t->kappa_t_per_block == 0 ? 8 : t->kappa_t_per_block;
  rt::g_walk_blocks = t->walk_blocks_per_sm == 0 ? 5 : t->walk_blocks_per_sm;
  rt::g_walk_refill = t->walk_refill_idle == 0 ? 16 : t->walk_refill_idle;
  rt::g_walk_group = t->walk_group;
  return RT_OK;
}

extern "C" rt_status rt_get_tuning(rt_tuning *t) {
  if (!t) return rt::fail(RT_E_INVAL, "rt_get_tuning: NULL");
  *t = rt_tuning{};
  t->kappa_t_per_block = rt::g_kappa_tpb;
  t->walk_blocks_per_sm = rt::g_walk_blocks;
  t->walk_refill_idle = rt::g_walk_refill;
  t->walk_group = rt::g_walk_group;
  return RT_OK;
}
