/*
 * rt.h -- C ABI of the GB300 Monte-Carlo line-by-line radiative-transfer library.
 *
 * The library computes the hot path of the method of Collange, Daumas and Defour,
 * "Graphic processors to speed-up simulations for the design of high performance
 * solar receptors" (Section 3): the absorption coefficient kappa(nu, T) of a gas
 * from a spectral line list (Eqs. S and tau), and Monte-Carlo rays traced cell by
 * cell through a grid of isothermal homogeneous finite volumes with Beer-Lambert
 * attenuation (Eq. I, first term), emitted according to the Planck function
 * (Eq. planck), with the absorbed power tallied per cell (the parallel reduction
 * of Section 3).
 *
 * Conventions shared by every entry point:
 *  - Memory: the caller owns every buffer.  "host" pointers are ordinary CPU
 *    memory, "device" pointers are CUDA device memory of the current device.
 *    The library allocates only temporary scratch, stream-ordered on the given
 *    stream (cudaMallocAsync / cudaFreeAsync), and releases it before the
 *    call's work completes.
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *    Calls are asynchronous on that stream unless stated otherwise.
 *  - Errors: every call returns an rt_status and never aborts the process.
 *    Arguments are validated on the host before any launch.  Conditions only the
 *    device can see (a non-finite temperature in a device field, a ray over its
 *    step cap, a bounded wait that ran out) are OR-ed into a caller-provided
 *    device status word; rt_tally() and rt_status_read() report them.
 *    rt_last_error() returns a thread-local message for the last failure.
 *  - Units: wavenumbers in cm^-1, lengths in m, temperatures in K, pressures in
 *    atm, absorption coefficients in cm^-1, powers in W.
 *  - Arithmetic: the line sum and the ray walk run in binary32 with compensated
 *    (Kahan) sums; binary64 is used on the device for the per-cell tally, the
 *    energy balance, and the exact conversion of the caller's binary64 line
 *    positions into grid coordinates.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_E_INVAL = 1,      /* bad argument: NULL pointer, size or range */
  RT_E_NOMEM = 2,      /* scratch allocation failed */
  RT_E_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  RT_E_STEPCAP = 4,    /* a ray exceeded nx+ny+nz+4 cell visits (device-reported) */
  RT_E_TIMEOUT = 5,    /* a bounded device wait ran out (device-reported) */
  RT_E_UNSORTED = 6,   /* line list not sorted by ascending centre */
  RT_E_NONFINITE = 7   /* NaN / Inf / non-positive value where a positive finite one is needed */
} rt_status;

/* Device status word bits (OR-ed by kernels into rt_tally_buf.status etc.). */
#define RT_DEV_STEPCAP   (1u << 0)
#define RT_DEV_TIMEOUT   (1u << 1)
#define RT_DEV_NONFINITE (1u << 2)
#define RT_DEV_UNSORTED  (1u << 3)
#define RT_DEV_COLUMN    (1u << 4)

enum { RT_PROFILE_LORENTZ = 0, RT_PROFILE_VOIGT = 1 };
enum { RT_MEM_HOST = 0, RT_MEM_DEVICE = 1 };

/* rt_trace flags */
#define RT_SRC_EMIT   0        /* thermal emission sampled over cells and wavenumbers */
#define RT_SRC_BEAM   1        /* collimated unit beams: ray r enters face x=0 at nu_(r mod n_nu) */
#define RT_TAU_CUT    (1 << 4) /* stop a ray once its optical depth exceeds 100 (lost < 4e-44) */
#define RT_COUNT_EVALS (1 << 5) /* rt_trace_mlp, rt_trace_mlp_bands only: tally->steps holds two
                                   counters and steps[1] also accumulates the number of network
                                   evaluations (one per 128-ray tile and walk step) */

/*
 * Spectral line list (Section 3, Eq. S: S(T_ref), nu, E_eta; Eq. tau: lines of one
 * absorbing gas).  Arrays hold n binary64 values, sorted by ascending nu0, in host
 * memory (memory = RT_MEM_HOST; validated on the host: RT_E_UNSORTED,
 * RT_E_NONFINITE) or device memory (memory = RT_MEM_DEVICE; validated on the
 * device into the status word given to rt_build_kappa).
 */
typedef struct {
  int64_t n;               /* number of lines, >= 0 */
  const double *nu0;       /* line centre, cm^-1, ascending */
  const double *S_ref;     /* intensity at T_ref, cm/molecule, > 0 */
  const double *gamma_ref; /* Lorentz half-width at T_ref and 1 atm, cm^-1, > 0 */
  const double *E_lower;   /* lower-state energy, cm^-1, >= 0 */
  double T_ref;            /* reference temperature, K (296 for HITRAN-style lists) */
  double n_T;              /* gamma(T) = gamma_ref (p / 1 atm) (T_ref / T)^n_T */
  double q_exp;            /* partition function Q(T) ~ T^q_exp */
  double mass_amu;         /* molecular mass, u (Doppler width) */
  int32_t memory;          /* RT_MEM_HOST or RT_MEM_DEVICE */
  int32_t pad;
} rt_lines;

/*
 * Spectral window and temperature grid of the kappa table (Section 3, Eq. tau).
 * Spectral samples nu_j = nu_min + j * dnu, j = 0 .. n_nu-1 (binary64).
 * Temperature nodes T_k = T_min + k (T_max - T_min) / (nT - 1), k = 0 .. nT-1;
 * nT = 1 is a single isothermal row at T_min.  Lines contribute at nu_j when
 * |nu_j - nu0| <= cutoff (binary64, inclusive), with no renormalisation.
 */
typedef struct {
  double nu_min;           /* cm^-1 */
  double dnu;              /* cm^-1, > 0 */
  int64_t n_nu;            /* number of spectral samples, >= 1 */
  double cutoff;           /* line-wing cutoff, cm^-1, >= 0 */
  int32_t profile;         /* RT_PROFILE_LORENTZ or RT_PROFILE_VOIGT */
  int32_t nT;              /* number of temperature nodes, >= 1 */
  double T_min, T_max;     /* K, 0 < T_min <= T_max (T_min < T_max when nT > 1) */
  double p_ref_atm;        /* pressure of the table, atm, > 0 */
  double x_ref;            /* absorber mole fraction of the table, > 0 */
  int32_t points_per_line; /* > 0: each line contributes at this many grid points around
                              its centre, j = jf - n/2 + 1 .. jf + n/2 with jf = floor((nu0 -
                              nu_min)/dnu) (Section 3: 16 contributions per line), instead of
                              the cutoff window; 0: cutoff window */
  int32_t accumulate;      /* rt_build_kappa: 1 adds into kappa (one call per absorbing gas of
                              a mixture, Eq. tau's sum over g), 0 overwrites it */
  double kappa_min;        /* > 0: adaptive points per line (the next version of Section 4:
                              points from the local temperature and the line's intensity):
                              at T node T_k line l contributes only where |nu_j - nu0| <= w =
                              min(cutoff, sqrt(A gamma / (pi kappa_min))), A = u(T_k) S(T_k),
                              gamma its Lorentz half-width at T_k (the distance at which its
                              Lorentz wing A gamma / (pi dnu^2) falls to kappa_min, cm^-1),
                              decided in binary64; requires points_per_line = 0; 0: off */
} rt_spectral;

/*
 * Finite-volume grid (Section 3, Fig. ray: isothermal homogeneous finite volumes
 * with temperature, pressure and absorber density).  Cell (ix, iy, iz) has flat
 * index ix + nx (iy + ny iz) and spans [ix hx, (ix+1) hx) etc.  An infinite cell
 * size makes that axis unbounded (hy = hz = INFINITY gives a plane-parallel slab;
 * the cell volume then counts 1 m per unbounded axis).  Fields are binary32
 * device arrays of nx*ny*nz values.  p_atm and x may be NULL (the table's
 * p_ref and x_ref); otherwise kappa of a cell is scaled by (p x)/(p_ref x_ref).
 */
typedef struct {
  int32_t nx, ny, nz, pad;
  double hx, hy, hz;       /* m, > 0 (or +INFINITY) */
  const float *T;          /* device [ncells], K, finite > 0 */
  const float *p_atm;      /* device [ncells] or NULL */
  const float *x;          /* device [ncells] or NULL */
} rt_grid;

/*
 * Tally buffers (device, caller-owned).  rt_trace ADDS into them, so several
 * calls (ray ranges, enclosures) can accumulate; zero them with rt_tally_zero().
 *   absorbed[ncells]  absorbed power per cell, W (binary64)
 *   scalars[4]        [0] emitted power, [1] total absorbed (set by rt_tally),
 *                     [2] power absorbed by the cold black walls, [3] relative
 *                     energy residual |emitted - absorbed - walls| / emitted
 *                     (set by rt_tally)
 *   steps[1]          number of ray-cell steps processed (steps[2] with RT_COUNT_EVALS:
 *                     [1] the surrogate walk's network evaluations)
 *   status[1]         sticky RT_DEV_* bits
 */
typedef struct {
  double *absorbed;
  double *scalars;
  unsigned long long *steps;
  uint32_t *status;
} rt_tally_buf;

/*
 * Optional per-ray record (device buffers) of rays [ray_begin, ray_begin + n_rays)
 * of a trace call: the visited cells and segment lengths (m) in walk order, the
 * number of visits, the emitted power and the power that reached a wall.
 */
typedef struct {
  int64_t n_rays;
  int32_t max_visits;      /* row length of cells/ds, >= nx+ny+nz+4 for complete rows */
  int32_t pad;
  int32_t *cells;          /* [n_rays * max_visits] */
  float *ds;               /* [n_rays * max_visits] */
  int32_t *n_visits;       /* [n_rays] */
  float *weight;           /* [n_rays] */
  float *escaped;          /* [n_rays] */
} rt_record;

/* Library version string. */
const char *rt_version(void);

/* Thread-local message describing the last non-RT_OK status of this thread. */
const char *rt_last_error(void);

/* Number of binary32 elements of the kappa table: nT * n_nu (0 on bad input). */
size_t rt_kappa_table_elems(const rt_spectral *spec);

/*
 * rt_build_kappa -- Eqs. (S) and (tau) of Section 3 on a temperature grid:
 *   kappa[k * n_nu + j] = u(T_k) * sum_{l : |nu_j - nu0_l| <= cutoff} S_l(T_k) f_l(nu_j - nu0_l; T_k)
 * with u = x_ref p_ref / (k_B T) the absorber number density [cm^-3], S_l(T) by
 * Eq. (S) with Q(T_ref)/Q(T) = (T_ref/T)^q_exp, and f the Lorentz profile (half-width
 * gamma = gamma_ref p_ref (T_ref/T)^n_T) or the Voigt profile (that Lorentz width and
 * the Doppler half-width nu0/c sqrt(2 ln2 k_B T / m)).  Binary32 with a Kahan sum
 * over lines in ascending nu0.
 *   kappa      device [nT * n_nu] binary32, cm^-1, written (T-major: row k is the
 *              spectrum at T_k).
 *   evals_out  optional device counter: adds the number of (T_k, line, nu_j)
 *              profile evaluations.
 *   status     device status word; required when lines->memory == RT_MEM_DEVICE
 *              (receives RT_DEV_UNSORTED / RT_DEV_NONFINITE), may be NULL otherwise.
 * Returns RT_E_INVAL / RT_E_UNSORTED / RT_E_NONFINITE before any launch on bad
 * host-visible input, RT_E_NOMEM / RT_E_CUDA on runtime failures.
 */
rt_status rt_build_kappa(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                         unsigned long long *evals_out, uint32_t *status, void *stream);

/*
 * rt_build_kappa_static -- rt_build_kappa for callers that cannot allocate device
 * memory.  The paper has no counterpart: this entry point exists for programs
 * that must not call the CUDA allocator once they run, for example a flow solver
 * that has handed all device memory to its own fixed pool, or a loop with a
 * latency budget in which an allocation could stall or fail.  Arguments, result
 * and errors are those of rt_build_kappa; the caller still provides the lines,
 * the table and the optional counters.
 * Scratch: a 32 MiB array in the library's device memory (a file-scope
 *   __device__ array that every GPU loading the library holds until the process
 *   exits); the call allocates and frees nothing.
 * Limit: 16 B per (T node, line) for Lorentz lines, 32 B for Voigt lines, + 16 B
 *   per line + 80 B per 256 wavenumbers, plus 32 B per line when the lines are
 *   host-resident, at most 32 MiB in all (about 2 million Lorentz or 1 million
 *   Voigt (T node, line) pairs, e.g. 64 T nodes x 15,000 Voigt lines).  Larger
 *   inputs return RT_E_INVAL with the required size before any work is queued.
 * Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture.  The address is kept for the life of the process, so a
 *   device reset (cudaDeviceReset) between calls is not supported.
 * Sharing: all calls use the same array and it keeps the last call's contents;
 *   every call writes the scratch it reads before reading it.  Calls whose work
 *   can overlap on the GPU (other streams, other host threads) race on the array:
 *   serialise them.
 */
rt_status rt_build_kappa_static(const rt_lines *lines, const rt_spectral *spec, float *kappa,
                                unsigned long long *evals_out, uint32_t *status, void *stream);

/*
 * rt_trace -- the Monte-Carlo ray-tracing estimator of Section 3 (Fig. ray).
 * Rays r in [ray_begin, ray_begin + n_rays) of an estimate over n_rays_total rays:
 *   RT_SRC_EMIT: Philox4x32-10 (key = seed, counter = (r_lo, r_hi, call, enclosure))
 *     draws the emission cell c and wavenumber index j uniformly, a uniform point in
 *     the cell and an isotropic direction (Marsaglia 1972).  The ray carries
 *       w = 4 pi V kappa_c(nu_j) I_b(nu_j, T_c) dnu * ncells n_nu / n_rays_total
 *     with I_b the Planck function of Eq. (planck) in wavenumber form.
 *   RT_SRC_BEAM: ray r enters the x = 0 face at the centre of cell (0, ny/2, nz/2)
 *     along +x with w = 1 at nu_(r mod n_nu).
 * The ray is walked cell by cell (Amanatides-Woo traversal, specified in binary32
 * round-to-nearest without contraction); in a cell crossed over length ds it leaves
 *   w exp(-tau) (1 - exp(-kappa_cell 100 ds))     (Eq. I, first term)
 * where tau is its (Kahan-summed) optical depth so far and kappa_cell is the table
 * interpolated linearly in T between the cell's bracketing nodes (clamped to the
 * table range) times the density scale.  What reaches a wall is absorbed there.
 *   kappa      device [nT * n_nu] table from rt_build_kappa for the same spec.
 *   tally      accumulated (see rt_tally_buf).
 *   record     optional (NULL = none).
 *   flags      RT_SRC_EMIT or RT_SRC_BEAM, optionally | RT_TAU_CUT.
 */
rt_status rt_trace(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                   uint64_t ray_begin, uint64_t n_rays, uint64_t n_rays_total,
                   uint64_t seed, uint32_t enclosure, int32_t flags,
                   const rt_tally_buf *tally, const rt_record *record, void *stream);

/*
 * Batched tracing of many independent enclosures (Section 3's walk on each), in
 * one persistent launch.  Enclosure e (0-based) is traced exactly as
 * rt_trace(grid_e, kappa, spec, 0, n_rays_e, n_rays_e, seed, e, flags, tally_e)
 * would trace it (Philox counter word 3 = e), into its own tally buffers.
 * Work is split into items of rays_per_item rays pulled by the kernel's warps
 * from one atomic counter, so grids of uneven size share the SMs.
 */
typedef struct {
  rt_grid grid;          /* the enclosure's grid and device fields */
  uint64_t n_rays;       /* rays of its estimate */
  rt_tally_buf tally;    /* its tallies (accumulated) */
} rt_enclosure;

typedef struct {
  int32_t rays_per_item; /* rays per work item (0 = 4096) */
  int32_t threads;       /* walk threads per block, multiple of 32, <= 256 (0 = 256) */
} rt_batch_opts;

typedef struct rt_batch rt_batch;  /* opaque plan */

/* Plan: validates every enclosure and uploads the per-enclosure tables to device
 * memory it allocates (synchronous).  Only RT_SRC_EMIT (optionally | RT_TAU_CUT). */
rt_status rt_batch_create(int32_t n_encl, const rt_enclosure *encl, const rt_spectral *spec,
                          uint64_t seed, int32_t flags, const rt_batch_opts *opts, rt_batch **out);
/* Trace all enclosures of a plan with the table kappa: one memset and two kernel
 * launches on the stream, no allocation and no host synchronisation. */
rt_status rt_batch_trace(rt_batch *plan, const float *kappa, void *stream);
/* Free a plan (after its traces have completed). */
rt_status rt_batch_destroy(rt_batch *plan);
/* One-shot create + trace + destroy, stream-ordered. */
rt_status rt_trace_batch(int32_t n_encl, const rt_enclosure *encl, const float *kappa,
                         const rt_spectral *spec, uint64_t seed, int32_t flags,
                         const rt_batch_opts *opts, void *stream);

/*
 * Process-wide launch shapes, set by an autotuner (no effect on results):
 * kappa_t_per_block = temperature nodes per rt_build_kappa block (1..8, 0 = 8);
 * walk_blocks_per_sm = resident 256-thread blocks per SM the rt_trace walk is
 *   compiled for (4: 64 registers per thread, 5: 48; 0 = 5);
 * walk_refill_idle = idle lanes of a warp that trigger loading new rays in the
 *   rt_trace walk (12 or 16; 0 = 16);
 * walk_group = rays of an rt_trace call grouped by wavenumber before the walk, so
 *   that the lanes of a warp read one row of the table (a counting pass over the
 *   rays' Philox draws; scratch of 4 bytes per ray + 8 per wavenumber): 1 never,
 *   2 always, 0 = when there are at least 32 rays per wavenumber.  Tallies are
 *   sums, so the grouping changes only their binary64 summation order.
 */
typedef struct {
  int32_t kappa_t_per_block;
  int32_t walk_blocks_per_sm;
  int32_t walk_refill_idle;
  int32_t walk_group;
  int32_t reserved[4];
} rt_tuning;
rt_status rt_set_tuning(const rt_tuning *t);
rt_status rt_get_tuning(rt_tuning *t);

/*
 * rt_march -- the paper's spectrally resolved kernel (Section 3, Eq. I and the
 * (I_in - I_out) reduction): for each of n_paths rays, starting at pos (device
 * [n_paths][3], m, inside the grid) with direction dir (device [n_paths][3]),
 * and each spectral sample nu_j, the intensity I_in(nu_j) (device [n_nu], W m^-2
 * sr^-1 (m^-1)^-1, NULL = 0) crosses the ray's cells (the binary32 walk of
 * rt_trace) as
 *   I <- I exp(-kappa l) + I_b(nu_j, T_cell) (1 - exp(-kappa l))
 * with kappa the cell's table value (as in rt_trace) and I_b Eq. (planck).
 *   I_out   optional device [n_paths][n_nu]: the intensity leaving the grid.
 *   power   device [n_paths] (binary64, overwritten): sum_j (I_in - I_out) dnu [m^-1],
 *           W m^-2 sr^-1 lost by the beam along the path.
 *   nvis    optional device [n_paths] (overwritten): the number of cells each path
 *           crosses (each crossing is n_nu updates of Eq. I).
 *   status  optional device status word (RT_DEV_NONFINITE, RT_DEV_STEPCAP).
 * 0 <= n_paths <= 65535 per call; with n_paths = 0 nothing is read or written and the
 * buffers may be NULL.  Asynchronous.
 */
rt_status rt_march(const rt_grid *grid, const float *kappa, const rt_spectral *spec,
                   int64_t n_paths, const float *pos, const float *dir, const float *I_in,
                   float *I_out, double *power, int32_t *nvis, uint32_t *status, void *stream);

/* Zero a tally buffer of ncells cells (asynchronous). */
rt_status rt_tally_zero(const rt_tally_buf *tally, int64_t ncells, void *stream);

/*
 * rt_tally -- final reduction of Section 3 (sum of the absorbed power over all
 * cells, binary64) and the energy balance.  Sets tally->scalars[1] and [3] on the
 * device, then copies scalars[0..3] into host_scalars (required) and, if
 * host_absorbed is not NULL, absorbed[0..ncells) into it.  SYNCHRONISES the stream.
 * Returns the device status bits as a status: RT_E_NONFINITE, RT_E_STEPCAP,
 * RT_E_TIMEOUT, RT_E_UNSORTED, RT_E_INVAL (missing table column), else RT_OK.
 */
rt_status rt_tally(const rt_tally_buf *tally, int64_t ncells, double *host_absorbed,
                   double host_scalars[4], void *stream);

/*
 * Surrogate network for the kappa lookup (the learned part; the paper has no
 * network: it stands in for Eq. tau evaluated at a cell's state).  An MLP
 * 4 -> 128 -> 128 -> 128 -> 128 -> 1 with SiLU on the four hidden layers maps
 * u = affine(log nu, T, p, x) in [-1, 1]^4 to y, and log kappa = out_mean +
 * out_scale * y (kappa in cm^-1, natural log).  Parameters are one binary32
 * device vector of RT_MLP_NPARAM values, row-major W[out][in]:
 *   W1[128][4] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
 *   W4[128][128] b4[128] w5[128] b5[1].
 * The hidden 128x128 layers run on the tensor cores in BF16 with FP32
 * accumulation; the first layer, the head and the loss are FP32.
 */
#define RT_MLP_NPARAM 50305
#define RT_MLP_GRAD_ONLY 1   /* rt_mlp_train_step: gradient only, no Adam update */

typedef struct {
  float in_lo[4], in_hi[4];  /* raw input range of (log nu [ln cm^-1], T [K], p [atm], x) */
  float out_mean, out_scale; /* log kappa = out_mean + out_scale * y */
} rt_mlp_norm;

/* log kappa for n raw inputs (device [n][4]) into out (device [n]); n = 0 reads and
 * writes nothing (the buffers may then be NULL).  Asynchronous. */
rt_status rt_mlp_forward(const float *params, const rt_mlp_norm *norm, const float *inputs,
                         int64_t n, float *out, uint32_t *status, void *stream);

/*
 * One training step on a batch of n samples (device inputs [n][4], targets [n] =
 * log kappa): loss = 0.5 mean((y - (target - out_mean)/out_scale)^2), its
 * gradient into grad (device [RT_MLP_NPARAM], overwritten), and unless
 * flags & RT_MLP_GRAD_ONLY one Adam update (beta 0.9 / 0.999, eps 1e-8, bias
 * corrected with `step` >= 1) of params with moments adam_m, adam_v (device
 * [RT_MLP_NPARAM], caller-zeroed before the first step).  loss (device [1]) is
 * overwritten.  Asynchronous.
 */
rt_status rt_mlp_train_step(float *params, float *adam_m, float *adam_v, float *grad,
                            const float *inputs, const float *targets, int64_t n,
                            const rt_mlp_norm *norm, float lr, int32_t step, int32_t flags,
                            float *loss, uint32_t *status, void *stream);

/*
 * n_steps consecutive training steps without a host round trip per step.  Step
 * s = step_first - 1 + i (i = 0 .. n_steps - 1; step_first >= 1) is
 * rt_mlp_train_step on the batch of `batch` samples starting at row
 * (s mod (n / batch)) * batch of inputs / targets (device [n][4], [n]; the
 * n mod batch trailing rows are not used), with Adam step number s + 1 and the
 * cosine learning rate
 *   lr(s) = lr1 + (lr0 - lr1) (1 + cos(pi s / max(1, total_steps - 1))) / 2
 * evaluated in binary64 and rounded to binary32.  losses (optional device
 * [n_steps]) receives each step's loss; grad receives the last step's gradient
 * (the earlier steps' are not stored).  Requires 1 <= batch <= n and
 * step_first - 1 + n_steps <= total_steps.  Asynchronous.
 */
rt_status rt_mlp_train_steps(float *params, float *adam_m, float *adam_v, float *grad,
                             const float *inputs, const float *targets, int64_t n, int64_t batch,
                             const rt_mlp_norm *norm, double lr0, double lr1, int32_t step_first,
                             int32_t n_steps, int32_t total_steps, float *losses, uint32_t *status,
                             void *stream);

/*
 * rt_trace_mlp -- rt_trace (RT_SRC_EMIT) with the absorption coefficient of every
 * visited cell taken from the surrogate network at the cell's state:
 *   kappa = exp(MLP(log nu_j, T_cell, p_cell, x_cell)) [cm^-1]
 * (p_cell = p_ref, x_cell = x_ref where the grid has no p / x field; no table,
 * no interpolation, no density scaling).  The rays, walk, deposits and tallies
 * are those of rt_trace; the emission weight uses the network's kappa of the
 * emitting cell.  Rays are processed in 128-ray tiles, several tiles per block
 * sharing the resident weights; each tile's live rays' queries are evaluated
 * together on the tensor cores at every step.  A ray whose transmission has
 * underflowed to zero (and no RT_TAU_CUT) needs no further kappa: it takes its
 * remaining steps at once, without network evaluations, and its lane takes a new
 * ray (the visits, deposits and escaped weight are unchanged).
 */
rt_status rt_trace_mlp(const rt_grid *grid, const float *params, const rt_mlp_norm *norm,
                       const rt_spectral *spec, uint64_t ray_begin, uint64_t n_rays,
                       uint64_t n_rays_total, uint64_t seed, uint32_t enclosure, int32_t flags,
                       const rt_tally_buf *tally, const rt_record *record, void *stream);

/*
 * rt_mlp_make_samples -- n training samples for the surrogate drawn from n_p
 * line-by-line tables (device kappa[n_p][nT][n_nu] from rt_build_kappa at
 * pressures p_nodes (device [n_p]) and the spec's T grid and x_ref).  Sample i:
 * Philox4x32-10 counter (i, 0, 0, 0x6d6c70), key = seed, picks j, the T node, the
 * pressure node and x uniform in [x_lo, x_hi]; inputs[i] = (log nu_j, T_k, p, x),
 * targets[i] = log(kappa x / x_ref) (kappa is linear in the mole fraction).
 */
rt_status rt_mlp_make_samples(const float *tables, int32_t n_p, const float *p_nodes,
                              const rt_spectral *spec, float x_lo, float x_hi, uint64_t seed,
                              int64_t n, float *inputs, float *targets, void *stream);

/*
 * Spectral-band ensembles of surrogate networks (the learned part; no paper
 * passage).  One network of the layout above per band of band_pts consecutive
 * wavenumber indices: network b serves j in [b band_pts, min((b + 1) band_pts,
 * n_nu)), n_bands = ceil(n_nu / band_pts) <= 65535.  A network for a narrow band
 * only has to resolve that band's lines, which one network for the whole window
 * cannot.  Parameters: device [n_nets][RT_MLP_NPARAM] (network b at b *
 * RT_MLP_NPARAM); norms: DEVICE array of n_nets rt_mlp_norm (each band's log nu
 * range and output scale).  The caller owns every buffer; the calls allocate only
 * stream-ordered scratch (BF16 weight tiles: 96 KB per network for a walk, 192 KB
 * for training, plus the training step's activations and gradient partials; a
 * banded walk also 4 bytes per ray for the band-grouped order).  Bad sizes, NULL
 * buffers or out-of-range arguments return RT_E_INVAL before any launch; a bounded
 * device wait that gives up sets RT_DEV_TIMEOUT in the status word.  The norms are
 * read on the device and are not validated.
 */

/* Training samples for an ensemble: n_per_band samples per band b (rows b n_per_band
 * .. of inputs device [n_bands][n_per_band][4], targets [n_bands][n_per_band]),
 * drawn as in rt_mlp_make_samples but with j in the band's own wavenumbers: Philox4x32-10
 * counter (i, i >> 32, b + 1, 0x6d6c70), key = seed.  j is uniform in the band, except for
 * a fraction emission_mix (in [0, 1], decided per sample by the low byte of word 3 against
 * round(256 emission_mix)) drawn with probability proportional to kappa I_b(nu_j, T_k) at
 * the sample's (p, T) node: the emission the walk samples.  Asynchronous. */
rt_status rt_mlp_make_samples_bands(const float *tables, int32_t n_p, const float *p_nodes,
                                    const rt_spectral *spec, int32_t band_pts, float x_lo, float x_hi,
                                    float emission_mix, uint64_t seed, int64_t n_per_band, float *inputs,
                                    float *targets, void *stream);

/* rt_mlp_train_steps for n_nets independent networks at once (one launch per kernel
 * and step for all of them): network b trains on its own n samples (rows b n .. of
 * inputs [n_nets][n][4], targets [n_nets][n]) with its own norm (norms: device
 * [n_nets]), parameters and Adam moments (params, adam_m, adam_v, grad: device
 * [n_nets][RT_MLP_NPARAM]).  Step s uses batch s mod (n / batch) of every network,
 * the learning-rate schedule of rt_mlp_train_steps; losses[i] (optional) is the
 * mean over the networks of their step-i losses.  Requires 1 <= n_nets <= 65535
 * and batch * n_nets <= 2^30.  Asynchronous. */
rt_status rt_mlp_train_steps_nets(int32_t n_nets, float *params, float *adam_m, float *adam_v, float *grad,
                                  const float *inputs, const float *targets, int64_t n, int64_t batch,
                                  const rt_mlp_norm *norms, double lr0, double lr1, int32_t step_first,
                                  int32_t n_steps, int32_t total_steps, float *losses, uint32_t *status,
                                  void *stream);

/* rt_mlp_forward for n_nets networks: network b maps rows b n .. of inputs (device
 * [n_nets][n][4]) to out[b n ..] (device [n_nets][n]) with norms[b] (device).
 * Asynchronous. */
rt_status rt_mlp_forward_nets(int32_t n_nets, const float *params, const rt_mlp_norm *norms, const float *inputs,
                              int64_t n, float *out, uint32_t *status, void *stream);

/*
 * rt_trace_mlp_bands -- rt_trace_mlp with a spectral-band ensemble: the kappa of a
 * ray at wavenumber index j comes from network floor(j / band_pts).  The rays,
 * walk, deposits and tallies are those of rt_trace (the same Philox rays); the
 * rays are grouped by band (a counting pass over their Philox draws) and each block
 * takes work items of one band's rays with that band's network resident.  Tallies
 * are sums, so the grouping changes only the binary64 summation order.  At most
 * 2^32 - 1 rays per call when there is more than one band.  Asynchronous.
 */
rt_status rt_trace_mlp_bands(const rt_grid *grid, int32_t band_pts, const float *params,
                             const rt_mlp_norm *norms, const rt_spectral *spec, uint64_t ray_begin,
                             uint64_t n_rays, uint64_t n_rays_total, uint64_t seed, uint32_t enclosure,
                             int32_t flags, const rt_tally_buf *tally, const rt_record *record, void *stream);

/*
 * rt_trace_lbl -- rt_trace with the absorption coefficient of every visited cell
 * summed line by line at the cell's own (T, p, x): Eqs. (S) and (tau) evaluated
 * per step over the lines within the cutoff of nu_j, in binary32 with a Kahan
 * sum (no table, no interpolation).  One warp per ray; lines as in rt_build_kappa.
 */
rt_status rt_trace_lbl(const rt_grid *grid, const rt_lines *lines, const rt_spectral *spec,
                       uint64_t ray_begin, uint64_t n_rays, uint64_t n_rays_total, uint64_t seed,
                       uint32_t enclosure, int32_t flags, const rt_tally_buf *tally,
                       const rt_record *record, void *stream);

/* Self-test of the tensor-core path: D = A B^T for 128x128 FP32 row-major A, B
 * (rounded to BF16), D FP32 row-major [128][128].  Asynchronous. */
rt_status rt_tc_selftest(const float *A, const float *B, float *D, uint32_t *status, void *stream);

/* Self-test of the transposed operand path: D = A^T B (D[m][n] = sum_k A[k][m]
 * B[k][n]) for 128x128 FP32 row-major A, B (rounded to BF16), both written as tiles
 * with one row per contraction index and read by the tensor core MN-major, as the
 * training backward pass reads its output-gradient and activation tiles.
 * Asynchronous. */
rt_status rt_tc_selftest_mn(const float *A, const float *B, float *D, uint32_t *status, void *stream);

/*
 * rt_alu_probe -- measured ALU ceilings of the current GPU, for the line sum's
 * roofline: out[0] = binary32 FMA lane operations per second, out[1] = MUFU
 * reciprocal (rcp.approx) lane operations per second, each from a kernel of
 * independent chains filling every SM, best of three timed launches (CUDA
 * events).  Synchronises the stream.
 */
rt_status rt_alu_probe(double *out, void *stream);

/*
 * rt_wait_probe -- exercises the bounded waits that guard the library's bulk copies and
 * tensor-core products (failure detection without a fault): one block waits on an
 * mbarrier with the kernels' bounded try-wait loop for `limit` iterations (1 .. 2^24).
 * arrive = 0: nothing arrives, the wait gives up and RT_DEV_TIMEOUT is OR-ed into the
 * device status word (rt_status_read then returns RT_E_TIMEOUT); arrive = 1: the
 * barrier completes first and the status is left as it was.  Asynchronous.
 */
rt_status rt_wait_probe(uint32_t limit, int32_t arrive, uint32_t *status, void *stream);

/* Synchronise the stream and translate a device status word into an rt_status. */
rt_status rt_status_read(const uint32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
