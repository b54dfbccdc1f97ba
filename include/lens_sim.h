/*
 * lens_sim.h -- C ABI of the GB300 (sm_103a) lensed-image simulation library.
 *
 * The library implements the image-simulation pipeline of JAXtronomy (section
 * "Improvements over lenstronomy in image simulation"): a coordinate grid in the
 * observer's angles is ray-traced through the deflectors back to the source plane,
 * the source surface brightness is evaluated on the traced grid, and the lensed
 * image is convolved with the PSF.  The deflector and light models are those of
 * the paper's deflection table (EPL, NIE/SIE, SHEAR, SIS, NFW, TNFW) and light
 * table (SERSIC, SERSIC_ELLIPSE, SERSIC_ELLIPSE_Q_PHI); the subhalo population is
 * the "tens of thousands of dark matter substructures" of the statement of need.
 * The chi^2 log-likelihood and its gradient serve the gradient-based fitting of
 * section "Improvements over lenstronomy in lens modelling".
 *
 * Conventions (apply to every call):
 *  - Angles in arcsec, position angles in radians measured from +x toward +y.
 *  - Images are FP32, row-major [ny][nx]; row i is at y = y0 + (i - (ny-1)/2) * pixel_scale,
 *    column j at x = x0 + (j - (nx-1)/2) * pixel_scale.  With supersampling s, a pixel
 *    holds pixel_scale^2 times the mean of its s x s sub-pixel samples (flux per pixel).
 *  - PSF convolution is the zero-padded 'same'-size true convolution with an odd k x k
 *    kernel: out[i][j] = sum_{a,b} K[a][b] in[i + c - a][j + c - b], c = (k-1)/2.
 *  - Every call returns a lens_status.  No exception or abort crosses the ABI; on an
 *    error nothing is launched and lens_sim_last_error() describes it.
 *  - The caller owns every input and output buffer.  Registered PSFs and subhalo tables
 *    are copied into library-owned device memory, freed by lens_sim_destroy.
 *  - `stream` is a cudaStream_t (may be NULL for the legacy default stream).  Work is
 *    enqueued on it; buffers must stay valid until that work completes.
 *  - Pointers documented "host or device" are classified with cudaPointerGetAttributes.
 *  - A handle is not thread-safe: one thread at a time per lens_sim (the server below
 *    owns its own).
 */
#ifndef LENS_SIM_H
#define LENS_SIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LENS_OK = 0,
  LENS_ERR_INVALID_ARG = -1,  /* bad type, size, parameter range or pointer */
  LENS_ERR_OOM = -2,          /* device memory or memory budget exhausted */
  LENS_ERR_CUDA = -3,         /* a CUDA runtime call failed; see lens_sim_last_error */
  LENS_ERR_TIMEOUT = -4,      /* a bounded wait ran out */
  LENS_ERR_BUSY = -5,         /* admission refused (server) or result still pending (poll) */
  LENS_ERR_UNSUPPORTED = -6,  /* valid request outside what this library implements */
  LENS_ERR_CANCELLED = -7     /* the request was cancelled before it ran */
} lens_status;

#define LENS_MAX_DEFLECTORS 8
#define LENS_MAX_SUPERSAMPLE 8
#define LENS_MAX_PSF 135
#define LENS_N_FREE_PARAMS 15
#define LENS_PROFILE_PARAMS 12       /* floats in lens_profile.p (the widest layout uses 12) */
#define LENS_MAX_SHAPELET_NMAX 10    /* SHAPELETS order limit: at most 66 amplitudes */
#define LENS_MAX_SHAPELET_COEFFS ((LENS_MAX_SHAPELET_NMAX + 1) * (LENS_MAX_SHAPELET_NMAX + 2) / 2)
#define LENS_MAX_MULTIPOLE_ORDER 32
#define LENS_MAX_MULTIPOLE_ELL_ORDER 32  /* elliptical multipoles (LENS_MULTIPOLE_ELL) */

/* Deflector profile types and their parameter layouts p[] (deflection table rows). */
typedef enum {
  LENS_SIS = 0,         /* theta_E, cx, cy                 alpha = theta_E (dx,dy)/r          */
  LENS_SIE = 1,         /* theta_E, q, phi, cx, cy          Kormann et al. 1994, q in (0,1]   */
  LENS_EPL = 2,         /* theta_E, gamma, q, phi, cx, cy   Tessore & Metcalf 2015 series      */
  LENS_SHEAR = 3,       /* gamma1, gamma2                   about the origin                   */
  LENS_POINT_MASS = 4,  /* theta_E, cx, cy                                                     */
  LENS_NFW = 5,         /* Rs, alpha_Rs, cx, cy             alpha_Rs = deflection at Rs        */
  LENS_TNFW = 6,        /* Rs, alpha_Rs, r_t, cx, cy        Baltz, Marshall & Oguri 2009       */
  LENS_EPL_E1E2 = 7,    /* theta_E, gamma, e1, e2, cx, cy  q = (1-c)/(1+c), c = |e|, phi = arg(e)/2 */
  LENS_SIE_E1E2 = 8,    /* theta_E, e1, e2, cx, cy                                              */
  LENS_MULTIPOLE = 9,   /* m, a_m, phi_m, cx, cy, r_E      circular multipole of integer order
                         * m in [1, LENS_MAX_MULTIPOLE_ORDER], r_E > 0:
                         * kappa = r_E a_m cos(m (phi - phi_m)) / (2 r); potential
                         * r_E a_m r cos(m dphi) / (1 - m^2), or (r_E a_1 / 2) r ln(r/r_E) cos(dphi)
                         * for m = 1                                                           */
  LENS_EPL_MULTIPOLE_M1M3M4 = 10, /* theta_E, gamma, e1, e2, cx, cy, a_1, dphi_1, a_3, dphi_3, a_4,
                         * dphi_4: EPL_E1E2 plus the m = 1, 3, 4 multipoles about its centre with
                         * r_E = theta_E and phi_m = phi + dphi_m (phi = the EPL position angle) */
  LENS_CSE = 11,        /* A, s, e1, e2, cx, cy               cored steep ellipsoid (Oguri 2021),
                         * kappa = A / (2 (s^2 + x'^2 + y'^2/q^2)^(3/2)), s > 0              */
  LENS_NFW_ELLIPSE_CSE = 12, /* Rs, alpha_Rs, e1, e2, cx, cy   NFW convergence on ellipses
                         * xi^2 = q x'^2 + y'^2/q, evaluated as a sum of 44 CSEs (deflection
                         * within 1e-7 of the exact profile's maximum on 1e-3 < xi/Rs < 1e3) */
  LENS_HERNQUIST_ELLIPSE_CSE = 13, /* sigma0, Rs, e1, e2, cx, cy  kappa = sigma0 ((2 + x^2) F(x) - 3)
                         * / (x^2 - 1)^2, x = xi/Rs (Hernquist 1990 projection), 44 CSEs     */
  LENS_MULTIPOLE_ELL = 14 /* m, a_m, phi_m, q, phi_e, cx, cy, r_E  elliptical multipole: kappa =
                         * r_E a_m cos(m (varphi - phi_m)) / (2 R) in the frame of an ellipse of
                         * axis ratio q and angle phi_e, R^2 = q x''^2 + y''^2/q, varphi =
                         * atan2(y''/sqrt(q), x'' sqrt(q)); m an integer in [1, LENS_MAX_MULTIPOLE_ELL_ORDER],
                         * q in [0.2, 1], r_E > 0, at most one per system.  Evaluated from the
                         * Fourier series of 2 kappa r (its up to 321 coefficients computed on the
                         * host once per call and copied to the device beside the system). */
} lens_profile_type;

/* Source light profile types (light table rows). I = amp exp(-b_n [(R/R_s)^(1/n) - 1]),
 * R = sqrt(q x'^2 + y'^2/q), b_n = 1.9992 n - 0.3271. */
typedef enum {
  LIGHT_SERSIC_ELLIPSE_Q_PHI = 0, /* amp, R_sersic, n, q, phi, cx, cy */
  LIGHT_SERSIC_ELLIPSE = 1,       /* amp, R_sersic, n, e1, e2, cx, cy */
  LIGHT_SERSIC = 2,               /* amp, R_sersic, n, cx, cy         */
  LIGHT_SHAPELETS = 3             /* n_max, beta, cx, cy: Cartesian shapelets (Refregier 2003),
                                   * I = sum_k amp_k phi_n1(x'/beta) phi_n2(y'/beta) / beta with
                                   * the orthonormal Hermite functions phi_n; integer n_max in
                                   * [0, LENS_MAX_SHAPELET_NMAX]; the (n_max+1)(n_max+2)/2
                                   * amplitudes come from lens_system.source_coeffs, ordered by
                                   * n = n1 + n2 = 0..n_max and within n by n1 = n, n-1, ..., 0 */
} light_profile_type;

typedef struct { int type; float p[LENS_PROFILE_PARAMS]; } lens_profile;
typedef struct { int type; float p[8]; } light_profile;

/* Grid spec: nx, ny >= 1; supersample in [1, 8]; pixel_scale > 0; (x0, y0) = grid centre. */
typedef struct { int nx, ny, supersample; float pixel_scale, x0, y0; } lens_grid;

/* One lens system.  `deflectors` is HOST memory (at most LENS_MAX_DEFLECTORS entries).
 * Subhalos (truncated NFW) are either a structure of arrays `subhalos` = [5][n_subhalos]
 * (cx, cy, Rs, alpha_Rs, r_t; host or device memory) with subhalo_table = -1, or a
 * resident table id from lens_sim_register_subhalos (then `subhalos` is ignored).
 * psf_id = -1 skips the PSF step (the binned, unconvolved image is returned). */
typedef struct {
  lens_grid grid;
  const lens_profile* deflectors;
  int n_deflectors;
  const float* subhalos;
  int n_subhalos;
  int subhalo_table;
  light_profile source;
  int psf_id;
  const float* source_coeffs;  /* HOST memory: SHAPELETS amplitudes (else NULL, 0) */
  int n_source_coeffs;
} lens_system;

typedef struct {
  int device;               /* CUDA device ordinal                                   */
  size_t mem_budget_bytes;  /* 0 = no limit; workspace growth beyond it -> LENS_ERR_OOM */
  int max_batch;            /* largest n_sys / n_points accepted per call (0 = 4096)  */
  unsigned flags;           /* reserved, must be 0                                   */
} lens_sim_config;

typedef struct lens_sim lens_sim;

/* Create a handle bound to config->device (NULL config = device 0, no budget).
 * Allocates nothing on the device until first use. */
int lens_sim_create(const lens_sim_config* config, lens_sim** out);

/* Synchronise the handle's work and free everything it owns.  NULL is a no-op. */
void lens_sim_destroy(lens_sim* sim);

/* Text of the last error on this handle; valid until the next call on it. */
const char* lens_sim_last_error(const lens_sim* sim);

/* Copy an odd k x k FP32 kernel (host memory, row-major, 1 <= k <= LENS_MAX_PSF) into
 * device memory and return its id.  The kernel is used as given (not re-normalised). */
int lens_sim_register_psf(lens_sim* sim, const float* kernel, int k, int* psf_id);

/* Copy a subhalo population (SoA [5][n], host or device) into a resident device table
 * with its per-subhalo constants precomputed, and return its id.  n may be 0. */
int lens_sim_register_subhalos(lens_sim* sim, const float* soa, int n, int* table_id);

/* Simulate n_sys lensed images (image simulation steps 1-3 plus the supersample
 * bin-down).  out_images is a HOST array of n_sys pointers, each to ny*nx floats in
 * host or device memory (host outputs are staged and copied back on `stream`; the call
 * then synchronises the stream before returning).  Systems may differ in every size. */
int lens_sim_image(lens_sim* sim, const lens_system* systems, int n_sys, float* const* out_images,
                   void* stream);

/* Ray-shooting: total deflection of `sys` (deflector list + subhalos) at n points.
 * x, y, ax, ay are DEVICE arrays of n floats.  The grid, source and PSF are ignored. */
int lens_sim_deflection(lens_sim* sim, const lens_system* sys, const float* x, const float* y, int n,
                        float* ax, float* ay, void* stream);

/* PSF step alone: convolve n_img DEVICE images [n_img][ny][nx] with a registered PSF. */
int lens_sim_convolve(lens_sim* sim, const float* in, int n_img, int ny, int nx, int psf_id, float* out,
                      void* stream);

/* Launch variants of the fused trace kernel (0: one CTA of 8 warps per work unit; 1: one CTA of
 * 4 warps that sums the unit's 8 subhalo slices in two passes; 2-4: thread-block clusters of
 * 2, 4 or 8 CTAs per unit).  Every variant gives
 * bitwise-identical images; only the speed differs.  lens_sim_autotune times each variant
 * on `sample` (reps launches each, CUDA events on `stream`, synchronising it), makes the
 * fastest the handle's default for single-system calls, and reports the index and the mean
 * milliseconds of each variant (ms_per_variant may be NULL; n_ms entries are written at most).
 * lens_sim_set_variant sets it directly (0 .. LENS_TRACE_VARIANTS-1). */
#define LENS_TRACE_VARIANTS 5
int lens_sim_autotune(lens_sim* sim, const lens_system* sample, int reps, int* best_variant,
                      float* ms_per_variant, int n_ms, void* stream);
int lens_sim_set_variant(lens_sim* sim, int variant);

/* Far-field interpolation of the subhalo sum (optional; off by default; CHANGES RESULTS within
 * the bound below).  The paper's method sums every subhalo at every traced point ("Statement of
 * need": ray tracing through tens of thousands of substructures); this option approximates the
 * far part of that sum.  With kappa > 0, lens_sim_image and lens_sim_autotune sum a subhalo that
 * is at least kappa * h from a work unit's box of traced points (h: the larger half-width of the
 * box; the subhalos the kernel's near-field test marks are never approximated) at the box's
 * 8 x 8 Chebyshev nodes instead of at the unit's 288 points, and interpolate the unit's summed
 * node values to its points with the tensor Lagrange basis: the local-expansion step of a
 * black-box fast multipole method (Fong and Darve 2009).  Error bound, per approximated
 * subhalo, as the largest error of its deflection over the box relative to its largest value
 * there (FP64 analysis over tau in [0.5, 20], Rs in [0.002, 0.1], all directions, box aspect
 * 1:1 .. 4:1): kappa = 3: 1.2e-6, 4: 1.4e-7, 6: 6e-9; the error of a traced point's total
 * deflection is below that fraction of the sum of the approximated subhalos' magnitudes, plus
 * FP32 rounding of the interpolation (Lebesgue constant of the 8 x 8 grid below 6).
 * kappa = 0 restores the exact sum; 0 < kappa < 3 or a non-finite kappa is LENS_ERR_INVALID_ARG.
 * It applies to every lens_sim_image call of the handle (single systems and the batched launch
 * of n_sys > 1 alike, each system's image the same either way under the same convolution, see
 * lens_sim_set_conv_method) and to both autotuners.  Every
 * launch variant and batch schedule still gives bitwise-identical images.  Ray shooting
 * (lens_sim_deflection), the likelihood and its adjoint, the server and the no-alloc entry
 * point always use the exact sum. */
int lens_sim_set_far_field(lens_sim* sim, float kappa);

/* Schedule of the batched launch (lens_sim_image with n_sys > 1; the batched configuration of
 * the paper's workloads): `form` is the persistent trace kernel (0: CTAs of 4 warps summing a
 * unit's 8 subhalo slices in two passes; 1: CTAs of 8 warps; 2: clusters of 2 CTAs x 4 warps),
 * `order` the unit queue (0: systems by per-unit cost, largest first; 1: as given).  Every
 * schedule gives bitwise-identical images.  lens_sim_autotune_batch runs the batch once per
 * schedule to warm it up, then times `reps` calls (CUDA events on `stream`, synchronising it),
 * makes the fastest the handle's schedule and returns it; `ms` (may be NULL) receives the mean
 * milliseconds per call of the 2 * LENS_BATCH_FORMS schedules, indexed form * 2 + order.  The
 * outputs receive the batch's images.  Needs n_sys >= 2; on an error the schedule is left as it
 * was. */
#define LENS_BATCH_FORMS 3
int lens_sim_set_batch_schedule(lens_sim* sim, int form, int order);
int lens_sim_autotune_batch(lens_sim* sim, const lens_system* systems, int n_sys, float* const* out_images,
                            int reps, int* best_form, int* best_order, float* ms, void* stream);

/* PSF method of lens_sim_image (single system) and lens_sim_convolve.  LENS_CONV_DIRECT: tiled
 * direct convolution.  LENS_CONV_FFT: FFT convolution (the paper's method for large kernels):
 * the kernel's central 7 x 7 core convolved directly plus its wings (the rest) by four-step
 * FFTs of real rows on a grid padded to powers of two >= (n + (k-1)/2) in each direction, at
 * most 1024; larger images return LENS_ERR_UNSUPPORTED.  The wings' spectrum is computed once
 * per (psf_id, padded size) and kept by the handle.  LENS_CONV_AUTO (the default): FFT when
 * k >= LENS_CONV_FFT_MIN_K and the padded size fits, else direct.  Both compute the same
 * convolution; they differ by FP32 rounding only (the FFT's, carried by the wings alone, is of
 * order eps log2(M) of their contribution, below 1e-5 relative L-inf).  The batched and
 * likelihood paths always use the direct form, so a batched image equals its single-system
 * image bitwise when that call convolves directly (always for k < LENS_CONV_FFT_MIN_K). */
#define LENS_CONV_AUTO 0
#define LENS_CONV_DIRECT 1
#define LENS_CONV_FFT 2
#define LENS_CONV_FFT_MIN_K 33
int lens_sim_set_conv_method(lens_sim* sim, int method);

/* Chi^2 log-likelihood of n_points parameter vectors against DEVICE data [ny][nx]:
 *   sigma^2 = sigma_bkg^2 + max(m, 0)/t_exp,   logL = -1/2 sum (d - m)^2 / sigma^2,
 * with m the PSF-convolved model.  params is DEVICE [n_points][15] in the order
 * EPL_E1E2 (theta_E, gamma, e1, e2, cx, cy), SHEAR (g1, g2),
 * SERSIC_ELLIPSE (amp, R, n, e1, e2, cx, cy); `sys` supplies the grid, PSF and the fixed
 * subhalos (its deflector list and source are ignored).  out_logL: DEVICE [n_points];
 * out_grad: DEVICE [n_points][15] or NULL for the likelihood only. */
int lens_sim_grad(lens_sim* sim, const lens_system* sys, const float* data, float sigma_bkg, float t_exp,
                  const float* params, int n_points, float* out_logL, float* out_grad, void* stream);

/* Linear amplitude solver (the paper's lens-modelling section: solving linear amplitudes reduces
 * the number of sampled parameters).  For each of n_points parameter vectors (layout of
 * lens_sim_grad; the amplitude entry is ignored) the source amplitude is the weighted
 * least-squares solution against DEVICE data [ny][nx]:
 *   amp = sum w d m1 / sum w m1^2,   w = 1 / (sigma_bkg^2 + max(d, 0)/t_exp),
 * with m1 the PSF-convolved model per unit amplitude (data-based weights keep the problem
 * linear), and out_logL (DEVICE [n_points], may be NULL) = -1/2 sum w (d - amp m1)^2.
 * out_amp: DEVICE [n_points]. */
int lens_sim_linear_amp(lens_sim* sim, const lens_system* sys, const float* data, float sigma_bkg, float t_exp,
                        const float* params, int n_points, float* out_amp, float* out_logL, void* stream);

/* ---------------------------------------------------------------- allocation-free form
 * The paper has no counterpart to this entry point; it is a deployment convenience.
 * lens_sim_image_noalloc simulates one system for callers that cannot allocate device
 * memory: applications whose device memory is reserved up front by their own pool allocator,
 * and latency-critical loops that forbid cudaMalloc/cudaFree after start-up because those
 * calls can synchronise the whole device.  It runs lens_sim_image's single-system kernels
 * (subhalo constants and the fused trace kernel) and always the direct PSF convolution (where
 * lens_sim_image's automatic choice takes the FFT for k >= LENS_CONV_FFT_MIN_K; both compute
 * the same convolution, within the image tolerance).  It takes no handle and calls no
 * cudaMalloc, cudaFree or allocating library routine.  Its scratch (per-subhalo constants, the
 * unconvolved image and an elliptical multipole's harmonics) is one fixed array of
 * LENS_NOALLOC_SCRATCH_BYTES of device memory that every GPU loading the library holds until
 * the process exits.  A system with an elliptical multipole costs one copy of its harmonics
 * from pageable host memory, which waits for the stream's earlier work.
 *  - It runs on the CURRENT device.  sys: grid (as for lens_sim_image: 1..16384 pixels per
 *    side, a finite positive pixel scale, a finite centre), HOST deflector list, source;
 *    subhalos in device memory (SoA [5][n]); subhalo_table must be -1; psf_id is ignored.
 *  - psf: device pointer to an odd k x k kernel (1 <= k <= LENS_MAX_PSF), or NULL (or k = 0)
 *    to skip the PSF step.  out_image: caller-owned device buffer of ny*nx floats.  Every
 *    buffer must be memory of the current device: a host pointer or another GPU's memory
 *    returns LENS_ERR_INVALID_ARG with nothing launched.
 *  - n_subhalos > LENS_NOALLOC_MAX_SUBHALOS or nx*ny > LENS_NOALLOC_MAX_PIXELS returns
 *    LENS_ERR_OOM with nothing launched; bad arguments return LENS_ERR_INVALID_ARG and a
 *    failed CUDA call LENS_ERR_CUDA (there is no handle, hence no error text).
 *  - Each call looks up the array's device address in the current device's context
 *    (cudaGetSymbolAddress, which allocates nothing).  The first call on a device also loads
 *    the library's kernels there: make that first call before any stream capture.
 *  - All calls share the one array, which keeps the last call's contents; each call writes
 *    everything it reads.  Calls that overlap on the GPU (different streams, or several host
 *    threads) race on the array: serialise them on one stream. */
#define LENS_NOALLOC_MAX_SUBHALOS 20000
#define LENS_NOALLOC_MAX_PIXELS (512 * 512)
#define LENS_NOALLOC_SCRATCH_BYTES (LENS_NOALLOC_MAX_SUBHALOS * 224 + LENS_NOALLOC_MAX_PIXELS * 4 + 642 * 4)
int lens_sim_image_noalloc(const lens_system* sys, const float* psf, int k, float* out_image, void* stream);

/* ---------------------------------------------------------------- measurement
 * lens_sim_pipe_rates measures the handle's GPU pipes that bound its ALU-bound kernels (the
 * subhalo sum: FP32 FMAs and one MUFU reciprocal square root per pair), the denominators of
 * their rooflines.  Each rate comes from a short launch of independent dependency chains of
 * one instruction kind (32 warps per SM), timed by every block with the SM clock, so it is
 * per SM and per SM clock, independent of the clock the GPU ran at: the median over SMs of the
 * lane operations of an SM's blocks over the longest of their times.  rates[0]: FP32 lane
 * operations (an FMA counted once) with packed FFMA2 chains; rates[1]: the same with scalar
 * FFMA chains; rates[2 .. 5]: MUFU results with rsqrt.approx.ftz, ex2.approx.ftz,
 * lg2.approx.ftz and rcp.approx.ftz chains.  The first min(n_rates, LENS_PIPE_RATES) entries
 * are written (later ones set to 0).  It synchronises its own stream, takes a few
 * milliseconds and a scratch of about 4 KB per SM (within the memory budget), and is not
 * meant for a timed region.  rates NULL or n_rates < 1: LENS_ERR_INVALID_ARG; a failed CUDA
 * call: LENS_ERR_CUDA. */
#define LENS_PIPE_RATES 6
int lens_sim_pipe_rates(lens_sim* sim, double* rates, int n_rates);

/* ---------------------------------------------------------------- serving
 * A server owns its own lens_sim state, streams and a worker thread that admits requests
 * by a device-memory budget, batches what is waiting, and overlaps batches on the device.
 * Requests reference HOST buffers: for kind 0 (image) `out` receives ny*nx floats; for
 * kind 1 (likelihood + gradient) `data` holds the ny*nx observation, `params` the 15
 * parameters, `out` the log-likelihood (1 float) and `out_grad` 15 floats.  The buffers
 * must stay valid until wait/poll returns LENS_OK, LENS_ERR_CANCELLED or an error. */
typedef struct lens_server lens_server;
typedef struct {
  int kind;                 /* 0 image, 1 log-likelihood + gradient */
  lens_system sys;          /* psf_id refers to the server's lens_sim (see lens_serve_sim) */
  const float* data;
  float sigma_bkg, t_exp;
  const float* params;
  float* out;
  float* out_grad;
} lens_request;

int lens_serve_create(const lens_sim_config* config, int max_inflight, lens_server** out);
/* The server's own handle, for lens_sim_register_psf / lens_sim_register_subhalos before
 * submitting requests that use them (registration is safe while other requests run: the
 * registry is shared under a lock and read as copies). */
lens_sim* lens_serve_sim(lens_server* srv);
/* Text of the server's most recent failed request ("" if none); the calling thread's copy,
 * valid until its next call. */
const char* lens_serve_last_error(lens_server* srv);
/* Enqueue a request; LENS_ERR_BUSY when max_inflight requests are already queued or running. */
int lens_serve_submit(lens_server* srv, const lens_request* req, unsigned long long* ticket);
/* Wait up to timeout_ms (>= 0) for a ticket: LENS_OK, LENS_ERR_TIMEOUT, LENS_ERR_CANCELLED,
 * or the request's own error.  Never blocks longer than timeout_ms plus one poll period. */
int lens_serve_wait(lens_server* srv, unsigned long long ticket, int timeout_ms);
/* LENS_OK when done, LENS_ERR_BUSY while pending, or the request's error. */
int lens_serve_poll(lens_server* srv, unsigned long long ticket);
/* Cancel a request that has not started; LENS_ERR_BUSY if it is already running. */
int lens_serve_cancel(lens_server* srv, unsigned long long ticket);
/* Hold (paused = 1) or release (0) admission: queued requests stay queued and can be
 * cancelled; running work completes.  For draining a device and for tests that need a
 * request to stay pending. */
int lens_serve_pause(lens_server* srv, int paused);
/* Latency percentiles (submit -> completion) and throughput over completed requests. */
int lens_serve_stats(lens_server* srv, double* p50_ms, double* p99_ms, double* requests_per_s);
/* Forget the latency samples (e.g. between arrival-rate sweeps). */
int lens_serve_reset_stats(lens_server* srv);
/* Stop the worker, cancel what is still queued, wait for running work, free everything.
 * No wait/poll may be in progress on another thread. */
void lens_serve_destroy(lens_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* LENS_SIM_H */
