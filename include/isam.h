/*
 * isam.h -- C ABI of the GB300 (sm_103a) full-range dispersion-encoded ISAM
 * library: the forward model, its adjoint and the weighted-l1 MBIR solve of
 * Mason, Davies & Bagnaninchi, "Blur resolved OCT: full-range ISAM through
 * dispersion encoding" (arXiv 1905.06058).
 *
 * Model (paper §2-§3):
 *   s = A eta = Re( diag(e^{j phi}) K eta )                       Eq. (12)-(13)
 *   K = F_lat^{-1} o [Stolt-mapped axial transform, min-max NUFFT] o F_lat
 *                                                                  Eq. (3), (16)
 *   phi(k) = sum_{i=1..n_disp} a_i (k - k0)^i                      Eq. (7)
 *   A^H y = F_lat^{-1} N'( conj(e^{j phi}) F_lat y )               Eq. (17)
 *   eta~ = argmin 1/2 ||A eta - s_d||^2 + lambda w^T |eta|         Eq. (12)
 *   solved by FISTA with weighted complex soft threshold            Alg. 1, Eq. (14)
 *   and the relative-residual stop rule                             Eq. (15)
 *
 * Conventions (the paper leaves them open; they are fixed here):
 *   k_j = k_min + j dk, j < nk, dk = (k_max - k_min)/(nk - 1), k0 = (k_min+k_max)/2
 *   z_n = (n - nz/2) dz, dz = pi / (nz dk)   (full complex range pi/dk)
 *   q   = 2 pi fftfreq(nx, dx) (and ny, dy); lateral FFTs are unitary;
 *   the axial transform carries 1/sqrt(nz) and the focus phase e^{j(2k+beta)z0},
 *   beta = -sqrt(4k^2 - q^2); samples with 4k^2 <= q^2 are zero in A and ignored in A^H;
 *   NUFFT: oversampling K = 2 nz, J-neighbour min-max interpolation (J = 4, 6 or 8)
 *   with Kaiser-Bessel-shaped scaling (alpha = 2.34 J) over the design set
 *   n' = -nz/2..nz/2; FISTA uses step 1/L and threshold lambda w / L, L = ||A||^2.
 *
 * Layouts (row-major, last index fastest), element types by plan precision:
 *   image eta : complex [ny][nx][nz]  (interleaved re,im; float2 or double2)
 *   spectra s : real    [ny][nx][nk]  (float or double), A-scans contiguous
 *   weights w : real    [nz]          (per image row, broadcast over x, y)
 *
 * Ownership and threading: the caller owns every buffer passed in; a plan owns
 * its device workspace and tables.  Calls are asynchronous on the plan's
 * stream unless stated; device pointers must be valid CUDA device (or managed)
 * memory of the plan's device.  Errors found before launch are returned
 * immediately; a CUDA launch failure returns ISAM_ERR_CUDA.  A plan may be
 * used by one host thread at a time; distinct plans are independent.
 */
#ifndef ISAM_H
#define ISAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISAM_OK = 0,
  ISAM_ERR_INVALID = 1,     /* bad argument (null pointer, size, range)     */
  ISAM_ERR_OOM = 2,         /* device allocation failed                     */
  ISAM_ERR_CUDA = 3,        /* a CUDA call or kernel launch failed          */
  ISAM_ERR_NONFINITE = 4,   /* the solve produced a NaN or Inf              */
                            /* 5 is not used: no kernel waits on a flag,    */
                            /* a counter or another kernel                  */
  ISAM_ERR_UNSUPPORTED = 6  /* valid but not implemented (size, J, os)      */
} isam_status;

enum { ISAM_FP32 = 0, ISAM_FP64 = 1 };

/* Acquisition geometry and numerics: the problem as the paper states it
 * (spectral samples, lateral grid, NA and focus, dispersion; §2, §4.1). */
typedef struct {
  int32_t nx, ny;      /* lateral samples, 2^p or 3*2^p (p >= 3), <= 4096; ny = 1: B-scan */
  int32_t nk;          /* spectral samples per A-scan (power of two, 16..4096)      */
  int32_t nz;          /* depth samples of the image (power of two, >= 16); 0: nk   */
  double k_min, k_max; /* band edges, rad/m (k_max > k_min > 0)                     */
  double dx, dy;       /* lateral pitch, m (dy ignored when ny = 1)                 */
  double na;           /* numerical aperture (recorded; the unfiltered model, b = 1) */
  double z0;           /* focal depth on the z grid, m (Stolt origin)               */
  int32_t n_disp;      /* number of dispersion coefficients used (0..4)             */
  double disp[4];      /* a_1..a_4, rad m^i, about k0 (Eq. 7)                       */
  int32_t precision;   /* ISAM_FP32 or ISAM_FP64                                    */
  int32_t nufft_J;     /* interpolation neighbours: 4, 6 or 8 (0: 6)               */
  int32_t nufft_os;    /* oversampling factor: 2 (0: 2)                            */
  int32_t flags;       /* ISAM_FLAG_* bits (0: defaults)                          */
} isam_params;

/* Stolt positions and spectral phases depend on (|q|, k) only; by default a
 * plan tabulates them when the table takes at most 64 MiB (B-scans) and the
 * kernels evaluate them otherwise (volumes).  This flag forces evaluation. */
#define ISAM_FLAG_NO_STOLT_TABLE 1
/* The 1-D dispersion-encoded model of each A-scan on its own, the model of the
 * DEFR objective (Eq. 10, our scaling): every column uses the q = 0 Stolt map
 * (beta = -2k), so there is no lateral coupling and no focus term; dx, dy, na
 * and z0 have no effect.  Forward, adjoint, solve and calibration calls then
 * work on this model (MBIR on Eq. 10 with the weighted l1 prior). */
#define ISAM_FLAG_AXIAL_MODEL 4

typedef struct isam_plan isam_plan;

/* Options of the MBIR solve (Alg. 1, §3.1). */
typedef struct {
  double lambda_rel;        /* lambda = lambda_rel * ||A^H s_d||_inf ...          */
  double lambda_abs;        /* ... unless lambda_abs > 0, which is used as is     */
  int32_t max_iter;         /* FISTA iterations (>= 1)                            */
  double tol;               /* stop when r_r < tol (Eq. 15); 0 disables the rule  */
  int32_t check_every;      /* iterations between stop-rule evaluations (>= 1);   */
                            /* an evaluating iteration reads z^{k-2} as well and   */
                            /* forms the norm partials, the others update from the */
                            /* lateral spectrum of eta^k - g/L (same iterates).    */
                            /* r_r is evaluated on the device and read by the host */
                            /* two iterations later: a solve that stops has queued */
                            /* up to two more, whose kernels write nothing         */
  const void* w_dev;        /* nullable device [nz] weights w (real, plan type)   */
  int32_t residual_addback; /* 1: return z + (1/L) A^H (s_d - A z) (Alg. 1 end)   */
  double L;                 /* step 1/L; 0: power-iteration estimate, cached      */
  double eps;               /* r_r denominator guard (0: 1e-30)                   */
  int32_t prior;            /* ISAM_PRIOR_* (0: the weighted l1 of Eq. 12)         */
  int32_t objective;        /* 1: report the Eq. 12 objective of z^K in the info   */
  int32_t prior_iters;      /* ISAM_PRIOR_TV: dual steps per prox (0: 20)          */
} isam_solve_opts;

/* Priors of the MBIR objective (§3.1: Eq. 12 extends to other convex priors):
 * ISAM_PRIOR_L1: lambda w^T |eta| (Eq. 12), prox = the soft threshold of Eq. 14.
 * ISAM_PRIOR_HAAR_DEPTH: lambda ||details(W eta)||_1, W the orthonormal Haar
 *   transform along depth of every A-scan (all log2(nz) levels, the coarsest
 *   approximation coefficient unpenalised); prox = W^H T_{lambda/L}(W u).
 * ISAM_PRIOR_TV: lambda TV(eta), isotropic total variation over (x, z) of each
 *   B-scan slice (forward differences, zero at the far edge); the prox is
 *   found on its dual by fast gradient projection, prior_iters steps per
 *   FISTA iteration, warm started from the previous iteration within a solve.
 * Both need w_dev = NULL and tol = 0, and TV no resumed state (k > 0)
 * (ISAM_ERR_UNSUPPORTED otherwise); neither is available to the unrolled
 * (calibration) entry points. */
enum { ISAM_PRIOR_L1 = 0, ISAM_PRIOR_HAAR_DEPTH = 1, ISAM_PRIOR_TV = 2 };

/* Resumable solver state (checkpoint/restart).  z1 = z^{k}, z2 = z^{k-1} are
 * caller-owned device images; k iterations are done.  Pass k = 0 to start. */
typedef struct {
  void* z1;
  void* z2;
  int32_t k;
  double lambda;
  double L;
} isam_solve_state;

typedef struct {
  int32_t iterations;  /* iterations performed by this call                   */
  double rr;           /* last evaluated relative residual (-1 if never)      */
  double lambda;       /* regularisation used                                 */
  double L;            /* Lipschitz constant used                             */
  int32_t status;      /* isam_status of the solve                            */
  double objective;    /* 1/2 ||A z^K - s_d||^2 + lambda w^T |z^K| (Eq. 12) when
                          asked for with the l1 prior, else -1; z^K before any
                          add-back; one extra A and two reductions            */
} isam_solve_info;

/* Device memory of plans (workspace and tables) comes from cudaMalloc unless
 * an allocator is installed: alloc(bytes, ctx) returns device memory of the
 * current device or NULL (reported as ISAM_ERR_OOM, and the partly built plan
 * is released); free(ptr, ctx) returns it.  Process-wide; each block is given
 * back to the allocator that made it, even after another one is installed.
 * Both NULL restores cudaMalloc; exactly one NULL is ISAM_ERR_INVALID.  For
 * pooling allocators of a host framework, and for injecting allocation
 * failures in tests.  Pinned host staging memory is not affected. */
typedef void* (*isam_alloc_fn)(size_t bytes, void* ctx);
typedef void (*isam_free_fn)(void* ptr, void* ctx);
isam_status isam_set_allocator(isam_alloc_fn alloc, isam_free_fn free_fn, void* ctx);

/* Create a plan: validates p, builds the NUFFT tables (FP64 on the device),
 * allocates workspace on the current device, binds `stream` (a cudaStream_t,
 * NULL for the legacy default stream).  Synchronous.  *out is NULL on error. */
isam_status isam_plan_create(const isam_params* p, void* stream, isam_plan** out);
void isam_plan_destroy(isam_plan* plan);
isam_status isam_set_stream(isam_plan* plan, void* stream);

/* s = A eta (Eq. 12-13, 16).  eta: device image, s: device spectra. */
isam_status isam_forward(isam_plan* plan, const void* eta, void* s);

/* eta = A^H s (Eq. 17), exact adjoint of isam_forward under <a,b> = Re(a^H b). */
isam_status isam_adjoint(isam_plan* plan, const void* s, void* eta);

/* MBIR solve (Alg. 1): s_d device spectra -> eta_out device image.  Synchronises
 * the plan's stream before returning (it reads back the stop rule and status).
 * state may be NULL. info may be NULL. */
isam_status isam_solve(isam_plan* plan, const void* s_d, const isam_solve_opts* opts,
                       void* eta_out, isam_solve_state* state, isam_solve_info* info);

/* The same solve with host buffers: copies s_d in, solves, copies eta out. */
isam_status isam_solve_host(isam_plan* plan, const void* s_d_host,
                            const isam_solve_opts* opts, void* eta_out_host,
                            isam_solve_info* info);

/* L = ||A^H A|| by power iteration from the device start image v0 (NULL: a fixed
 * deterministic start), in FP64 on the device whatever the plan precision (when
 * the FP64 kernels fit the shared memory, else in the plan precision).  Stops
 * after `iters` steps or when the estimate changes by <= rtol relative;
 * iters = 0 selects the default used by isam_solve (1000 steps, 1e-11).
 * Synchronous.  The result is cached in the plan and used by isam_solve. */
isam_status isam_lipschitz(isam_plan* plan, int32_t iters, double rtol, const void* v0,
                           double* L_out);

/* The data term of the MBIR objective (Eq. 12): *value = 1/2 ||A eta - s_d||^2
 * (host double, the sum of squares taken in FP64) for a device image eta and
 * device spectra s_d; when r_out is not NULL the residual spectra A eta - s_d
 * are written there (device, [ny][nx][nk], the plan's precision; r_out may
 * alias neither eta nor s_d).  With it a caller differentiates the data
 * fidelity without leaving the library: d/d eta = A^H r (isam_adjoint),
 * d/d theta = <dA/dtheta eta, r> (isam_param_grad).  Synchronous. */
isam_status isam_data_fidelity(isam_plan* plan, const void* eta, const void* s_d, void* r_out,
                               double* value);

/* max |eta_i| of a device image (used for lambda = c ||A^H s||_inf).  A NaN in
 * the image makes the result NaN.  Synchronous. */
isam_status isam_max_abs(isam_plan* plan, const void* eta, double* out);

/* max |x_i| over n complex device elements (FP32: float2, FP64: double2),
 * written to the device double *out; asynchronous on `stream`.  It allocates
 * nothing, for callers that cannot: a thread recording a stream capture owned
 * by another framework, an acquisition loop whose memory was fixed at
 * start-up, or code whose device memory is held by a pooling allocator.  The
 * paper has no counterpart; it is the reduction behind lambda = c ||A^H s||_inf.
 * Scratch is a static device array of ISAM_NOALLOC_MAX_PARTIALS doubles
 * (512 KiB, held by every GPU that loads the library until exit); n above
 * ISAM_NOALLOC_MAX_PARTIALS * 2048 returns ISAM_ERR_UNSUPPORTED.  A NaN in x
 * makes *out NaN.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and must come before any stream capture; the address
 * is kept per CUDA context, so after cudaDeviceReset (a new primary context)
 * the next call looks it up again and must likewise come before any capture.
 * Calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. */
#define ISAM_NOALLOC_MAX_PARTIALS 65536
isam_status isam_max_abs_noalloc(const void* x, int64_t n, int32_t precision, double* out,
                                 void* stream);

/* The filter B(q, k) of Eq. 3 (b of Eq. 16) for the lens and the intensity
 * drop-off; the paper's results use B = 1 (§3.2), which is the default.
 * b: host complex table, interleaved (re, im) doubles, [ny/2 + 1][nx/2 + 1][nk]
 * (one row block when ny = 1); entry (|my|, |mx|, j) multiplies the spectral
 * sample (q = (±mx, ±my) in FFT index, k_j), so B is symmetric in q.  NULL
 * restores B = 1.  A, A^H, solves, calibration and batches then use
 * S = B . e^{j phi} e^{j(2k+beta)z0} . H.  Rebuilds the phase tables, forgets
 * the cached L; ISAM_ERR_INVALID for non-finite entries.  Synchronous. */
isam_status isam_set_filter(isam_plan* plan, const double* b);

/* The direct dispersion-compensated reconstruction of Eq. 9 on the full-range
 * depth grid, A-scan by A-scan (the exact adjoint of the ISAM_FLAG_AXIAL_MODEL
 * operator, evaluated as an nz-point FFT):
 *   eta(x, n) = (1/sqrt(nz)) sum_j s_d(x, k_j) e^{-j phi(k_j)} e^{-j 2 k_j z_n}.
 * s_d: device spectra, eta: device image.  Asynchronous on the plan's stream. */
isam_status isam_dispersion_compensated_ifft(isam_plan* plan, const void* s_d, void* eta);

/* ---- Calibration of the dispersion coefficients and the focal depth -------
 * The paper notes that a (Eq. 7) may be found by an autofocus method (§2)
 * and places the focus at a known depth; here theta = (a_1, a_2, a_3, a_4, z0)
 * can instead be fitted by gradient descent through the model.  A depends on
 * theta only through the spectral phase e^{j phi(k)} e^{j (2k + beta) z0}, so
 *   dA/dtheta x = Re F^{-1}( j D_theta . e^{j phi} e^{j(2k+beta)z0} . N(F x) ),
 *   D_{a_i} = (k - k0)^i,  D_{z0} = 2k + beta  (zero on evanescent samples).
 * Derivatives are taken with respect to a_i in rad m^i and z0 in m. */
#define ISAM_N_PARAMS 5

/* Replace theta of an existing plan (a_1..a_{n_disp}; the rest become 0):
 * rebuilds the phase and Stolt tables and forgets the cached L (||A||^2
 * depends on phi).  Synchronous.  Other tables and workspace are kept. */
isam_status isam_set_model(isam_plan* plan, int32_t n_disp, const double* disp, double z0);

/* grad[i] = <dA/dtheta_i x, y> (real inner product on spectra), i < 5: the
 * gradient of <A x, y> with respect to theta.  x: device image, y: device
 * spectra; grad: host double[ISAM_N_PARAMS].  Sums in FP64.  Synchronous. */
isam_status isam_param_grad(isam_plan* plan, const void* x, const void* y, double* grad);

/* Unrolled FISTA with checkpoints, for differentiating the reconstruction:
 * K = opts->max_iter iterations of Alg. 1 from z^0 = 0 with lambda =
 * opts->lambda_abs (> 0) and step 1/opts->L (> 0) held fixed, no stop rule,
 * no add-back (ISAM_ERR_INVALID otherwise), weights opts->w_dev.  Writes z^K
 * to z_out and, if ckpt is not NULL, the pair (z^{c e}, z^{c e - 1}) before
 * iteration c e + 1 to images 2c, 2c+1 of ckpt, e = every; ckpt holds
 * isam_unrolled_checkpoint_images(K, every) images of the plan's type.
 * Synchronous; ISAM_ERR_NONFINITE if an iterate is not finite. */
int32_t isam_unrolled_checkpoint_images(int32_t K, int32_t every);
isam_status isam_fista_unrolled(isam_plan* plan, const void* s_d, const isam_solve_opts* opts,
                                int32_t every, void* ckpt, void* z_out);

/* Gradient of <z_bar, z^K> (real inner product) through the iterations of
 * isam_fista_unrolled (same s_d, opts, every and the ckpt it wrote, theta
 * unchanged since): grad (host double[5]) with respect to theta and, when
 * s_bar (device spectra) is not NULL, with respect to s_d.  Each segment of
 * `every` iterations is recomputed from its checkpoint, then reversed:
 *   ubar = J_T(u^k)^T zbar^k   (Jacobian of the soft threshold, Eq. 14),
 *   etabar = ubar - (1/L) A^H A ubar,
 *   grad -= (1/L)(<dA ubar, A eta^k - s_d> + <A ubar, dA eta^k>),
 *   s_bar += (1/L) A ubar,
 *   zbar^{k-1} += (1 + mu_{k-1}) etabar,  zbar^{k-2} -= mu_{k-1} etabar.
 * Workspace: 2 every + 8 images and two spectra, kept by the plan.  Synchronous. */
isam_status isam_fista_unrolled_vjp(isam_plan* plan, const void* s_d,
                                    const isam_solve_opts* opts, int32_t every,
                                    const void* ckpt, const void* z_bar, void* s_bar,
                                    double* grad);

/* ---- Batched solves as one CUDA graph --------------------------------------
 * Many independent MBIR solves (Alg. 1), each with its own plan (geometry,
 * dispersion, focus), data, lambda, L, weights and iteration count, recorded
 * once into one CUDA graph; isam_batch_run replays the whole batch with one
 * launch.  Each entry runs on its own forked stream, so entries overlap on
 * the GPU; one entry is the same kernel sequence as isam_solve.  With
 * opts[i].tol > 0 the stop rule runs on the device: every iteration after the
 * first check carries the stop flag (its kernels write nothing once the rule
 * has fired), eta_out[i] receives the iterate of the stopping check, and
 * isam_batch_run reports that check's iteration and r_r.
 * Create: plans distinct, on one device, profiling off; L = 0 is estimated now
 * (cached per plan);
 * lambda_rel is evaluated on the device at every run from the s_d[i] contents
 * then.  The batch keeps the pointers: plans, s_d[i] (device spectra) and
 * eta_out[i] (device images) must stay valid, and the plans unused by other
 * calls while a run is in flight.  Synchronous.  `stream` must not be the
 * legacy default stream (capture is not allowed there); NULL makes the batch
 * create its own.  Run: launches the graph on that stream, waits, and fills
 * info[i] (nullable; rr = -1); returns the first non-OK entry status.  The
 * caller orders earlier work on s_d before the run (e.g. synchronises).
 * The graph records the plans' tables and launch shapes: while a batch
 * exists, isam_set_model, isam_set_filter, isam_autotune, isam_autotune_ex
 * and isam_set_tuning on its plans return ISAM_ERR_INVALID, and the plans must
 * not be destroyed. */
typedef struct isam_batch isam_batch;
isam_status isam_batch_create(isam_plan* const* plans, int32_t n, const void* const* s_d,
                              const isam_solve_opts* opts, void* const* eta_out, void* stream,
                              isam_batch** out);
isam_status isam_batch_run(isam_batch* batch, isam_solve_info* info);
/* Kernel launches recorded in the batch's graph (-1 for NULL). */
int64_t isam_batch_kernel_count(const isam_batch* batch);
/* Per-entry latency of the last isam_batch_run: ms[i] = device time from the
 * start of the graph to the end of entry i's solve (timing events recorded as
 * nodes of the graph), ms[n].  ISAM_ERR_INVALID before the first run.  The
 * paper has no counterpart (it solves one B-scan at a time). */
isam_status isam_batch_entry_ms(const isam_batch* batch, double* ms);
void isam_batch_destroy(isam_batch* batch);

/* Launch shapes and FFT radices of a plan.  The paper has no counterpart (it
 * states the method, not its kernels); none of these changes what is computed,
 * only the order of rounding (the radices) or nothing at all (tile, table).
 *   lateral_tile   pairs of depth columns per block of the lateral update: 1, 2,
 *                  4 or 8 where they fit (threads = 8 x tile x L/8 <= 512, tile
 *                  <= columns/2), 0 for the built-in choice (reported as used)
 *   stolt_table    1: read the plan's table of Stolt positions and phases; 0:
 *                  evaluate them in the kernels (the only mode without a table)
 *   axial_radix    16: column-split radix-16 passes for the FP32 axial
 *                  transforms at K = 2048 and 4096 (three shared-memory passes);
 *                  8: radix-8 passes on column pairs (four); other plans run
 *                  radix 8 whatever the value
 *   lateral_radix  the same choice for the FP32 lateral tiles of L = 1024 (4
 *                  pairs) and L = 256 (8 pairs) */
typedef struct {
  int32_t lateral_tile;
  int32_t stolt_table;
  int32_t axial_radix;
  int32_t lateral_radix;
} isam_tuning;

/* Pick launch shapes and radices by timing the plan's own FISTA iteration
 * (CUDA events on the plan's stream, zero data, 10 timed iterations per
 * candidate): every feasible tile width, table versus evaluated positions when
 * the plan holds a table, and radix 8 versus 16 where both forms exist.  The
 * fastest is kept in the plan and used by later calls; *out (nullable)
 * receives it.  Overwrites the plan's workspace.  When the environment
 * variable ISAM_AUTOTUNE_CACHE names a file, a choice recorded there for the
 * same device, sizes, precision, J and table mode is used without timing (if
 * still feasible), and new choices are appended as lines
 * "<key> -> tile=<t> stolt=<m> radix=<axial>/<lateral>".  ISAM_ERR_INVALID
 * while a batch records the plan.  Synchronous. */
isam_status isam_autotune_ex(isam_plan* plan, isam_tuning* out);
/* isam_autotune_ex reporting the tile and the table mode only. */
isam_status isam_autotune(isam_plan* plan, int32_t* tile, int32_t* stolt_table);
/* The plan's current tuning (the built-in choices until tuned or set). */
isam_status isam_get_tuning(const isam_plan* plan, isam_tuning* out);
/* Install a tuning chosen elsewhere (offline, or to compare the forms):
 * ISAM_ERR_INVALID for values out of range or a tile that does not fit,
 * ISAM_ERR_UNSUPPORTED for stolt_table = 1 on a plan without a table, and
 * ISAM_ERR_INVALID while a batch records the plan. */
isam_status isam_set_tuning(isam_plan* plan, const isam_tuning* tuning);

/* Kernel launches issued by the last isam_forward / isam_adjoint / isam_solve. */
int64_t isam_last_launch_count(const isam_plan* plan);

/* Optional per-kernel timing: while enabled, every kernel launch of the plan is
 * bracketed by CUDA events on the plan's stream and its device time is added to
 * one of these classes.  Measurement support; not part of the method. */
enum {
  ISAM_KCLASS_AX_FWD = 0,      /* Stolt NUFFT forward (axial)               */
  ISAM_KCLASS_AX_ADJ = 1,      /* Stolt NUFFT adjoint (axial)               */
  ISAM_KCLASS_AX_FUSED = 2,    /* Stolt NUFFT, residual, adjoint NUFFT      */
  ISAM_KCLASS_LAT_UPDATE = 3,  /* fused lateral IFFT, FISTA step, FFT       */
  ISAM_KCLASS_LAT_FFT = 4,     /* plain lateral FFT passes                  */
  ISAM_KCLASS_MISC = 5,        /* reductions and elementwise kernels        */
  ISAM_KCLASS_COUNT = 6
};
/* Enable (1) or disable (0) the timing; synchronises the plan's stream. */
isam_status isam_profile_enable(isam_plan* plan, int32_t on);
/* Synchronise the stream, then copy accumulated milliseconds and launch counts
 * per class into ms[ISAM_KCLASS_COUNT], counts[ISAM_KCLASS_COUNT]; reset if asked. */
isam_status isam_profile_read(isam_plan* plan, double* ms, int64_t* counts, int32_t reset);

const char* isam_status_string(isam_status s);

#ifdef __cplusplus
}
#endif
#endif /* ISAM_H */
