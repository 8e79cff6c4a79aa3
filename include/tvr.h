/*
 * tvr.h -- C ABI of the GB300 TV-CT gradient-method library (libtvr.so).
 *
 * Problem (Sec. II-A, eq. TVobjectivefunction, eq. TV):
 *     x* = argmin_{x in Q} phi(x),  phi(x) = 1/2 ||A x - b||_2^2 + alpha TV_tau(x),
 *     Q = R_+^N (Sec. IV-A),
 * where A is the ray-voxel system matrix (Siddon intersection lengths) and
 * TV_tau(x) = sum_j h_tau(D_j x) is the Huber-smoothed discrete TV with
 * forward differences D_j (h_tau(z) = ||z|| - tau/2 for ||z|| >= tau,
 * ||z||^2 / (2 tau) otherwise; a difference leaving the grid is 0).
 *
 * Conventions shared by every call:
 *   - volume: n x n x n unit voxels centred at the origin; voxel
 *     j = ix + n*iy + n*n*iz (x fastest); N = n^3;
 *   - rays: view v, detector pixel (p, q) -> row i = v*Pu*Pv + q*Pu + p;
 *     m = V*Pu*Pv;
 *   - vectors are float32, contiguous; x, grad: N entries; b, resid: m.
 *   - "host or device": a vector argument may point to device memory or to
 *     host memory (pageable or pinned); host vectors are staged through
 *     device buffers owned by the system, with the copies on `stream`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is asynchronous on `stream` unless a call says that it
 *     synchronises.  Calls that use one tvr_system share its workspace and
 *     must be ordered on one stream (or otherwise serialised by the caller).
 *   - Return value: a tvr_status; no exception crosses the ABI.
 *     tvr_last_error() gives a message for the calling thread's last error.
 */
#ifndef TVR_H
#define TVR_H

#include <stdint.h>

#if defined(__GNUC__)
#define TVR_API __attribute__((visibility("default")))
#else
#define TVR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tvr_status {
  TVR_OK = 0,
  TVR_NOT_CONVERGED = 1,   /* warning: stopped at k_max */
  TVR_ERR_ARG = -1,        /* invalid argument; nothing was launched */
  TVR_ERR_OOM = -2,        /* a device allocation failed */
  TVR_ERR_CUDA = -3,       /* a CUDA runtime call failed */
  TVR_ERR_LINESEARCH = -4, /* a line search hit its trial cap */
  TVR_ERR_NONFINITE = -5   /* a control scalar became NaN or Inf */
} tvr_status;

typedef enum tvr_geometry_kind {
  TVR_CONE = 0,     /* every ray of a view starts at the view's point source */
  TVR_PARALLEL = 1  /* ray of pixel (p, q) starts at src + pixel offset */
} tvr_geometry_kind;

typedef enum tvr_storage {
  TVR_STORAGE_FP32 = 0,         /* CSR and CSC, float32 values, int32 indices, int64 pointers */
  TVR_STORAGE_BF16_ROWSCALE = 1, /* values a_ij = s_i q_ij: per-row FP32 scale s_i = max_j a_ij and
                                   bfloat16 codes q_ij = bf16(a_ij / s_i) (round to nearest even),
                                   the same codes in CSR and CSC; FP32 accumulation; the back
                                   projection applies exactly the transpose of the forward matrix */
  TVR_STORAGE_U16_ROWSCALE = 3,  /* values a_ij = t_i q_ij: per-row FP32 step t_i = fl(s_i / 65535)
                                   with s_i = max_j a_ij, and 16-bit unsigned fixed-point codes
                                   q_ij = min(65535, rint(a_ij / t_i)), the same codes in CSR and
                                   CSC; 2 bytes per entry like BF16 storage, but each entry within
                                   half a step (s_i / 131070) of a_ij instead of 2^-9 of it; FP32
                                   accumulation; exact transpose as for BF16 */
  TVR_STORAGE_MATRIX_FREE = 2   /* no stored A: every projection computes its entries on the fly as
                                   the float32 length of the ray segment (source to pixel centre)
                                   inside the voxel's unit box, from float32 view constants; the
                                   forward (per ray, walking the slabs of its major axis) and the
                                   back projection (per voxel, over the pixels of its projected
                                   footprint) evaluate the same entry function, so they are exact
                                   transposes.  The entries differ from the FP64 Siddon lengths of
                                   the stored kinds by the float32 rounding of the ray geometry.
                                   Cone-beam scans whose views all separate into x-y and z parts
                                   (detector u and normal without z component, w along z, as on a
                                   circular orbit about z) project by stacks instead, with the
                                   same entries: the forward walks the x-y path that the rays of
                                   a detector column share once for 4 of them, the back
                                   projection the x-y footprint of 4 voxels stacked along z once
                                   for all 4; such systems hold N + 4 m more floats (the stacks'
                                   sums).  Not available: CSR/CSC export, the FP64 entry points,
                                   tvr_solve_sweep */
} tvr_storage;

/* Number of doubles per view record. */
#define TVR_VIEW_FIELDS 12

/*
 * Scan geometry.  `views` is a HOST array of n_views records of 12 doubles:
 * source (or source-plane centre for TVR_PARALLEL) [3], detector centre [3],
 * detector column step u [3] and row step w [3] (pixel pitch included).
 * Pixel (p, q) has centre det + (p - (Pu-1)/2) u + (q - (Pv-1)/2) w.
 */
typedef struct tvr_geometry {
  int32_t n;         /* grid edge, >= 1 */
  int32_t n_views;   /* V >= 1 */
  int32_t det_cols;  /* Pu >= 1 */
  int32_t det_rows;  /* Pv >= 1 */
  int32_t kind;      /* tvr_geometry_kind */
  int32_t reserved;  /* must be 0 */
  const double *views;
} tvr_geometry;

typedef struct tvr_system tvr_system; /* opaque; owns A and all workspace */

/*
 * Build A for a geometry (Sec. II-A: A maps the image to ray sums; its entries
 * here are Siddon ray-voxel intersection lengths computed in FP64 and stored in
 * FP32): each ray is clipped to the volume box, the crossing parameters of all
 * grid planes are merged in increasing order (equal values once), and each
 * consecutive pair gives one entry (voxel of the midpoint, length (t_b - t_a)|d|).
 * Stores CSR (rows in traversal order) and its transpose CSC (rows ascending
 * within a column), with values as `storage` says (tvr_storage).
 * Synchronises `stream` (to size the arrays).
 * *out receives a new system owned by the caller, freed by tvr_system_free.
 * Errors: TVR_ERR_ARG (bad geometry, n^3 >= 2^31), TVR_ERR_OOM, TVR_ERR_CUDA.
 */
TVR_API int tvr_build_system(const tvr_geometry *geom, int32_t storage, void *stream,
                     tvr_system **out);

/* Free a system and every device buffer it owns (synchronises the device). */
TVR_API int tvr_system_free(tvr_system *sys);

/* Shape of A: m rows (rays), N columns (voxels), nnz stored entries (host outputs, nullable). */
TVR_API int tvr_system_shape(const tvr_system *sys, int64_t *m, int64_t *N, int64_t *nnz);

/*
 * Copy A to caller-owned HOST buffers (synchronous): CSR row_ptr[m+1],
 * col[nnz], val[nnz]; CSC col_ptr[N+1], row[nnz], val[nnz].  Any pointer may be
 * NULL to skip that array.  For BF16 storage val holds s_i * q_ij rounded to
 * float32, the value the kernels apply.
 */
TVR_API int tvr_system_export_csr(const tvr_system *sys, int64_t *row_ptr, int32_t *col, float *val);
TVR_API int tvr_system_export_csc(const tvr_system *sys, int64_t *col_ptr, int32_t *row, float *val);

/* y = A x (forward projection).  x: N, y: m; host or device. */
TVR_API int tvr_forward(const tvr_system *sys, const float *x, float *y, void *stream);

/* z = A^T r (back projection, atomic-free CSC gather).  r: m, z: N; host or device. */
TVR_API int tvr_adjoint(const tvr_system *sys, const float *r, float *z, void *stream);

/*
 * phi and its gradient (eq. TVobjectivefunction):
 *   resid = A x - b,  phi = 1/2 ||resid||^2 + alpha TV_tau(x),
 *   grad  = A^T resid + alpha grad TV_tau(x),
 *   grad TV_tau(x) = sum_j D_j^T (D_j x / max(tau, ||D_j x||)).
 * x: N, b: m (host or device).  grad (N) and resid (m) are nullable outputs,
 * host or device; grad == NULL evaluates phi only (no back projection).
 * phi_dev: nullable DEVICE array of 3 doubles {phi, 1/2||r||^2, TV_tau(x)};
 * phi_host: nullable HOST array of 3 doubles, same content -- giving it
 * synchronises `stream`.  The reductions accumulate in double-single (~48-bit)
 * arithmetic and are delivered in FP64; results are deterministic.
 * alpha >= 0, tau > 0 (TVR_ERR_ARG otherwise).
 */
TVR_API int tvr_phi_and_grad(const tvr_system *sys, const float *x, const float *b, double alpha,
                     double tau, double *phi_dev, double *phi_host, float *grad,
                     float *resid, void *stream);

/*
 * FP64 variant of tvr_phi_and_grad (eq. TVobjectivefunction) for verification
 * by finite differences: x, b, grad, resid are DEVICE doubles; A's stored FP32
 * values are promoted to double, so it is the same function phi in double
 * arithmetic.  resid (m doubles) and grad (N doubles) are required outputs;
 * phi_dev / phi_host as in tvr_phi_and_grad.  The reductions are FP64.
 */
TVR_API int tvr_phi_and_grad_f64(const tvr_system *sys, const double *x, const double *b,
                                 double alpha, double tau, double *phi_dev, double *phi_host,
                                 double *grad, double *resid, void *stream);

/*
 * Backward of phi(x; b) for reverse-mode differentiation: with the residual
 * r = A x - b saved by a forward call and the upstream scalar w = *scale_dev
 * (a DEVICE double),
 *   grad_x = w (A^T r + alpha grad TV_tau(x)),   grad_b = -w r   (grad_b nullable).
 * All vectors DEVICE memory; float32 (tvr_phi_vjp) or float64 (tvr_phi_vjp_f64).
 * Asynchronous on `stream`.
 */
TVR_API int tvr_phi_vjp(const tvr_system *sys, const float *x, const float *resid, double alpha,
                        double tau, const double *scale_dev, float *grad_x, float *grad_b,
                        void *stream);
TVR_API int tvr_phi_vjp_f64(const tvr_system *sys, const double *x, const double *resid,
                            double alpha, double tau, const double *scale_dev, double *grad_x,
                            double *grad_b, void *stream);

/*
 * tvr_phi_and_grad without any device allocation (the paper has no
 * counterpart).  For callers that must not allocate device memory while they
 * evaluate phi: code whose device memory is owned by another framework's
 * caching allocator under a fixed budget (an allocation outside that
 * allocator can fail, or fragment what the allocator manages), and
 * latency-bound loops that must not enter the driver's allocator (cudaMalloc
 * and cudaFree can synchronise the device and take unbounded time).  Same
 * kernels and results as tvr_phi_and_grad (no resid output).  Its scratch --
 * the residual and three reduction slots -- is one fixed device array inside
 * the library, about 17.5 MiB (16 MiB residual, 1.5 MiB reductions), held on
 * every GPU that loads the library until the process exits, so:
 *   - the system's rays m must be <= 4,194,304, else TVR_ERR_ARG;
 *   - the system must store A as FP32 CSR or be matrix-free; BF16 and U16
 *     row-scale storage need a second, row-scaled residual and are refused (TVR_ERR_ARG);
 *     a matrix-free system of separable views also uses its own stack sums,
 *     allocated when it was built;
 *   - x, b (and grad, phi_dev when given) must be DEVICE memory (host data
 *     would need staging buffers), else TVR_ERR_ARG;
 *   - the first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture;
 *   - every call shares the array and zeroes its reduction counters first:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race; order them on one stream.
 * phi_dev / phi_host as in tvr_phi_and_grad (phi_host synchronises).
 */
TVR_API int tvr_phi_and_grad_noalloc(const tvr_system *sys, const float *x, const float *b,
                                     double alpha, double tau, double *phi_dev,
                                     double *phi_host, float *grad, void *stream);

/* In place x <- P_Q(x) = max(x, 0) on n DEVICE floats (Sec. III-A); NaN stays NaN. */
TVR_API int tvr_project_Q(float *x, int64_t n, void *stream);

/*
 * ||G_nu(x)||_2 with G_nu(x) = nu (x - P_Q(x - grad / nu)) (Sec. III-D) for
 * DEVICE vectors x, grad of N floats (N of `sys`, whose workspace is used);
 * the FP64 result is written to the HOST double *out (synchronises `stream`).
 * nu > 0 and finite.
 */
TVR_API int tvr_gradient_map_norm(const tvr_system *sys, const float *x, const float *grad, double nu,
                          double *out, void *stream);

/*
 * The sums behind the acceptance tests of one projected step (Alg. 1, Alg. 2;
 * the BT and nonmonotone tests of Sec. III-A and III-B), exactly as a solver's
 * trial computes them: from the base point p with gradient g and the step s,
 *   xbar = P_Q(p - s g) (float32, rounded as the trial rounds it), d = xbar - p,
 *   sums[0] = ||A xbar - b||^2     sums[1] = ||A d||^2
 *   sums[2] = g^T d                sums[3] = ||d||^2
 *   sums[4] = sum_j B_h(D_j xbar; D_j p)  (Huber Bregman divergence at tau)
 *   sums[5] = TV_tau(xbar)
 * accumulated on the device in double-single and finished in FP64, the
 * precision the line-search decisions rest on.  p, g (N floats), b (m floats)
 * and the optional outputs xbar (N floats) and resid (m floats, A xbar - b)
 * are DEVICE memory; sums is a HOST array of 6 doubles (the call
 * synchronises `stream`).  Uses the system's solver workspace: do not run it
 * concurrently with a solve on the same system.  s > 0 and tau > 0, finite.
 */
TVR_API int tvr_trial_sums(const tvr_system *sys, const float *p, const float *g, const float *b,
                           double s, double tau, double sums[6], float *xbar, float *resid,
                           void *stream);

/* Stopping normalisation of the gradient-map test (Sec. III-D). */
typedef enum tvr_stop_mode {
  TVR_STOP_REL = 0,   /* ||G_k|| / ||G_0|| <= eps (G_0: gradient map of iteration 0) */
  TVR_STOP_PER_N = 1  /* ||G_k|| / N <= eps, as printed in the paper */
} tvr_stop_mode;

/* Number of doubles per history record: k, ||G||, L or theta, mu, beta, trials, f, stop value.
   f = phi(x^(k+1)): GPBB keeps it as phi(x^(0)) plus the exact increments of the
   accepted steps; GP and UPN evaluate it from the accepted trial's residual and
   TV sums. */
#define TVR_HIST_FIELDS 8

typedef struct tvr_solve_opts {
  int32_t k_max;            /* iteration cap (default 20000) -> TVR_NOT_CONVERGED */
  int32_t stop_mode;        /* tvr_stop_mode (default TVR_STOP_REL) */
  int32_t gpbb_K;           /* GPBB memory K (default 2, Sec. III-A), 0..8 */
  int32_t gpbb_max_trials;  /* squarings of beta per GPBB iteration (default 12) */
  int32_t bt_max;           /* increases of L per BT call (default 60) */
  int32_t use_graph;        /* 1 (default): batches of passes replayed as CUDA graphs */
  int32_t batch;            /* passes launched between host checks (default 32) */
  int32_t gpbb_points;      /* GPBB trial points per forward pass: 2 (default; 0 means 2) or 1.
                               With 2, each pass also forms the trial the line search takes
                               after a rejection (step beta^2 theta) and uses it when the first
                               is rejected: the same decisions and iterates as one point per
                               pass, in fewer passes over A */
  int32_t sweep_lanes;      /* tvr_solve_sweep: lanes per row / column of its two projections
                               (the row split): 0 (default) = chosen by timing 2, 4 and 8 lanes
                               on the system at its first sweep, kept for later sweeps on
                               systems of the same shape on the same GPU; 2, 4 or 8 = fixed.
                               Changes only the order of additions */
  int32_t reserved;
  double gpbb_sigma;        /* default 0.1 (Sec. III-A) */
  double gpbb_beta0;        /* default 0.95 (Alg. 1) */
  double rho_L;             /* BT factor (Alg. 2), default 2 */
  double L_bar;             /* initial L estimate (Alg. 2 / Alg. 3), default 1 */
  double mu_bar;            /* initial mu (Alg. 3), default 0.1 * L_bar */
  double *history;          /* nullable HOST array [history_len * TVR_HIST_FIELDS] */
  int64_t history_len;      /* records available in history */
} tvr_solve_opts;

typedef struct tvr_solve_info {
  int32_t status;       /* tvr_status of the solve */
  int32_t iters;        /* accepted iterations (GP/GPBB: k+1; UPN: BT calls) */
  int32_t f_evals;      /* objective evaluations (forward projections of trial points) */
  int32_t g_evals;      /* gradient evaluations (back projections) */
  int32_t trials;       /* rejected line-search / BT trials in total */
  int32_t passes;       /* passes launched, including no-op passes after the stop */
  int32_t history_used; /* records written to opts->history */
  int32_t lanes;        /* tvr_solve_sweep: the row split its projections ran with, lanes per
                           row (forward) | lanes per column (back projection) << 8; 0 for the
                           other solvers */
  double phi;           /* phi(x*) evaluated afresh at the returned point */
  double gnorm;         /* ||G|| of the last iteration */
  double gnorm0;        /* ||G|| of iteration 0 */
  double stop_value;    /* the tested quantity of the last iteration */
  double L;             /* GP/UPN: last L_k; GPBB: 1/theta */
  double theta;         /* GPBB: last BB step; UPN: last theta_k */
  double mu;            /* UPN: last mu_k */
} tvr_solve_info;

/* Fill *opts with the defaults listed above. */
TVR_API void tvr_solve_opts_default(tvr_solve_opts *opts);

/*
 * Solvers.  x holds x^(0) on entry (host or device; N floats) and the result on
 * return.  b: m floats, host or device.  eps > 0.  opts nullable (defaults).
 * info nullable (host).  These calls synchronise `stream`.
 *
 * tvr_solve_gp   -- eq. (gradientmethod), x+ = P_Q(x - theta_k grad phi(x)) with
 *                   theta_k = 1/L_k from BT (Alg. 2) started at L_{k-1}; stop on
 *                   ||G_{L_k}(x^(k))||.
 * tvr_solve_gpbb -- Alg. 1: Barzilai-Borwein theta_k, beta from 0.95 squared until
 *                   f(xbar) < max_{i<=K} f(x^(k-i)) - sigma grad f^T (x - xbar);
 *                   stop on ||G_{1/theta_k}(x^(k))||.
 * tvr_solve_upn  -- Alg. 3: BT from y^(k), mu_k = min(mu_{k-1}, M(x^(k), y^(k)))
 *                   (eq. mu_k_estimate), theta_{k+1} the positive root of
 *                   theta^2 = (1 - theta) theta_k^2 + (mu_k / L_k) theta,
 *                   beta_k = theta_k (1 - theta_k) / (theta_k^2 + theta_{k+1}),
 *                   y^(k+1) = x^(k+1) + beta_k (x^(k+1) - x^(k)); stop on
 *                   ||G_{L_k}(y^(k))||.
 * Returns the solve status (also in info->status).
 */
TVR_API int tvr_solve_gp(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                 const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream);
TVR_API int tvr_solve_gpbb(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                   const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream);
TVR_API int tvr_solve_upn(const tvr_system *sys, const float *b, double alpha, double tau, double eps,
                  const tvr_solve_opts *opts, float *x, tvr_solve_info *info, void *stream);

/*
 * Batch of independent problems (each its own system, data b, alpha and
 * x^(0) / x*): solves them with one method (1 = GP, 2 = GPBB, 3 = UPN) at the
 * same tau, eps and options, side by side on one stream per system (each
 * stream relaunched as soon as its batch of passes drains) so that small
 * problems run concurrently on the GPU.  Arrays of `count` pointers
 * (HOST arrays; the vectors they point to are host or device, as in the
 * single solves); a system may appear only once.  infos: nullable HOST array
 * of count records.  Synchronises `stream` at entry and every system's work
 * at exit.  Returns TVR_OK if every problem converged, else the first error
 * status, else TVR_NOT_CONVERGED.  Not an entry of the paper: a batching of
 * its methods over problems.
 */
TVR_API int tvr_solve_batch(tvr_system *const *systems, int32_t count, int32_t method,
                            const float *const *bs, const double *alphas, double tau, double eps,
                            const tvr_solve_opts *opts, float *const *xs, tvr_solve_info *infos,
                            void *stream);

/*
 * Parameter sweep: k <= 8 solves of the same system and data b with
 * regularisation parameters alphas[0..k-1] (same tau, eps and options), run in
 * lockstep so that every forward and back projection reads A once for all of
 * them (sparse matrix times 8 interleaved vectors).  method: 1 = GP, 2 = GPBB,
 * 3 = UPN, each exactly as in tvr_solve_gp / _gpbb / _upn, per column.
 * X holds k columns of N floats (column c at X + c*N, host or device):
 * x^(0) on entry, x* on return.  infos: nullable HOST array of k records
 * (phi is not evaluated: NaN).  Each column stops on its own test; a stopped
 * column is masked out of the later passes.  The row split of the two
 * projections (lanes per row / column) is opts->sweep_lanes, or chosen by
 * timing at the first sweep on a system of this shape (see tvr_solve_opts);
 * infos report it.  Synchronises `stream`.
 * Returns TVR_OK if every column converged, else the first error status of a
 * column, else TVR_NOT_CONVERGED.  Not an entry of the paper: a batching of
 * its methods over alpha.
 */
TVR_API int tvr_solve_sweep(const tvr_system *sys, int32_t method, const float *b,
                            const double *alphas, int32_t k, double tau, double eps,
                            const tvr_solve_opts *opts, float *X, tvr_solve_info *infos,
                            void *stream);

/*
 * Kernel timing for measurement: bits 0-3 of `enable` select the kernel kinds
 * to time (0 = off, 1 = forward only, 15 = all); bits 8-15 give a sampling
 * stride for solves replayed as pass graphs (time every stride-th pass of a
 * batch; 0 or 1 = every pass).  While enabled, the library records a CUDA
 * event pair on the launch stream around every selected kernel (event nodes
 * inside a pass graph, so graph replays are timed too) and counts only the
 * launches that did work.  Kinds: 0 = forward projection (in a solve, the
 * trial kernel, which also carries the projected step over the voxels),
 * 1 = back projection (CSC + TV), 2 = step (no separate launches: fused into
 * kind 0, kept for the array layout), 3 = UPN extrapolation.
 * tvr_profile_read synchronises the events and returns, per kind, the number
 * of timed launches and their total time in milliseconds (host outputs), then
 * resets the counters.  Event nodes around a kernel break the programmatic
 * launch overlap at that point, so timed passes run slightly slower.
 */
TVR_API int tvr_profile_enable(tvr_system *sys, int32_t enable);
TVR_API int tvr_profile_read(tvr_system *sys, int64_t counts[4], double total_ms[4]);

/* Name of a status code. */
TVR_API const char *tvr_status_str(int status);

/* Message describing the calling thread's most recent error (never NULL). */
TVR_API const char *tvr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TVR_H */
