/*
 * pet_gb300.h -- C ABI of the GB300 (sm_103a) library for the subset-gradient path
 * of RDP-regularised PET reconstruction with preconditioned SGD / SAGA / SVRG
 * (Ehrhardt, Kereta, Schramm, "Fast PET Reconstruction with Variance Reduction and
 * Prior-Aware Preconditioning").
 *
 * Conventions for every entry point
 *   - Pointers named x, q, g, out, D, grad, hdiag, y, r, mu, sens_lor, kappa, ref are
 *     DEVICE pointers owned by the caller; the library never frees them.  Pointers to
 *     pet_geometry / option structs and the z1/z2 / order / pc_iters arrays are HOST
 *     pointers read during the call only.
 *   - Images are float32, layout [nz][ny][nx] (x fastest); voxel (ix,iy,iz) has centre
 *     ((ix-(nx-1)/2) dx, (iy-(ny-1)/2) dy, (iz-(nz-1)/2) dz) in mm.
 *   - Sinograms are laid out [view][plane][radial][tof]; a subset's compact sinogram
 *     is [j][plane][radial][tof] over its views v = s, s+n, s+2n, ... (Sec. 3.1: subsets
 *     are every n-th view).  Per-LOR arrays (sens_lor, m) drop the tof axis.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *     work is enqueued asynchronously on it; results are valid once the stream has
 *     reached that point.  Scalar results (double*) are device pointers too.
 *   - Every call returns a pet_status; no exception or abort crosses the ABI.
 *     Argument errors are detected on the host before anything is enqueued.  A data
 *     infeasibility seen by a kernel (ybar <= 0 where y > 0) is recorded in a device
 *     error word and reported by pet_plan_check().
 */
#ifndef PET_GB300_H
#define PET_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PET_OK = 0,
  PET_ERR_ARG = 1,         /* null pointer, out-of-range index or option */
  PET_ERR_SHAPE = 2,       /* geometry that the projector cannot represent */
  PET_ERR_INFEASIBLE = 3,  /* ybar <= 0 with y > 0: KL term infinite (Sec. 1.2) */
  PET_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  PET_ERR_CUDA = 5,        /* a CUDA runtime call failed */
  PET_ERR_UNSUPPORTED = 6, /* valid but not implemented (e.g. > 32 TOF bins) */
  PET_ERR_STATE = 7,       /* call order violated (e.g. data not set) */
  PET_ERR_NOMEM = 8        /* device allocation failed */
} pet_status;

typedef enum { PET_Y_U16 = 0, PET_Y_U32 = 1, PET_Y_F32 = 2 } pet_ytype;

typedef struct pet_plan pet_plan;
typedef struct pet_solver pet_solver;

/* Scanner and image description (forward model of Sec. 1.1 eq. 1; simulated
 * cylindrical scanner of Sec. 3.1).  View v has angle v*pi/nview; radial bin r sits at
 * signed distance (r-(nrad-1)/2)*drad from the axis; plane p joins axial positions
 * z1[p] (endpoint 1) and z2[p] (endpoint 2) on a cylinder of radius rdet (mm).
 * ntof <= 1 means non-TOF; otherwise bin b of width tof_bin (mm) is centred at
 * (b-(ntof-1)/2)*tof_bin from the LOR midpoint toward endpoint 2 and the timing
 * kernel is a Gaussian of std tof_sigma (mm) truncated at 3 sigma.  nsubsets is the
 * number n of view subsets (eq. 2).  res_fwhm > 0 adds the image-space resolution
 * model of Sec. 3.1: the system matrix becomes P G with G a separable Gaussian of
 * that FWHM (mm), sampled at the voxel offsets |k| <= ceil(3 sigma / delta) per axis
 * (at most 31), normalised to unit sum, zero outside the image, no axial pass when
 * nz = 1; the attenuation factors use P alone.  0 = no resolution model. */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  int nrad, nview, nplane, ntof;
  double drad, rdet;
  const double *z1, *z2;
  double tof_sigma, tof_bin;
  int nsubsets;
  double res_fwhm;
} pet_geometry;

/* Relative difference prior (eq. 3) parameters.  Outputs of pet_rdp are scaled by
 * `scale` (pass beta for beta*S, beta/n for the per-subset share of eq. 5).  Weights:
 * w_ij = min(dx,dy,dz) / |offset (mm)| over the 26-neighbourhood (8 in-plane when
 * nz == 1); neighbours outside the image are omitted.  kappa: device image or NULL. */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  float gamma, eps, scale;
  const float *kappa;
} pet_rdp_params;

/* ---------------------------------------------------------------- plan */

/* Validates the geometry (every LOR must have |s| < rdet and an in-plane driving
 * axis), builds the per-view / per-LOR / per-plane tables on the current device and
 * allocates the plan's scratch.  Returns PET_ERR_SHAPE or PET_ERR_UNSUPPORTED for a
 * geometry the projector cannot represent, PET_ERR_NOMEM on allocation failure. */
pet_status pet_plan_create(const pet_geometry *geom, pet_plan **out);
void pet_plan_destroy(pet_plan *plan);

/* Binds the measured data (borrowed: y [V][P][R][T] of type yt, r [V][P][R][T] float32)
 * and computes the multiplicative factors m = sens_lor * exp(-P mu) per LOR (Sec. 1.1:
 * A includes sensitivities and attenuation; mu in 1/mm, NULL = none; sens_lor NULL =
 * 1) and the sensitivity images A^T 1 and A_s^T 1 (Sec. 2.3).  The caller keeps y and
 * r alive while the plan uses them.  Synchronises `stream` before returning. */
pet_status pet_plan_set_data(pet_plan *plan, const void *y, pet_ytype yt, const float *r,
                             const float *mu, const float *sens_lor, void *stream);

/* Rebinds the counts and background only (borrowed, same layout and types as in
 * pet_plan_set_data), keeping the multiplicative factors and sensitivity images: the
 * next frame of a dynamic or gated acquisition on the same scanner and attenuation map
 * (Sec. 1.1: m and A^T 1 depend on neither y nor r).  No device work; calls issued after
 * it read the new arrays.  Solvers on the plan see them from their next iteration; their
 * gradient tables (SAGA, SVRG) still hold gradients of the old data until
 * pet_solver_set_image restarts them.  PET_ERR_STATE before pet_plan_set_data. */
pet_status pet_plan_set_counts(pet_plan *plan, const void *y, pet_ytype yt, const float *r);

/* Copies `bytes` from page-locked host memory (cudaHostAlloc / cudaHostRegister, or a
 * pinned torch tensor) into device memory with a kernel whose threads load the host
 * memory through the unified address space, 16 bytes at a time with several loads in
 * flight (the ingest of a frame's counts and background before pet_plan_set_counts).
 * max_blocks bounds the grid (blocks of 512 threads; 0 = four per SM): a few blocks keep
 * most SMs free for kernels running beside the copy on another stream.  Both pointers
 * 16-byte aligned; src must be page-locked host memory and dst device memory of the
 * current device, max_blocks >= 0, else PET_ERR_ARG.  Asynchronous on `stream`; the
 * caller keeps src unchanged until the stream passes the copy. */
pet_status pet_copy_to_device(void *dst, const void *src, size_t bytes, int max_blocks, void *stream);

/* Number of views of subset s (s = -1: all views). */
pet_status pet_subset_size(const pet_plan *plan, int subset, int *nviews);

/* Multiplicative factors m [V][P][R] computed by pet_plan_set_data (device pointer
 * owned by the plan, valid until destroy). */
const float *pet_plan_mult(const pet_plan *plan);

/* Sensitivity image A_s^T 1 (s = -1: all views) owned by the plan. */
const float *pet_plan_sensitivity(const pet_plan *plan, int subset);

/* Launch shape of the fused subset-gradient kernel: planes per thread (LORs of one view
 * and radial bin on different planes share their in-plane sample positions: 1, 2 or 4
 * without TOF; also 1, 2 or 4 with TOF when a sample meets at most 8 TOF bins, i.e.
 * (6 sigma + w)/w <= 8 for bin width w, and ntof <= 16 (the windowed TOF kernel; the
 * planes of a thread then have equal axial slope and share their TOF weights); else 1)
 * and parts per
 * LOR (1, 2, 4, 8 or 16: interleaved sets of the driving planes of one LOR processed by
 * different threads; 16 only without TOF; 8 without TOF, with the windowed TOF kernel or
 * with 11 or 13 TOF bins; else up to 4).  0 selects the built-in heuristic.  Results are
 * the same up to FP32 summation order.  PET_ERR_ARG for an unsupported shape. */
pet_status pet_plan_set_grad_shape(pet_plan *plan, int planes_per_thread, int parts);

/* Autotuner: times every valid launch shape on four subsets spread over the views of the
 * bound data (a uniform image), keeps the fastest in the plan and returns it; also times the RDP stencil tile
 * (32 x 8 voxels x 2, 4 or 8 slices per block) on the plan's image and keeps the fastest
 * for the plan's prior evaluations (solvers, pet_objective_grad).  Uses plan scratch;
 * synchronises `stream`.  Requires pet_plan_set_data. */
pet_status pet_plan_autotune(pet_plan *plan, void *stream, int *planes_per_thread, int *parts);

/* RDP stencil tile of the plan's prior evaluations: 2, 4 or 8 slices per block of 32 x 8
 * voxels (0 = the default, 4).  Results are identical for every tile.  PET_ERR_ARG for
 * other values. */
pet_status pet_plan_set_rdp_tile(pet_plan *plan, int slices);

/* Reads and clears the device error word after synchronising `stream`: PET_OK or
 * PET_ERR_INFEASIBLE. */
pet_status pet_plan_check(pet_plan *plan, void *stream);

/* ---------------------------------------------------------------- operators */

/* out = A_s x (Joseph forward projection of subset s, TOF-weighted when ntof > 1,
 * times m), compact subset layout.  eq. 5 needs A_s x for f_s. */
pet_status pet_forward(pet_plan *plan, int subset, const float *x, float *out, void *stream);

/* g = A_s^T q (matched transpose of pet_forward; q in compact subset layout).
 * deterministic = 0: ray-driven scatter with atomics (summation order varies run to
 * run); 1: voxel-driven gather with compensated sums in a fixed order (bitwise
 * reproducible). */
pet_status pet_back(pet_plan *plan, int subset, const float *q, float *g, int deterministic,
                    void *stream);

/* Subset objective f_s(x) = D_s(x) + scale_prior * S(x) and its gradient (eq. 5):
 * g = A_s^T (1 - y/(A_s x + r)) [+ prior->scale * grad S(x)].  prior may be NULL (data
 * term only).  obj (device double, may be NULL) receives f_s(x) summed in FP64.
 * flags: PET_GRAD_DETERMINISTIC uses the deterministic backprojector;
 * PET_OBJ_ONLY skips the backprojection (g untouched; recompute mode).  s = -1: all views. */
#define PET_GRAD_DETERMINISTIC 1
#define PET_OBJ_ONLY 2
pet_status pet_objective_grad(pet_plan *plan, int subset, const float *x, float *g, double *obj,
                              const pet_rdp_params *prior, int flags, void *stream);

/* KL ratio from a stored forward projection ax = A_s x (compact subset layout, e.g. from
 * pet_forward): q = 1 - y/(ax + r) (em = 0; the derivative of d(s, y) in s, Sec. 1.2) or
 * q = y/(ax + r) (em = 1), and obj (device double, may be NULL) = sum of d(ax + r, y)
 * over the subset in FP64.  q may be NULL.  g = pet_back(q) then completes the data
 * gradient of eq. 5 without projecting again. */
pet_status pet_ratio(pet_plan *plan, int subset, const float *ax, float *q, double *obj, int em,
                     void *stream);

/* One OSEM sub-iteration on subset s (MLEM for nsubsets = 1), in place:
 * x <- x / (A_s^T 1) * A_s^T (y_s / (A_s x + r_s)); voxels with A_s^T 1 = 0 keep their
 * value (Sec. 3.1 initialises runs with one OSEM epoch). */
pet_status pet_em_update(pet_plan *plan, int subset, float *x, void *stream);

/* RDP gradient, Hessian diagonal and value (eq. 3, Appendix A.1), each scaled by
 * p->scale: grad = scale dS/dx, hdiag = scale d2S/dx2, val = scale S (FP64).  Any of
 * grad, hdiag, val may be NULL.  accumulate is a bit set: PET_RDP_ACC_GRAD adds into
 * grad instead of writing it; PET_RDP_ACC_VAL adds scale S to *val instead of writing
 * it (e.g. onto the KL value of pet_ratio, giving the subset objective of eq. 5). */
#define PET_RDP_ACC_GRAD 1
#define PET_RDP_ACC_VAL 2
pet_status pet_rdp(const pet_rdp_params *p, const float *x, float *grad, float *hdiag,
                   double *val, int accumulate, void *stream);

/* Allocation-free variant of pet_rdp (the paper has no counterpart; this exists for
 * callers that cannot allocate device memory while running, e.g. a service whose
 * device memory is fully reserved at start-up, or a host framework that forbids
 * allocations outside its own allocator).  Same arguments, outputs and errors as
 * pet_rdp, but the FP64 partial sums of the value live in a fixed array inside this
 * library (PET_RDP_STATIC_MAX_PARTIALS doubles, 512 KiB, held by every GPU that loads
 * the library until the process exits) and the call allocates nothing.
 *   - Images needing more than PET_RDP_STATIC_MAX_PARTIALS stencil blocks of 32x8x4
 *     voxels (more than about 67 million voxels) are rejected with
 *     PET_ERR_UNSUPPORTED when val is requested.
 *   - A call with val != NULL on a stream that is not being captured looks up the
 *     array's device address on the current device (so an address cached before a
 *     cudaDeviceReset is never reused); a call on a capturing stream reuses the address
 *     cached by an earlier call on that device and fails with PET_ERR_STATE if there
 *     was none.  So make the first call on each device before any stream capture, and
 *     after a cudaDeviceReset call once outside capture before capturing again.
 *   - All calls share the one array, which keeps the last call's contents.  Calls
 *     that overlap on the GPU (different streams without ordering) race on it. */
#define PET_RDP_STATIC_MAX_PARTIALS 65536
pet_status pet_rdp_static(const pet_rdp_params *p, const float *x, float *grad, float *hdiag,
                          double *val, int accumulate, void *stream);

/* Diagonal preconditioner of Sec. 2.3 with delta = delta_rel * max(x):
 * hdiag_betaS == NULL: D_MLEM = (x+delta)/A^T 1;
 * otherwise the harmonic form of eq. 8: (x+delta)/(A^T 1 + alpha hdiag_betaS (x+delta)).
 * Entries with a zero denominator are 0. */
pet_status pet_precond(pet_plan *plan, const float *x, const float *hdiag_betaS, float alpha,
                       float delta_rel, float *D, void *stream);

/* NRMSE of Sec. 3.1: sqrt(mean over mask of (x-ref)^2) / mean over bg of ref, FP64;
 * mask and bg are device uint8 images; out is a device double. */
pet_status pet_nrmse(const float *x, const float *ref, const uint8_t *mask, const uint8_t *bg,
                     size_t n, double *out, void *stream);

/* ---------------------------------------------------------------- solver */

typedef enum { PET_SGD = 0, PET_SAGA = 1, PET_SVRG = 2 } pet_algo;
typedef enum {
  PET_STEP_CONST = 0,  /* tau0 */
  PET_STEP_VANISH = 1, /* tau0 / (1 + eta k / n)          (Sec. 2.2) */
  PET_STEP_ALG1 = 2,   /* piecewise 3, 2, 1.5, 1, 0.5      (Table 1, ALG1) */
  PET_STEP_BB = 3,     /* short Barzilai-Borwein step at SVRG refreshes (Sec. 2.2), in the
                          metric of the preconditioner D: p'q / q'Dq */
  PET_STEP_ALG2 = 4    /* BB capped at 3 / 2.2 / 1         (Table 1, ALG2/3) */
} pet_step_rule;

/* Subset sampling rules (Sec. 2.4).  z_k is output number k (0-based) of the splitmix64
 * stream started at the solver's seed. */
typedef enum {
  PET_SAMPLE_PERM = 0,      /* uniformly at random without replacement: one Fisher-Yates
                               permutation per epoch, j = z mod (i + 1) for i = n-1..1 */
  PET_SAMPLE_REPLACE = 1,   /* uniformly at random with replacement: ((z_k >> 32) n) >> 32 */
  PET_SAMPLE_HM = 2,        /* Herman-Meyer order (mixed-radix digit reversal over the
                               ascending prime factors of n), the same every epoch */
  PET_SAMPLE_COFACTOR = 3,  /* cofactor order: generators g of Z_n ranked by distance to
                               0.3 n / 0.7 n (ties: smaller g); epoch e visits j g mod n with
                               the (e mod count)-th generator */
  PET_SAMPLE_IMPORTANCE = 4 /* SVRG only: p_i = ||grad f_i(xhat)|| / sum_j ||grad f_j(xhat)||
                               at each refresh; iteration k takes the smallest i with
                               (z_k >> 11) 2^-53 < p_0 + ... + p_i, drawn on the device, and
                               weights the correction by 1/p_i (unbiased) */
} pet_sampling;

/* Options of the preconditioned proximal stochastic gradient method (eq. 6) with
 * the SGD, SAGA (eq. 7) or SVRG (eq. 9, Algorithm 1) estimator. */
typedef struct {
  int algo;               /* pet_algo */
  int omega;              /* SVRG snapshot period in epochs (default 2, Sec. 2.1) */
  int step_rule;          /* pet_step_rule */
  double tau0, eta;       /* constant / vanishing parameters; BB start value */
  int precond_kind;       /* 0 D_MLEM, 1 harmonic (eq. 8) */
  double alpha;           /* harmonic weight */
  double delta_rel;       /* delta = delta_rel * max(x) at each preconditioner update */
  const long long *pc_iters; int n_pc; /* iterations that recompute D (Algorithm 1) */
  float beta, gamma, eps; /* RDP strength and shape (eq. 3, eq. 4) */
  const float *kappa;     /* device image or NULL */
  unsigned long long seed;/* subset order: splitmix64-driven Fisher-Yates per epoch */
  const int *order;       /* host, optional explicit subset per iteration (overrides seed) */
  long long norder;
  int use_graph;          /* capture each epoch in a CUDA graph */
  int deterministic;      /* deterministic backprojector */
  int sampling;           /* pet_sampling (an explicit order overrides it, except importance) */
  int low_memory;         /* SVRG without the [n][N] table (Sec. 2.1): each inner iteration
                             recomputes the subset gradient at the snapshot (two fused
                             gradients per iteration); the refresh computes the full data
                             gradient in one pass over all views */
  long long bb_until;     /* BB step recomputed only at refreshes k <= bb_until, then kept
                             (Table 1: ends of epochs 2, 4, 6 for ALG2/ALG3); 0 = every refresh */
} pet_solver_opts;

pet_status pet_solver_create(pet_plan *plan, const pet_solver_opts *opts, pet_solver **out);
void pet_solver_destroy(pet_solver *s);
/* Copies the start image (device) into the solver; resets iteration count and tables. */
pet_status pet_solver_set_image(pet_solver *s, const float *x, void *stream);
/* Device pointer to the current iterate (owned by the solver, valid until the next run). */
const float *pet_solver_image(const pet_solver *s);
/* Runs niter further iterations of eq. 6 (Algorithm 1 for SVRG). */
pet_status pet_solver_run(pet_solver *s, long long niter, void *stream);
/* Host copy of the stepsizes used so far (up to cap entries); returns the count. */
long long pet_solver_taus(const pet_solver *s, double *taus, long long cap);
long long pet_solver_iteration(const pet_solver *s);
/* Host copy of the subset used by each iteration so far (-1 at SVRG snapshot refreshes),
 * up to cap entries; returns the count.  Synchronises with the device. */
long long pet_solver_subsets(const pet_solver *s, int *subsets, long long cap);

/* ---------------------------------------------------------------- batches */

/* Many independent reconstructions advanced together (batched instances of uneven image
 * and sinogram sizes, betas and count levels).  Each solver keeps its own plan, data,
 * options and subset order; the batch runs windows of iters_per_graph iterations, each
 * iteration as one launch per phase for all instances (fused subset gradient, RDP
 * gradient, estimator + step + prox, accumulator clear), captured once in a CUDA graph and
 * replayed after uploading each window's per-solver subsets and iteration indices.  An
 * instance whose window contains a preconditioner update or an SVRG snapshot refresh (n
 * subset gradients and a step), and every instance in a final window shorter than
 * iters_per_graph, runs that window alone (one iteration at a time, exactly as
 * pet_solver_run); the batched launches then skip it.  Instances whose options have no
 * batched form (TOF plans, the deterministic backprojector, the table-free SVRG,
 * importance sampling, the resolution model) run alone in every window, with the same
 * results as pet_solver_run.  Solvers with a kappa image (eq. 3 weights) and without one
 * are batched together.  Requirements (else PET_ERR_UNSUPPORTED / PET_ERR_ARG): one
 * algorithm (SGD, SAGA or SVRG) for all, distinct plans (a plan's scratch serves one
 * solver at a time).  The solvers are borrowed. */
typedef struct pet_batch pet_batch;
pet_status pet_batch_create(pet_solver *const *solvers, int n, int iters_per_graph, pet_batch **out);
void pet_batch_destroy(pet_batch *b);
/* Runs niter iterations of every solver (each solver's iteration counter advances). */
pet_status pet_batch_run(pet_batch *b, long long niter, void *stream);
/* Launch shape of the batched fused gradient (planes per thread 1, 2 or 4; parts per
 * LOR 1, 2, 4 or 8) and its autotuner (times each shape on subset 0 of every solver, then
 * the batched RDP stencil tile of 2, 4 or 8 slices per block; synchronises stream). */
pet_status pet_batch_set_grad_shape(pet_batch *b, int planes_per_thread, int parts);
pet_status pet_batch_autotune(pet_batch *b, void *stream, int *planes_per_thread, int *parts);

/* Event timing of the fused subset-gradient kernel launched by the solver (the
 * dominant kernel of an iteration), recorded on the launching stream and inside
 * captured graphs.  Slots are unique within one SVRG outer loop (omega*n iterations)
 * or one SGD/SAGA epoch, so read the time at least once per outer loop / epoch.
 * pet_solver_kernel_time synchronises on the recorded events, returns the summed
 * duration (ms) and the number of launches since the previous call, and resets. */
pet_status pet_solver_profile(pet_solver *s, int enable);
pet_status pet_solver_kernel_time(pet_solver *s, double *total_ms, long long *launches);

/* Number of kernels this library has launched in the process so far (a replayed
 * epoch graph counts its kernel nodes). */
long long pet_launch_count(void);

const char *pet_status_str(pet_status st);

#ifdef __cplusplus
}
#endif
#endif
