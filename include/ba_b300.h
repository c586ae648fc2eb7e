/* ba_b300.h -- C ABI of the B300 (sm_103a) Levenberg-Marquardt bundle adjuster
 * with metric depth priors and dynamic parameter extraction
 * (InstantSfM, arXiv 2510.13310: Sec. 3.2 BA objective, Sec. 3.3 LM,
 *  Sec. 4.1 depth-constrained Jacobian, Sec. 4.2 dynamic parameter extraction).
 *
 * One LM iteration runs five steps, all as CUDA kernels on one GPU:
 *  (a) per-observation reprojection + depth residuals and Jacobian blocks
 *      (Eq. BA objective with depth, Sec. 4.1),
 *  (b) normal-equation blocks U (camera), V (point), W (camera-point), the
 *      Schur right-hand side and the block-Jacobi preconditioner (Eq. LM),
 *  (c) dynamic active-set extraction: validity (z > min_depth, in image),
 *      optional sticky residual drop, threshold peeling, ascending ranks
 *      (Sec. 4.2 steps 1-2, Eqs. O_valid, C_active, P_active, rank),
 *  (d) block-Jacobi PCG on the reduced camera system, point back-substitution
 *      and scatter of the compact update (Sec. 4.2 step 3),
 *  (e) Marquardt damping and the gain-ratio accept/reject (Sec. 3.3).
 *
 * Camera parameters (9 doubles, row-major [C][9]): axis-angle w (world-to-camera
 * rotation), translation t, focal f, radial k1, k2.  A point X projects as
 * P = Exp(w) X + t (+z forward), (x, y) = (P_x, P_y) / P_z, rr = x^2 + y^2,
 * pixel = f (1 + k1 rr + k2 rr^2) (x, y) + (cx, cy).  Rotation updates are
 * left-multiplicative: w <- Log(Exp(dw) Exp(w)).
 *
 * Pointers.  Every array argument may be a host pointer (pageable or pinned)
 * or a device pointer of the problem's device; copies use unified addressing
 * (cudaMemcpyDefault).  The library copies inputs into buffers it owns; the
 * caller keeps ownership of everything it passes.  Outputs are written to
 * caller-owned memory.  Calls are ordered on the stream given to ba_create and
 * return once their results are in the destination.  Errors are returned as a
 * ba_status, never thrown or trapped; ba_last_error() gives a message.
 * A problem handle must not be used from two threads at once.
 */
#ifndef BA_B300_H
#define BA_B300_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1,   /* bad size, index, option or non-finite input */
  BA_ERR_CUDA = 2,          /* a CUDA call failed; see ba_last_error() */
  BA_ERR_OOM = 3,           /* device allocation failed */
  BA_ERR_NOT_CONVERGED = 4, /* PCG hit its iteration cap; the step is still usable */
  BA_ERR_NONFINITE = 5,     /* non-finite cost or step: the step was rejected */
  BA_ERR_STATE = 6,         /* call out of order (e.g. backward before a solve) */
  BA_ERR_TIMEOUT = 7        /* an in-kernel grid barrier gave up waiting */
} ba_status;

/* Arithmetic of steps (a)-(e).  The tensor-core form of the dense reduced camera
 * system (FP32 with the TF32 blocked Cholesky) is not a third precision here: it
 * is BA_FP32 with solver = BA_SOLVER_DENSE. */
typedef enum { BA_FP64 = 0, BA_FP32 = 1 } ba_precision;

typedef struct {
  ba_precision precision;      /* BA_FP64: every step in FP64.  BA_FP32: (a),(b),(d) in FP32;
                                  the cost in double-float arithmetic (FP32 pairs, ~48-bit
                                  significand; 1e-12 relative to the FP64 cost), the gain
                                  ratio in FP64, the extraction predicate with FP64 semantics
                                  (decisions within rounding of a threshold are re-evaluated
                                  in FP64) */
  int img_w, img_h;            /* image size for the in-frustum test (640, 480) */
  double cx, cy;               /* principal point, held fixed (320, 240) */
  double huber_delta;          /* Huber threshold on |r| in px (1.0); <= 0: squared loss */
  double depth_weight;         /* lambda_d: weight of the squared inverse-depth residual (1.0) */
  double invalid_depth_weight; /* weight of the zero-target depth residual of observations
                                  without a prior (Sec. 4.1 sentinel); default 0 */
  double min_depth;            /* validity: camera-frame z > min_depth (0.1) */
  int extract_every;           /* residual drop at iterations e, 2e, ...; 0 = never */
  double drop_residual_px;     /* drop observations with |r_uv| > this; <= 0 disables */
  int min_cam_obs, min_pt_obs; /* extraction thresholds (1, 1) */
  double lambda0;              /* initial damping (1e-4) */
  double pcg_rel_tol;          /* PCG stop: |r| <= tol |b| (1e-6) */
  int pcg_max_iters;           /* PCG cap (500) */
  const int32_t* fixed_cams;   /* host array of gauge cameras held constant ({0}) */
  int n_fixed;
  int solver;                  /* reduced camera system: BA_SOLVER_AUTO (explicit when
                                  9 x cameras <= 4608, else implicit), BA_SOLVER_IMPLICIT
                                  (matrix-free Schur matvec), BA_SOLVER_EXPLICIT (dense S
                                  formed per damping value, block-Jacobi PCG on it),
                                  BA_SOLVER_DENSE (FP32 only: S formed, factored by the
                                  tensor-core blocked Cholesky, CG preconditioned with
                                  that factor to pcg_rel_tol), BA_SOLVER_SPARSE (S formed
                                  as the 9x9 blocks of co-visible camera pairs only,
                                  block-Jacobi PCG with a block-row matvec: the sparse
                                  co-visibility regime).  AUTO above 4608 unknowns
                                  prices implicit, dense explicit and block-sparse per
                                  LM step from the problem's sizes and co-visible pairs */
  int extract_mode;            /* BA_EXTRACT_DYNAMIC: step (c) at the start of every iteration
                                  whose state changed (Sec. 4.2 steps 1-3).  BA_EXTRACT_ONCE:
                                  one-shot pruning, the alternative Sec. 4.2 argues against:
                                  validity and peeling at the first iteration only, the active
                                  set then frozen (no residual drops); ba_set_params and
                                  ba_set_state start a new run and extract again */
  int camera_model;            /* BA_CAMERA_RADIAL: [w, t, f, k1, k2], P = Exp(w) X + t with radial
                                  distortion (the workloads' camera).  BA_CAMERA_CENTRE: the
                                  parameterisation of Sec. 3.2 (camera centre, rotation, focal
                                  length, no distortion) in the same nine slots [w, c, f, k1, k2]:
                                  P = Exp(w) (X - c); k1, k2 are ignored and left unchanged (the
                                  paper stores the rotation as a quaternion; the axis-angle slots
                                  hold the same rotation, and the update is the same left
                                  increment).  Every solver and ba_backward support both
                                  models; under BA_CAMERA_CENTRE the solve holds the k1, k2
                                  unknowns with a unit diagonal (they stay zero). */
} ba_options;

enum { BA_SOLVER_AUTO = 0, BA_SOLVER_IMPLICIT = 1, BA_SOLVER_EXPLICIT = 2, BA_SOLVER_DENSE = 3,
       BA_SOLVER_SPARSE = 4 };
enum { BA_EXTRACT_DYNAMIC = 0, BA_EXTRACT_ONCE = 1 };
enum { BA_CAMERA_RADIAL = 0, BA_CAMERA_CENTRE = 1 };

typedef struct {
  double cost;        /* F(x) = 1/2 sum rho(|r_k|^2) over the iteration's active set */
  double rmse_px;     /* reprojection RMSE over the active set */
  double lambda;      /* damping used by this iteration's solve */
  double gain;        /* (F(x) - F(x + dx)) / predicted decrease */
  double pred_decrease;
  double cand_cost;   /* F(x + dx) over the same active set */
  int accepted;
  int pcg_iters;
  double pcg_rel_res;
  int64_t n_cam_act, n_pt_act, n_obs_act;
  float ms[8];        /* device time per phase: [0] extract, [1] linearize, [2] Schur terms
                         (for the explicit system the formation of S^ runs concurrently on the
                         main stream and [2] ends with the Schur-diagonal chain on a side stream),
                         [3] solve (d) from there, [4] the PCG kernel launch alone (inside [3]),
                         [5] candidate + evaluation, [6] total; [7] the co-visibility
                         product kernel alone (explicit system) */
} ba_iter_info;

typedef struct ba_problem ba_problem;

/* Fill *o with the defaults listed above (FP32, camera 0 fixed). */
void ba_default_options(ba_options* o);

/* Create a problem: cams [C][9], pts [P][3], obs_cam/obs_pt [N] (int32 indices),
 * obs_uv [N][2] pixels, depth [N] metric depth prior (<= 0 or NaN: none).
 * These are the unknowns and measurements of the BA objective with depth
 * (Sec. 3.2, Eq. BA objective; Sec. 4.1, depth residual with the mask m = 1 when
 * a prior is given): the parameter vector x = [c; p] and the observation set
 * from which Sec. 4.2 step 1 builds O_valid at every iteration.
 * Checks index ranges, finiteness and duplicate (camera, point) pairs on the
 * host (BA_ERR_INVALID_ARG).  Limits: N < 2^30, at most 256 observations per
 * point.  stream: a cudaStream_t (NULL = legacy default stream).  The problem
 * lives on the device current at the call.  Input arrays may be host or device
 * memory (host arrays are read in place); the call returns with the device idle.
 * The observation orderings are built on host threads (the hardware threads, at
 * most 32; the environment variable BA_HOST_THREADS overrides); the result does
 * not depend on the thread count. */
ba_status ba_create(const ba_options* opts, void* stream, int64_t n_cams, const double* cams,
                    int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                    const int32_t* obs_pt, const double* obs_uv, const double* depth,
                    ba_problem** out);

/* One LM iteration, steps (c) -> (a) -> (b) -> (d) -> (e).  info may be NULL.
 * Returns BA_ERR_NOT_CONVERGED when PCG hit its cap (the iteration still ran). */
ba_status ba_lm_step(ba_problem* pb, ba_iter_info* info);

/* Up to max_iters LM iterations (Sec. 3.3: the LM loop; each iteration is one
 * ba_lm_step); log has max_iters entries or is NULL.  Stops early only on an
 * error other than BA_ERR_NOT_CONVERGED; *n_done (nullable) gets the count. */
ba_status ba_solve(ba_problem* pb, int max_iters, ba_iter_info* log, int* n_done);

/* Current parameters, cams [C][9] and pts [P][3]: the full arrays c and p of
 * Sec. 4.2, inactive entries unchanged since they left the active set (step 3). */
ba_status ba_get_params(ba_problem* pb, double* cams, double* pts);

/* Replace the full parameter arrays c and p (Sec. 4.2); the next step re-runs
 * the validity check and extraction (step 1) and re-linearises. */
ba_status ba_set_params(ba_problem* pb, const double* cams, const double* pts);

/* Checkpoint and resume of an LM run.  The state is everything later iterations
 * depend on: the FP64 parameters, the damping lambda and nu, the iteration count
 * (which schedules the residual drop) and the sticky drop bits.  ba_get_state
 * with blob == NULL stores the size in *bytes; otherwise it writes *bytes bytes
 * (host memory) or fails with BA_ERR_INVALID_ARG if *bytes is too small.
 * ba_set_state restores a blob into a problem created from the same
 * observations (sizes, index arrays, precision; checked through a hash) and
 * re-extracts at the next step; continuing from a restored state repeats the
 * uninterrupted run bit for bit (every reduction has a fixed order). */
ba_status ba_get_state(ba_problem* pb, void* blob, size_t* bytes);
ba_status ba_set_state(ba_problem* pb, const void* blob, size_t bytes);

/* Active sets of the latest extraction (Sec. 4.2 step 2).  Masks are 0/1 bytes;
 * obs_mask is in the input observation order; cam_rank is the position among
 * active non-gauge cameras, pt_rank among active points, -1 otherwise.
 * Any output may be NULL. */
ba_status ba_get_active(ba_problem* pb, uint8_t* cam_mask, uint8_t* pt_mask, uint8_t* obs_mask,
                        int32_t* cam_rank, int32_t* pt_rank);

/* Run step (c) now on the current parameters (validity, optional residual drop
 * when drop != 0, peeling, ranks).  n_rounds (nullable) gets the peel rounds. */
ba_status ba_extract(ba_problem* pb, int drop, int* n_rounds);

/* Run steps (a)-(b) at the current parameters and active set and copy out FP64
 * blocks in full indexing: U [C][81], V [P][9], gc [C][9], gp [P][3] (rows of
 * inactive entries are zero) and W [N][27] (9x3 row-major, input order; zero
 * for inactive observations).  Any output may be NULL. */
ba_status ba_linearize(ba_problem* pb, double* U, double* V, double* W, double* gc, double* gp);

/* Step (d) for damping lambda at the current linearisation: the step in full
 * indexing, dc [C][9] and dp [P][3] (zero for inactive and gauge entries).
 * info (nullable) receives pcg_iters, pcg_rel_res and pred_decrease. */
ba_status ba_solve_damped(ba_problem* pb, double lambda, double* dc, double* dp,
                          ba_iter_info* info);

/* Cost 1/2 sum rho and RMSE of the given parameters over the current active
 * set (NULL cams/pts: the current parameters); FP64 for BA_FP64 problems,
 * double-float for BA_FP32 problems (see ba_options.precision). */
ba_status ba_eval_cost(ba_problem* pb, const double* cams, const double* pts, double* cost,
                       double* rmse_px);

/* Implicit-adjoint gradients at the current state (implicit function theorem on
 * the stationarity of Sec. 3.3's normal equations): with the active set of the
 * latest extraction and the IRLS weights frozen, solve H mu = a with the
 * undamped Gauss-Newton matrix H through the Schur complement (the LM step's
 * solver at lambda = 0, PCG to pcg_rel_tol), then per active observation
 *   dL/du_k = rho'_k (J_k mu)_0,  dL/dv_k = rho'_k (J_k mu)_1,
 *   dL/dd_k = -rho'_k sqrt(w_k) (J_k mu)_2 / d_k^2  (zero without a prior).
 * dL_dcams [C][9] and dL_dpts [P][3] are the loss gradient in the stored
 * parameters; a is that gradient in the LM update's coordinates: the rotation
 * block is Jl(w)^-T dL/dw (inverse left Jacobian of SO(3)), gauge and inactive
 * entries are dropped.  Outputs: dL_duv [N][2], dL_ddepth [N] in the input
 * order, zero for inactive observations.  Gradients with respect to the initial
 * parameters are zero (not returned).  The next LM step re-linearises.
 * BA_FP32 problems refine mu four times against the FP64 residual a - H mu (H
 * from the FP64 state), each correction solved with the same FP32 solver; the
 * corrections reuse the formed reduced camera system (explicit and block-sparse
 * solvers) or its tensor-core factor (dense solver), and mu and the outputs are
 * formed in FP64.  The first ba_backward of an FP32 problem allocates the
 * refinement's buffers (about 24 N + 72 P + 144 C bytes of device memory). 
 * Errors: BA_ERR_NONFINITE if the undamped system is singular, BA_ERR_NOT_CONVERGED
 * if PCG hit pcg_max_iters (outputs still written). */
ba_status ba_backward(ba_problem* pb, const double* dL_dcams, const double* dL_dpts,
                      double* dL_duv, double* dL_ddepth);

/* FP64 cost of a state without allocating device memory.  The paper has no
 * counterpart: this is an interface for callers that cannot call cudaMalloc,
 * such as code running under a framework that owns all device memory (its
 * allocator accounts for every byte, or the budget is fixed at start-up), or
 * latency-critical code that must avoid the device-wide synchronisation an
 * allocation can cause.  Returns on the stream (asynchronously)
 * out[0] = 1/2 sum rho(|r_k|^2), out[1] = reprojection RMSE, out[2] = number of
 * observations counted, over observations with obs_mask[k] != 0 (NULL: all),
 * in the input order; the camera model (opts->camera_model), Huber loss, depth
 * residual and weights are those of ba_lm_step, taken from opts (precision,
 * solver and extraction fields are ignored).  Observations whose indices are out of range are skipped.
 * Every array (inputs and out) must be readable/writable by kernels of the
 * current device: device memory of that device, managed memory, or mapped
 * page-locked host memory passed as its device alias (the same address under
 * unified addressing); anything else is rejected (BA_ERR_INVALID_ARG).  Sizes
 * are not checked against the arrays: each must hold its stated count.
 * Scratch is a fixed device array in the library (about 0.55 MB per device
 * that loads it, held until exit): n_cams above 4096 is rejected with
 * BA_ERR_INVALID_ARG.  The first call on a device looks that array up
 * (cudaGetSymbolAddress) and keeps its address for the life of the process;
 * make it before any stream capture, and do not call this after a reset of the
 * device (cudaDeviceReset) in the same process.  Every call
 * shares the array, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race; order them on one stream.  Nothing in the scratch
 * needs clearing: each call writes every entry it reads. */
ba_status ba_eval_cost_noalloc(const ba_options* opts, void* stream, int64_t n_cams,
                               const double* cams, int64_t n_pts, const double* pts,
                               int64_t n_obs, const int32_t* obs_cam, const int32_t* obs_pt,
                               const double* obs_uv, const double* depth,
                               const uint8_t* obs_mask, double* out);

/* ---------------------------------------------------------------------------
 * Depth-constrained global positioning (GP), the stage before BA (Sec. 3.1,
 * Eq. GP objective; Sec. 4.1, GP paragraph), on the same LM (Sec. 3.3, Eq. LM).
 *
 * Unknowns: camera centres t [C][3] (rotations are known and held), points
 * X [P][3] and one scale s_k per observation; residual u_k = v_k - s_k (X_j - t_i)
 * for observation k of point j in camera i, v_k the unit ray from the camera
 * centre toward the feature in the world frame; cost F = 1/2 sum rho(|u_k|^2)
 * with rho Huber (threshold huber_delta on |u|).  An observation with a metric
 * depth d_k (the distance along its ray, > 0 and finite) has its scale pinned,
 * s_k = 1/d_k, and removed from the unknowns; the others keep a free scale,
 * compacted by its rank among the free observations (ascending input order).
 * Each LM step eliminates the free scales and the points exactly and solves the
 * dense reduced centre system (order 3 x free cameras) by block-Jacobi PCG or the
 * tensor-core Cholesky-preconditioned CG (ba_gp_options.solver); FP32
 * arithmetic, the cost and gain ratio in FP64.
 * Gauge: the centres of fixed_cams are held; the metric scale comes from the
 * pinned scales (without any, it is left to the damping).
 * ------------------------------------------------------------------------- */
typedef struct {
  double huber_delta;          /* Huber threshold on |u| (0.1); <= 0: squared loss */
  double lambda0;              /* initial damping (1e-4) */
  double pcg_rel_tol;          /* CG stop on the centre system: |r| <= tol |b| (1e-6) */
  int pcg_max_iters;           /* CG cap (500) */
  const int32_t* fixed_cams;   /* host array of gauge cameras ({0}) */
  int n_fixed;
  int solver;                  /* centre system: BA_SOLVER_AUTO or BA_SOLVER_EXPLICIT (block-Jacobi
                                  PCG, three cameras per 9x9 preconditioner block, the explicit
                                  PCG kernel of BA) or BA_SOLVER_DENSE (tensor-core Cholesky
                                  preconditioned CG) */
} ba_gp_options;

typedef struct ba_gp_problem ba_gp_problem;

/* Fill *o with the defaults listed above. */
void ba_gp_default_options(ba_gp_options* o);

/* Create a GP problem: centres [C][3], pts [P][3], obs_cam/obs_pt [N] (int32),
 * rays [N][3], depth [N] (metric distance along the ray; <= 0 or NaN: none, the
 * scale is free), scales0 [N] initial scales of the free observations (NULL: 1;
 * entries of pinned observations are ignored).  Host or device pointers; the
 * library copies them.  Errors: BA_ERR_INVALID_ARG for bad sizes (N < 2^30),
 * indices, duplicate (camera, point) pairs, more than 256 observations per point
 * or non-finite centres, points, rays or scales. */
ba_status ba_gp_create(const ba_gp_options* opts, void* stream, int64_t n_cams, const double* centres,
                       int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                       const int32_t* obs_pt, const double* rays, const double* depth, const double* scales0,
                       ba_gp_problem** out);

/* One LM iteration (Sec. 3.3): linearise, eliminate the free scales and the
 * points, solve the centre system, back-substitute, evaluate the candidate and
 * accept or reject it (gain > 1e-3; Nielsen damping update).  info (nullable):
 * cost, rms (sqrt of the mean |u|^2, in ray units), lambda, gain, the CG
 * iterations; n_cam_act = free cameras, n_pt_act = points, n_obs_act = free scales. */
ba_status ba_gp_lm_step(ba_gp_problem* pb, ba_iter_info* info);

/* Up to max_iters LM iterations; log has max_iters entries or is NULL. */
ba_status ba_gp_solve(ba_gp_problem* pb, int max_iters, ba_iter_info* log, int* n_done);

/* Current centres [C][3], points [P][3] and scales [N] (input order; pinned
 * observations report 1/d).  Any output may be NULL. */
ba_status ba_gp_get_params(ba_gp_problem* pb, double* centres, double* pts, double* scales);

/* The free/pinned partition of Sec. 4.1: free_rank [N] = rank among the free
 * observations, -1 for pinned ones; *n_free = their number.  Either may be NULL. */
ba_status ba_gp_get_free(ba_gp_problem* pb, int32_t* free_rank, int64_t* n_free);

/* The damped step at damping lambda from the current state, in full indexing:
 * dt [C][3] (zero for fixed cameras and cameras without observations), dX [P][3],
 * ds [N] (zero for pinned observations); info (nullable) gets pred_decrease and
 * the CG iterations.  The state is not changed. */
ba_status ba_gp_solve_damped(ba_gp_problem* pb, double lambda, double* dt, double* dX, double* ds,
                             ba_iter_info* info);

/* FP64 cost F and rms of the current state. */
ba_status ba_gp_eval_cost(ba_gp_problem* pb, double* cost, double* rms);

/* Number of this library's kernels launched for the problem since creation. */
int64_t ba_gp_kernel_launches(const ba_gp_problem* pb);

/* Free a GP problem (the paper has no counterpart: resource management). */
void ba_gp_destroy(ba_gp_problem* pb);

/* C = alpha A B^T + beta C on the tensor cores (tcgen05.mma kind::tf32: FP32
 * operands enter as TF32, FP32 accumulation).  The dense-system factorisation's
 * building block, exposed on its own.  A [M][lda], B [N][ldb], C [M][ldc]
 * row-major device pointers of the current device; lda, ldb multiples of 4 and
 * A, B 16-byte aligned (tensor-map rules); M, N, K < 2^31.  Ordered on stream;
 * returns after completion. */
ba_status ba_tc_gemm_nt(void* stream, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float beta, float* C, int64_t ldc);

/* Blocked Cholesky A = L L^T of an n x n symmetric positive definite FP32 matrix
 * (lower triangle of A read; host or device pointers, row-major) on the tensor
 * cores: 128 x 128 tiles, diagonal tiles factored and inverted in FP32, the
 * off-diagonal solves and the trailing updates as TF32 products (so L carries
 * TF32-level error, ~1e-3 relative; it is meant as a preconditioner or for
 * refinement).  L [n][ldl] receives the lower factor with zeros above.  flags
 * (nullable): bit 32 = a pivot was not positive (BA_ERR_NONFINITE). n <= 65536. */
ba_status ba_dense_cholesky(void* stream, int64_t n, const float* A, int64_t lda, float* L, int64_t ldl,
                            int* flags);

/* Diagnostic of failure detection: launches one block that waits, with the
 * given limit (ms, at most 5000), on a device flag that nothing sets, using
 * the bounded wait of the library's cross-block kernels.  Returns
 * BA_ERR_TIMEOUT (the expected outcome: the wait gave up, the error was reported
 * through device memory and the context stays usable), or BA_ERR_CUDA. */
ba_status ba_selftest_wait_timeout(void* stream, double timeout_ms);

/* Diagnostic of ba_create's observation layout: builds it on the device (as
 * ba_create does) and with the host reference builder, from host arrays (the
 * arguments of ba_create; depth is not needed), and compares every array:
 * *mismatch = 0 when they are identical bit for bit, else a bitmask: 1 orders,
 * 2 offsets, 4 tile descriptors, 8 tile records, 16 camera chunks, 32 structure
 * hash, 64 co-visibility runs (with_covis != 0), 128 the two disagree on
 * rejecting the input.  Invalid input is not an error here (both builders must
 * reject it alike).  Returns BA_OK, BA_ERR_INVALID_ARG (bad arguments),
 * BA_ERR_OOM or BA_ERR_CUDA. */
ba_status ba_selftest_layout(int64_t n_cams, const double* cams, int64_t n_pts, const double* pts, int64_t n_obs,
                             const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv, int with_covis,
                             int* mismatch);

/* Number of this library's kernels launched since creation (counts launches). */
int64_t ba_kernel_launches(const ba_problem* pb);

/* Index checks of the debug build.  A library compiled with -DBA_DEBUG_BOUNDS
 * (libba_b300_debug.so) checks every index it loads from the observation layout
 * or the co-visibility runs before the gather that uses it; a failed check
 * records the kernel site and the index (the first failure per source file) and
 * the access uses index 0 instead, so a corrupted layout cannot read or write
 * out of bounds.  This call reports the first recorded failure: *site = -1 for a
 * release build (no checks; no CUDA call is made), 0 when no check failed, else
 * the site number (>= 1) with the failing index in *index; reset != 0 clears
 * the records.  Synchronises with the device.  Returns BA_OK or BA_ERR_CUDA. */
ba_status ba_debug_bounds(int reset, int64_t* site, int64_t* index);

/* The reduced-camera-system solver the problem resolved to at creation:
 * BA_SOLVER_IMPLICIT, BA_SOLVER_EXPLICIT, BA_SOLVER_DENSE or BA_SOLVER_SPARSE
 * (0 for a NULL handle). */
int ba_solver_kind(const ba_problem* pb);

/* Placement of the explicit solver's working set, fixed at creation (all
 * outputs optional, set to 0 for other solvers or a NULL handle):
 * *rows_in_smem = 1 when each block keeps its rows of S^ in shared memory
 * (S^ is read from device memory once per solve), 0 when the rows are streamed
 * from device memory on every matvec; *vecs_in_smem = 1 when the PCG vectors sit
 * in shared memory, 0 when they sit in per-block device scratch; *grid = blocks
 * of the persistent PCG launch. */
void ba_explicit_layout(const ba_problem* pb, int* rows_in_smem, int* vecs_in_smem, int* grid);

/* The kernel that forms the off-diagonal blocks of an explicit reduced camera
 * system (Eq. LM, Schur form), chosen at creation from the co-visibility runs:
 * 1 one warp per camera pair (k_form_S_runs), 2 one lane per camera pair
 * (k_form_S_lanes: FP64 with very many short runs), 3 camera-owned formation
 * (k_form_S_cam: FP32 with very many short runs), 4 one warp per camera pair from
 * observation records (k_form_S_rec: FP32 otherwise; the environment variable
 * BA_FORM_RECORDS=0, read by ba_create, selects kernel 1 instead); 0 for the
 * implicit solver or a NULL handle. */
int ba_formation_kernel(const ba_problem* pb);

/* Free a problem (the paper has no counterpart: resource management of this
 * interface).  Its device buffers go to a process-wide cache that later
 * ba_create calls draw from (no new device mappings when problems of similar
 * sizes are created repeatedly), and ba_create's temporary layout scratch comes
 * from a pool that keeps its memory; ba_release_cache returns every cached buffer
 * and the pool's unused memory to the driver.  Setting BA_NO_ALLOC_CACHE=1 in the
 * environment disables the buffer cache. */
void ba_destroy(ba_problem* pb);
void ba_release_cache(void);
const char* ba_status_string(ba_status s);
const char* ba_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
