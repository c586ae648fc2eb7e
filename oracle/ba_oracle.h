/* ba_oracle.h -- plain FP64 CPU reference for the depth-prior Levenberg-Marquardt
 * bundle adjustment with dynamic parameter extraction (InstantSfM, arXiv 2510.13310).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the oracle that the CUDA path is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the product path never does.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Every function follows the paper's equations step by step in FP64:
 *   - objective with Huber robustifier:         Eq. (BA objective), Sec. 3.2
 *   - metric depth residual 1/Depth - 1/d:       Sec. 4.1, Eq. (depth residual)
 *   - heterogeneous depth mask d~^-1 = m d^-1:    Sec. 4.1, Eq. (masked inverse depth)
 *   - LM normal equations with Marquardt scaling: Sec. 3.3, Eq. (LM)
 *   - validity check, unique active sets, rank remap, compacted solve, scatter:
 *                                                Sec. 4.2 steps 1)-3), Eqs. (O_valid), (C/P_active)
 * Readings of points the paper leaves open are listed beside each function.
 *
 * Camera: 9 doubles [w0 w1 w2 t0 t1 t2 f k1 k2], world-to-camera P = Exp(w) X + t,
 * +z forward, pixel = f (1 + k1 rr + k2 rr^2) (P_x/P_z, P_y/P_z) + (cx, cy).
 * Rotation increments are left-multiplicative: w <- Log(Exp(dw) Exp(w)).
 */
#ifndef BA_ORACLE_H
#define BA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n_cams, n_pts, n_obs;
  const int32_t* obs_cam;   /* [N] camera of each observation */
  const int32_t* obs_pt;    /* [N] point of each observation */
  const double* obs_uv;     /* [N][2] measured pixel */
  const double* depth;      /* [N] metric depth prior; <= 0 or NaN: none (m = 0) */
  const uint8_t* fixed;     /* [C] 1 = gauge camera (held constant) */
} oracle_problem;

typedef struct {
  int img_w, img_h;
  double cx, cy;
  double huber_delta;           /* <= 0: plain squared loss */
  double depth_weight;          /* lambda_d, weight on the squared depth residual */
  double invalid_depth_weight;  /* weight of the zero-target depth residual of m = 0 entries */
  double min_depth;             /* validity needs camera-frame z > min_depth */
  int extract_every;            /* residual drop at iterations k = e, 2e, ...; 0 = never */
  double drop_residual_px;      /* drop threshold on |r_uv|; <= 0 disables */
  int min_cam_obs, min_pt_obs;  /* extraction thresholds */
  double lambda0;
  double pcg_rel_tol;
  int pcg_max_iters;
  int solver;                   /* 0: dense Cholesky of the Schur system; 1: block-Jacobi PCG */
  int extract_mode;             /* 0: extraction at every iteration whose state changed (Sec. 4.2);
                                   1: one-shot, at the first iteration only, active set frozen */
  double nu0;                   /* initial damping growth factor nu (<= 0: 2, the rule's start) */
  int camera_model;             /* 0: radial [w, t, f, k1, k2], P = R X + t;
                                   1: Sec. 3.2's centre + rotation + focal, [w, c, f, -, -], P = R (X - c) */
} oracle_opts;

typedef struct {
  double cost;        /* F(x) at the start of the iteration over its active set */
  double rmse_px;     /* reprojection RMSE over the active set */
  double lambda;      /* damping used by this iteration's solve */
  double gain;        /* rho = (F(x) - F(x+dx)) / predicted decrease */
  double pred_decrease, cand_cost;
  int accepted, pcg_iters;
  double pcg_rel_res;
  int64_t n_cam_act, n_pt_act, n_obs_act;
} oracle_iter_log;

void oracle_default_opts(oracle_opts* o);

/* rotations */
void oracle_rotvec_to_matrix(const double w[3], double R[9]);
void oracle_rotvec_compose(const double a[3], const double b[3], double out[3]);

/* One observation: stacked residual r = [u^ - u, v^ - v, sqrt(wt)(1/z - tau)],
 * camera block Jc (3x9 row-major, left rotation increment) and point block Jp (3x3). */
void oracle_observe(const double cam[9], const double X[3], const double uv[2], double tau,
                    double wt, double cx, double cy, double r[3], double Jc[27], double Jp[9],
                    double* z, double uvhat[2]);

/* oracle_observe for a camera model (see oracle_opts.camera_model). */
void oracle_observe_model(int model, const double cam[9], const double X[3], const double uv[2],
                          double tau, double wt, double cx, double cy, double r[3], double Jc[27],
                          double Jp[9], double* z, double uvhat[2]);

/* Per-observation residuals / Jacobians / depth / projection for all N observations.
 * Any output may be NULL. */
void oracle_eval_obs(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                     const double* pts, double* r, double* Jc, double* Jp, double* z,
                     double* uvhat);

/* F = 1/2 sum rho(|r_k|^2) over observations with mask[k] != 0 (mask NULL = all). */
double oracle_cost(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                   const double* pts, const uint8_t* mask, double* rmse_px);

/* Geometric validity (z > min_depth and inside the image) and |r_uv| per observation. */
void oracle_predicate(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                      const double* pts, uint8_t* geom_valid, double* res_px);

/* Active-set extraction from per-observation validity.  Returns the number of
 * peeling rounds.  cam_rank: rank among active non-gauge cameras or -1;
 * pt_rank: rank among active points or -1. */
int oracle_extract(const oracle_problem* pb, const oracle_opts* o, const uint8_t* valid,
                   uint8_t* cam_mask, uint8_t* pt_mask, uint8_t* obs_mask, int32_t* cam_rank,
                   int32_t* pt_rank, int64_t* n_cam_free, int64_t* n_pt_act);

/* Robust-weighted normal-equation blocks over observations with obs_mask != 0:
 * U [C][81], V [P][9], W [N][27] (9x3 row-major), gc [C][9], gp [P][3]. */
void oracle_normal_equations(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                             const double* pts, const uint8_t* obs_mask, double* U, double* V,
                             double* W, double* gc, double* gp);

/* Dense damped Schur system S [nf][nf], rhs b [nf] (nf = 9 * n_cam_free). */
void oracle_schur_dense(const oracle_problem* pb, const double* U, const double* V,
                        const double* W, const double* gc, const double* gp,
                        const uint8_t* obs_mask, const int32_t* cam_rank, const int32_t* pt_rank,
                        int64_t n_cam_free, double lambda, double* S, double* b);

/* Damped LM step: dc [C][9] and dp [P][3] (zero for inactive/gauge entries).
 * Returns PCG iterations (0 for the direct solve), or -1 if the factorisation failed. */
int oracle_solve_step(const oracle_problem* pb, const oracle_opts* o, const double* U,
                      const double* V, const double* W, const double* gc, const double* gp,
                      const uint8_t* obs_mask, const int32_t* cam_rank, const int32_t* pt_rank,
                      int64_t n_cam_free, double lambda, double* dc, double* dp,
                      double* pred_decrease, double* pcg_rel_res);

/* x <- x (+) dx: rotation by left composition, the rest additive. */
void oracle_apply_step(int64_t n_cams, int64_t n_pts, const double* cams, const double* pts,
                       const double* dc, const double* dp, double* cams_out, double* pts_out);

/* Accept test of one LM step: 1 when gain = (F - Fc) / pred > 1e-3 with Fc
 * finite and pred > 0 (Sec. 3.3; Nielsen's rule). */
int oracle_lm_accept(double F, double Fc, double pred);

/* Damping update after a step: accepted, lambda *= max(1/3, 1 - (2 gain - 1)^3)
 * and nu = 2; rejected, lambda *= nu and nu *= 2. */
void oracle_lm_damping(int accepted, double gain, double* lambda, double* nu);

/* Full LM loop.  cams/pts are updated in place; log has max_iters entries (or NULL);
 * alive [N] is the sticky residual-drop state (NULL = internal, all alive).
 * Returns the number of iterations run. */
int oracle_lm(const oracle_problem* pb, const oracle_opts* o, int max_iters, double* cams,
              double* pts, oracle_iter_log* log, uint8_t* alive);

/* Implicit adjoint at a converged state: solves H mu = (dL/dcams, dL/dpts) with the
 * undamped Gauss-Newton matrix of the active set (IRLS weights frozen) and returns
 * dL/duv [N][2] and dL/ddepth [N]. */
/* Inverse left Jacobian of SO(3) (row-major 3x3). */
void oracle_so3_left_jacobian_inv(const double w[3], double J[9]);

int oracle_backward(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                    const double* pts, const uint8_t* obs_mask, const int32_t* cam_rank,
                    const int32_t* pt_rank, int64_t n_cam_free, const double* dL_dcams,
                    const double* dL_dpts, double* dL_duv, double* dL_ddepth);

void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
