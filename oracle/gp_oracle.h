/* gp_oracle.h -- plain FP64 CPU reference for the depth-constrained global
 * positioning (GP) stage of InstantSfM (arXiv 2510.13310).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle that the CUDA GP path is checked
 * against; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * What it computes, in the paper's terms:
 *   - GP objective (Sec. 3.1, Eq. GP objective): sum_k rho(|u_k|^2) with
 *     u_k = v_k - s_k (X_j - t_i) for observation k = (camera i, point j), v_k the
 *     unit ray from the camera centre t_i toward the observed feature (world
 *     frame, rotations known and fixed), s_k a per-observation scale, rho Huber.
 *   - Depth constraint (Sec. 4.1, GP paragraph): an observation with a metric
 *     depth d_k has its scale pinned, s_k = 1/d_k, and removed from the unknowns;
 *     the others keep s_k free.  The partition S_pin = {k | m_k = 1},
 *     S_free = {k | m_k = 0} is a set-membership test; free scales are compacted
 *     by their rank among the free observations.
 *   - LM (Sec. 3.3, Eq. LM): (J^T J + lambda diag(J^T J)) dx = -J^T r over the
 *     free centres, the points and the free scales; the same accept rule and
 *     damping schedule as the BA oracle (oracle_lm_accept, oracle_lm_damping).
 * Readings of what the paper leaves open are stated beside each function.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>

#include "ba_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t n_cams, n_pts, n_obs;
  const int32_t* obs_cam;  /* [N] */
  const int32_t* obs_pt;   /* [N] */
  const double* rays;      /* [N][3] unit direction from the camera centre toward the point */
  const double* depth;     /* [N] metric distance along the ray; <= 0 or NaN: none (free scale) */
  const uint8_t* fixed;    /* [C] 1 = gauge camera (centre held constant) */
} oracle_gp_problem;

typedef struct {
  double huber_delta;  /* Huber threshold on |u| (<= 0: squared loss) */
  double lambda0;      /* initial damping */
} oracle_gp_opts;

/* One observation: u = v - s (X - t) and its Jacobian blocks with respect to
 * t (3x3), X (3x3) and s (3x1), row-major. */
void oracle_gp_residual(const double t[3], const double X[3], const double v[3], double s,
                        double u[3], double Jt[9], double JX[9], double Js[3]);

/* Sec. 4.1 partition: free_rank[k] = rank of k among the free-scale observations
 * (no valid depth), -1 for pinned ones.  Returns |S_free|. */
int64_t oracle_gp_free_set(const oracle_gp_problem* pb, int32_t* free_rank);

/* Scale used by observation k: 1/d_k when pinned, scales[k] when free. */
double oracle_gp_scale(const oracle_gp_problem* pb, const double* scales, int64_t k);

/* F = 1/2 sum rho(|u_k|^2) over all observations; rms (nullable) = sqrt(mean |u_k|^2). */
double oracle_gp_cost(const oracle_gp_problem* pb, const oracle_gp_opts* o, const double* centres,
                      const double* pts, const double* scales, double* rms);

/* Robust-weighted normal-equation blocks (undamped):
 * U [C][9] (centre), V [P][9] (point), W [N][9] (centre-point of each observation),
 * Hts [N][3], HXs [N][3] (centre-scale and point-scale), Q [N] (scale-scale),
 * gt [C][3], gX [P][3], gs [N]; the scale entries are zero for pinned observations. */
void oracle_gp_normal_equations(const oracle_gp_problem* pb, const oracle_gp_opts* o,
                                const double* centres, const double* pts, const double* scales,
                                double* U, double* V, double* W, double* Hts, double* HXs,
                                double* Q, double* gt, double* gX, double* gs);

/* Damped LM step at damping lambda: dt [C][3] (zero for gauge cameras and
 * cameras without observations), dX [P][3], ds [N] (zero for pinned
 * observations) and the predicted decrease.  Returns 0, or -1 when the
 * factorisation fails. */
int oracle_gp_solve_step(const oracle_gp_problem* pb, const oracle_gp_opts* o, const double* centres,
                         const double* pts, const double* scales, double lambda, double* dt,
                         double* dX, double* ds, double* pred_decrease);

/* Full LM loop; centres [C][3], pts [P][3], scales [N] updated in place; log has
 * max_iters entries or is NULL (n_cam_act = free cameras, n_pt_act = points with
 * observations, n_obs_act = free scales).  Returns the iterations run. */
int oracle_gp_lm(const oracle_gp_problem* pb, const oracle_gp_opts* o, int max_iters, double* centres,
                 double* pts, double* scales, oracle_iter_log* log);

#ifdef __cplusplus
}
#endif
#endif
