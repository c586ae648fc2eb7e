/* ba_oracle.c -- plain FP64 CPU reference of the depth-prior LM bundle adjustment
 * with dynamic parameter extraction (InstantSfM, arXiv 2510.13310).
 *
 * TEST INFRASTRUCTURE ONLY: the oracle the CUDA path is checked against.  It is
 * written for readability, in the order the paper states each step; loops that
 * run in parallel (OpenMP) only ever write their own outputs, and every sum is
 * taken in a fixed order, so results do not depend on the thread count.
 */
#include "ba_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* options                                                                    */
/* ------------------------------------------------------------------------- */

void oracle_default_opts(oracle_opts* o) {
  o->img_w = 640;
  o->img_h = 480;
  o->cx = 320.0;
  o->cy = 240.0;
  o->huber_delta = 1.0;
  o->depth_weight = 1.0;
  o->invalid_depth_weight = 0.0;
  o->min_depth = 0.1;
  o->extract_every = 0;
  o->drop_residual_px = 0.0;
  o->min_cam_obs = 1;
  o->min_pt_obs = 1;
  o->lambda0 = 1e-4;
  o->pcg_rel_tol = 1e-6;
  o->pcg_max_iters = 500;
  o->solver = 0;
  o->extract_mode = 0;
  o->nu0 = 2.0;
  o->camera_model = 0;
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* rotations: axis-angle <-> unit quaternion <-> matrix                       */
/* ------------------------------------------------------------------------- */

static void rotvec_to_quat(const double w[3], double q[4]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double c, s; /* q = (cos(th/2), sin(th/2)/th * w) */
  if (th < 1e-8) {
    c = 1.0 - th2 / 8.0;
    s = 0.5 - th2 / 48.0;
  } else {
    c = cos(0.5 * th);
    s = sin(0.5 * th) / th;
  }
  q[0] = c;
  q[1] = s * w[0];
  q[2] = s * w[1];
  q[3] = s * w[2];
}

static void quat_to_rotvec(const double qin[4], double w[3]) {
  double q[4] = {qin[0], qin[1], qin[2], qin[3]};
  if (q[0] < 0) { /* same rotation, angle in [0, pi] */
    q[0] = -q[0]; q[1] = -q[1]; q[2] = -q[2]; q[3] = -q[3];
  }
  double vn = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double k; /* w = 2 atan2(|v|, q0) / |v| * v */
  if (vn < 1e-8) {
    k = 2.0 / q[0] * (1.0 - vn * vn / (3.0 * q[0] * q[0]));
  } else {
    k = 2.0 * atan2(vn, q[0]) / vn;
  }
  w[0] = k * q[1];
  w[1] = k * q[2];
  w[2] = k * q[3];
}

static void quat_mul(const double a[4], const double b[4], double o[4]) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

void oracle_rotvec_to_matrix(const double w[3], double R[9]) {
  /* Rodrigues: R = I + sin(th) K + (1 - cos(th)) K^2, K = [w/th]x */
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double a, b; /* R = I + a [w]x + b [w]x^2 */
  if (th < 1e-8) {
    a = 1.0 - th2 / 6.0;
    b = 0.5 - th2 / 24.0;
  } else {
    a = sin(th) / th;
    b = (1.0 - cos(th)) / th2;
  }
  double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int l = 0; l < 3; ++l) s += K[3 * i + l] * K[3 * l + j];
      K2[3 * i + j] = s;
    }
  for (int i = 0; i < 9; ++i) R[i] = a * K[i] + b * K2[i];
  R[0] += 1.0;
  R[4] += 1.0;
  R[8] += 1.0;
}

void oracle_rotvec_compose(const double a[3], const double b[3], double out[3]) {
  double qa[4], qb[4], q[4];
  rotvec_to_quat(a, qa);
  rotvec_to_quat(b, qb);
  quat_mul(qa, qb, q);
  quat_to_rotvec(q, out);
}

/* ------------------------------------------------------------------------- */
/* one observation: Eq. (BA objective) residual + depth residual (Sec. 4.1)   */
/* ------------------------------------------------------------------------- */

/* Observation weight of the depth row.  Sec. 4.1: the inverse-depth target is
 * d~^-1 = m d^-1, so entries without a valid prior (m = 0) target 0; reading:
 * their squared residual is weighted by invalid_depth_weight (0 by default,
 * i.e. no prior), valid entries by lambda_d. */
static int has_prior(double d) { return d > 0.0 && isfinite(d); }

static double depth_tau(double d) { return has_prior(d) ? 1.0 / d : 0.0; }

static double depth_wt(const oracle_opts* o, double d) {
  return has_prior(d) ? o->depth_weight : o->invalid_depth_weight;
}

void oracle_observe(const double cam[9], const double X[3], const double uv[2], double tau,
                    double wt, double cx, double cy, double r[3], double Jc[27], double Jp[9],
                    double* zout, double uvhat[2]) {
  oracle_observe_model(0, cam, X, uv, tau, wt, cx, cy, r, Jc, Jp, zout, uvhat);
}

/* Camera models.  0: the 9-parameter radial camera, P = R X + t.  1: the
 * parameterisation of Sec. 3.2 (camera centre, rotation, focal length; no
 * distortion), stored in the same nine slots as [w, c, f, 0, 0]: P = R (X - c),
 * the rotation increment left-multiplicative as for model 0; the k1, k2 slots are
 * ignored (no column), so the step leaves them unchanged. */
void oracle_observe_model(int model, const double cam[9], const double X[3], const double uv[2],
                          double tau, double wt, double cx, double cy, double r[3], double Jc[27],
                          double Jp[9], double* zout, double uvhat[2]) {
  double R[9];
  oracle_rotvec_to_matrix(cam, R);
  const double* t = cam + 3;
  double f = cam[6], k1 = model == 1 ? 0.0 : cam[7], k2 = model == 1 ? 0.0 : cam[8];
  double RX[3], P[3];
  if (model == 1) {
    double d[3] = {X[0] - t[0], X[1] - t[1], X[2] - t[2]};
    for (int i = 0; i < 3; ++i) P[i] = R[3 * i + 0] * d[0] + R[3 * i + 1] * d[1] + R[3 * i + 2] * d[2];
    /* the rotation increment acts on R (X - c) = P */
    for (int i = 0; i < 3; ++i) RX[i] = P[i];
  } else {
    for (int i = 0; i < 3; ++i) {
      RX[i] = R[3 * i + 0] * X[0] + R[3 * i + 1] * X[1] + R[3 * i + 2] * X[2];
      P[i] = RX[i] + t[i];
    }
  }
  double z = P[2];
  double xn = P[0] / z, yn = P[1] / z;
  double rr = xn * xn + yn * yn;
  double dist = 1.0 + k1 * rr + k2 * rr * rr;
  double uh = f * dist * xn + cx;
  double vh = f * dist * yn + cy;
  double sw = sqrt(wt);
  if (zout) *zout = z;
  if (uvhat) { uvhat[0] = uh; uvhat[1] = vh; }
  if (r) {
    r[0] = uh - uv[0];
    r[1] = vh - uv[1];
    r[2] = sw * (1.0 / z - tau);
  }
  if (!Jc && !Jp) return;

  /* d(residual rows)/dP, 3x3 */
  double iz = 1.0 / z;
  double dxn[3] = {iz, 0.0, -xn * iz};
  double dyn[3] = {0.0, iz, -yn * iz};
  double drr[3];
  for (int i = 0; i < 3; ++i) drr[i] = 2.0 * xn * dxn[i] + 2.0 * yn * dyn[i];
  double ddist = k1 + 2.0 * k2 * rr; /* d dist / d rr */
  double D[3][3];
  for (int i = 0; i < 3; ++i) {
    D[0][i] = f * (dist * dxn[i] + xn * ddist * drr[i]);
    D[1][i] = f * (dist * dyn[i] + yn * ddist * drr[i]);
  }
  D[2][0] = 0.0;
  D[2][1] = 0.0;
  D[2][2] = -sw * iz * iz;

  if (Jc) {
    /* dP/d(dw) = -[R X]x (model 0) or -[R (X - c)]x (model 1) for the left
     * increment Exp(dw) R */
    double A[3][3] = {{0.0, RX[2], -RX[1]}, {-RX[2], 0.0, RX[0]}, {RX[1], -RX[0], 0.0}};
    for (int m = 0; m < 3; ++m) {
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int l = 0; l < 3; ++l) s += D[m][l] * A[l][j];
        Jc[9 * m + j] = s; /* rotation */
        if (model == 1) {  /* centre: dP/dc = -R */
          double sc = 0;
          for (int l = 0; l < 3; ++l) sc += D[m][l] * R[3 * l + j];
          Jc[9 * m + 3 + j] = -sc;
        } else {
          Jc[9 * m + 3 + j] = D[m][j]; /* translation: dP/dt = I */
        }
      }
    }
    /* intrinsics */
    Jc[9 * 0 + 6] = dist * xn;
    Jc[9 * 0 + 7] = f * xn * rr;
    Jc[9 * 0 + 8] = f * xn * rr * rr;
    Jc[9 * 1 + 6] = dist * yn;
    Jc[9 * 1 + 7] = f * yn * rr;
    Jc[9 * 1 + 8] = f * yn * rr * rr;
    Jc[9 * 2 + 6] = 0.0;
    Jc[9 * 2 + 7] = 0.0;
    Jc[9 * 2 + 8] = 0.0;
    if (model == 1)
      for (int m = 0; m < 3; ++m) Jc[9 * m + 7] = Jc[9 * m + 8] = 0.0;
  }
  if (Jp) { /* dP/dX = R */
    for (int m = 0; m < 3; ++m)
      for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int l = 0; l < 3; ++l) s += D[m][l] * R[3 * l + j];
        Jp[3 * m + j] = s;
      }
  }
}

void oracle_eval_obs(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                     const double* pts, double* r, double* Jc, double* Jp, double* z,
                     double* uvhat) {
  int64_t N = pb->n_obs;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    int c = pb->obs_cam[k], p = pb->obs_pt[k];
    double d = pb->depth[k];
    oracle_observe_model(o->camera_model, cams + 9 * (int64_t)c, pts + 3 * (int64_t)p, pb->obs_uv + 2 * k, depth_tau(d),
                   depth_wt(o, d), o->cx, o->cy, r ? r + 3 * k : NULL, Jc ? Jc + 27 * k : NULL,
                   Jp ? Jp + 9 * k : NULL, z ? z + k : NULL, uvhat ? uvhat + 2 * k : NULL);
  }
}

/* Huber on the squared norm s (Sec. 3.1/3.2: rho is Huber).  Reading: rho acts on
 * s = |r|^2 of the stacked 3-row residual, rho(s) = s (s <= delta^2) or
 * 2 delta sqrt(s) - delta^2; IRLS weight rho'(s) = min(1, delta / sqrt(s)). */
static double huber_rho(double s, double delta) {
  if (delta <= 0.0 || s <= delta * delta) return s;
  return 2.0 * delta * sqrt(s) - delta * delta;
}

static double huber_w(double s, double delta) {
  if (delta <= 0.0 || s <= delta * delta) return 1.0;
  return delta / sqrt(s);
}

double oracle_cost(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                   const double* pts, const uint8_t* mask, double* rmse_px) {
  int64_t N = pb->n_obs;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  double* e2 = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    rho[k] = 0.0;
    e2[k] = 0.0;
    if (mask && !mask[k]) continue;
    double r[3];
    double d = pb->depth[k];
    oracle_observe_model(o->camera_model, cams + 9 * (int64_t)pb->obs_cam[k], pts + 3 * (int64_t)pb->obs_pt[k],
                   pb->obs_uv + 2 * k, depth_tau(d), depth_wt(o, d), o->cx, o->cy, r, NULL,
                   NULL, NULL, NULL);
    double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    rho[k] = huber_rho(s, o->huber_delta);
    e2[k] = r[0] * r[0] + r[1] * r[1];
  }
  double F = 0.0, E = 0.0;
  int64_t n = 0;
  for (int64_t k = 0; k < N; ++k) {
    F += rho[k];
    E += e2[k];
    if (!mask || mask[k]) ++n;
  }
  free(rho);
  free(e2);
  if (rmse_px) *rmse_px = n > 0 ? sqrt(E / (double)n) : 0.0;
  return 0.5 * F;
}

/* ------------------------------------------------------------------------- */
/* dynamic parameter extraction (Sec. 4.2, steps 1 and 2)                     */
/* ------------------------------------------------------------------------- */

/* Step 1 validity: projected depth z > min_depth (Eq. O_valid); reading of the
 * "out-of-frustum" clause: the distorted projection must fall in [0,W) x [0,H). */
void oracle_predicate(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                      const double* pts, uint8_t* geom_valid, double* res_px) {
  int64_t N = pb->n_obs;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    double r[3], z, uvh[2];
    double d = pb->depth[k];
    oracle_observe_model(o->camera_model, cams + 9 * (int64_t)pb->obs_cam[k], pts + 3 * (int64_t)pb->obs_pt[k],
                   pb->obs_uv + 2 * k, depth_tau(d), depth_wt(o, d), o->cx, o->cy, r, NULL,
                   NULL, &z, uvh);
    int ok = z > o->min_depth && uvh[0] >= 0.0 && uvh[0] < (double)o->img_w && uvh[1] >= 0.0 &&
             uvh[1] < (double)o->img_h;
    if (geom_valid) geom_valid[k] = (uint8_t)ok;
    if (res_px) res_px[k] = sqrt(r[0] * r[0] + r[1] * r[1]);
  }
}

/* Step 2: cameras / points that keep enough valid observations.  With the
 * paper's thresholds (1, 1) this is exactly unique(i_c), unique(i_p) over
 * O_valid (Eqs. C_active, P_active).  With larger thresholds (Fig. 2's
 * "observed by fewer cameras than a threshold") removing a point can drop a
 * camera below its threshold and vice versa; reading: peel until nothing
 * changes, which gives the largest sub-incidence meeting both thresholds.
 * Gauge cameras are never peeled.  Ranks are ascending positions (Eq. rank). */
int oracle_extract(const oracle_problem* pb, const oracle_opts* o, const uint8_t* valid,
                   uint8_t* cam_mask, uint8_t* pt_mask, uint8_t* obs_mask, int32_t* cam_rank,
                   int32_t* pt_rank, int64_t* n_cam_free, int64_t* n_pt_act) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  int64_t* cc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(C + 1));
  int64_t* pc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P + 1));
  for (int64_t c = 0; c < C; ++c) cam_mask[c] = 1;
  for (int64_t p = 0; p < P; ++p) pt_mask[p] = 1;
  int rounds = 0;
  for (;;) {
    ++rounds;
    for (int64_t k = 0; k < N; ++k)
      obs_mask[k] = (uint8_t)(valid[k] && cam_mask[pb->obs_cam[k]] && pt_mask[pb->obs_pt[k]]);
    memset(cc, 0, sizeof(int64_t) * (size_t)C);
    memset(pc, 0, sizeof(int64_t) * (size_t)P);
    for (int64_t k = 0; k < N; ++k)
      if (obs_mask[k]) {
        cc[pb->obs_cam[k]]++;
        pc[pb->obs_pt[k]]++;
      }
    int changed = 0;
    for (int64_t c = 0; c < C; ++c) {
      uint8_t m = (uint8_t)(pb->fixed[c] || (cam_mask[c] && cc[c] >= o->min_cam_obs));
      if (m != cam_mask[c]) changed = 1;
      cam_mask[c] = m;
    }
    for (int64_t p = 0; p < P; ++p) {
      uint8_t m = (uint8_t)(pt_mask[p] && pc[p] >= o->min_pt_obs);
      if (m != pt_mask[p]) changed = 1;
      pt_mask[p] = m;
    }
    if (!changed) break;
  }
  for (int64_t k = 0; k < N; ++k)
    obs_mask[k] = (uint8_t)(valid[k] && cam_mask[pb->obs_cam[k]] && pt_mask[pb->obs_pt[k]]);
  int64_t nc = 0, np = 0;
  for (int64_t c = 0; c < C; ++c) cam_rank[c] = (cam_mask[c] && !pb->fixed[c]) ? (int32_t)nc++ : -1;
  for (int64_t p = 0; p < P; ++p) pt_rank[p] = pt_mask[p] ? (int32_t)np++ : -1;
  if (n_cam_free) *n_cam_free = nc;
  if (n_pt_act) *n_pt_act = np;
  free(cc);
  free(pc);
  return rounds;
}

/* ------------------------------------------------------------------------- */
/* normal equations (Sec. 3.3, Eq. LM) with IRLS-weighted Huber                */
/* ------------------------------------------------------------------------- */

/* CSR of observation indices grouped by key, ascending observation index. */
typedef struct {
  int64_t* off;
  int64_t* idx;
} csr_t;

static csr_t build_csr(int64_t nkeys, int64_t N, const int32_t* key) {
  csr_t g;
  g.off = (int64_t*)calloc((size_t)(nkeys + 1), sizeof(int64_t));
  g.idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t k = 0; k < N; ++k) g.off[key[k] + 1]++;
  for (int64_t i = 0; i < nkeys; ++i) g.off[i + 1] += g.off[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nkeys + 1));
  memcpy(fill, g.off, sizeof(int64_t) * (size_t)(nkeys + 1));
  for (int64_t k = 0; k < N; ++k) g.idx[fill[key[k]]++] = k;
  free(fill);
  return g;
}

static void free_csr(csr_t* g) {
  free(g->off);
  free(g->idx);
}

void oracle_normal_equations(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                             const double* pts, const uint8_t* obs_mask, double* U, double* V,
                             double* W, double* gc, double* gp) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  /* per observation: weighted J_c^T J_c, J_p^T J_p, J_c^T J_p, J^T r */
  double* r = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
  double* Jc = (double*)malloc(sizeof(double) * 27 * (size_t)(N > 0 ? N : 1));
  double* Jp = (double*)malloc(sizeof(double) * 9 * (size_t)(N > 0 ? N : 1));
  double* wk = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  oracle_eval_obs(pb, o, cams, pts, r, Jc, Jp, NULL, NULL);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    const double* rk = r + 3 * k;
    double s = rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2];
    wk[k] = (obs_mask && !obs_mask[k]) ? 0.0 : huber_w(s, o->huber_delta);
    for (int a = 0; a < 9; ++a)
      for (int b = 0; b < 3; ++b) {
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += Jc[27 * k + 9 * m + a] * Jp[9 * k + 3 * m + b];
        W[27 * k + 3 * a + b] = wk[k] * acc;
      }
  }
  csr_t byc = build_csr(C, N, pb->obs_cam);
  csr_t byp = build_csr(P, N, pb->obs_pt);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < C; ++c) {
    double* Uc = U + 81 * c;
    double* g = gc + 9 * c;
    memset(Uc, 0, sizeof(double) * 81);
    memset(g, 0, sizeof(double) * 9);
    for (int64_t q = byc.off[c]; q < byc.off[c + 1]; ++q) {
      int64_t k = byc.idx[q];
      if (wk[k] == 0.0) continue;
      const double* J = Jc + 27 * k;
      for (int a = 0; a < 9; ++a) {
        for (int b = 0; b < 9; ++b) {
          double acc = 0;
          for (int m = 0; m < 3; ++m) acc += J[9 * m + a] * J[9 * m + b];
          Uc[9 * a + b] += wk[k] * acc;
        }
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += J[9 * m + a] * r[3 * k + m];
        g[a] += wk[k] * acc;
      }
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p) {
    double* Vp = V + 9 * p;
    double* g = gp + 3 * p;
    memset(Vp, 0, sizeof(double) * 9);
    memset(g, 0, sizeof(double) * 3);
    for (int64_t q = byp.off[p]; q < byp.off[p + 1]; ++q) {
      int64_t k = byp.idx[q];
      if (wk[k] == 0.0) continue;
      const double* J = Jp + 9 * k;
      for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
          double acc = 0;
          for (int m = 0; m < 3; ++m) acc += J[3 * m + a] * J[3 * m + b];
          Vp[3 * a + b] += wk[k] * acc;
        }
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += J[3 * m + a] * r[3 * k + m];
        g[a] += wk[k] * acc;
      }
    }
  }
  free_csr(&byc);
  free_csr(&byp);
  free(r);
  free(Jc);
  free(Jp);
  free(wk);
}

/* ------------------------------------------------------------------------- */
/* small dense helpers                                                        */
/* ------------------------------------------------------------------------- */

/* Marquardt damping (Eq. LM): A + lambda diag(A); reading: the diagonal used for
 * scaling is clamped to [1e-6, 1e32]. */
static double damp_diag(double a) {
  if (a < 1e-6) return 1e-6;
  if (a > 1e32) return 1e32;
  return a;
}

/* In-place Cholesky A = L L^T of an n x n row-major matrix (lower part used). */
static int chol_small(double* A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[n * j + j];
    for (int l = 0; l < j; ++l) s -= A[n * j + l] * A[n * j + l];
    if (!(s > 0.0)) return -1;
    double d = sqrt(s);
    A[n * j + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[n * i + j];
      for (int l = 0; l < j; ++l) t -= A[n * i + l] * A[n * j + l];
      A[n * i + j] = t / d;
    }
  }
  return 0;
}

static void chol_solve_small(const double* L, int n, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int l = 0; l < i; ++l) s -= L[n * i + l] * x[l];
    x[i] = s / L[n * i + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int l = i + 1; l < n; ++l) s -= L[n * l + i] * x[l];
    x[i] = s / L[n * i + i];
  }
}

/* Dense Cholesky by columns (Crout); rows of each column are independent. */
static int chol_dense(double* A, int64_t n) {
  int fail = 0;
  for (int64_t j = 0; j < n && !fail; ++j) {
    double s = A[n * j + j];
    for (int64_t l = 0; l < j; ++l) s -= A[n * j + l] * A[n * j + l];
    if (!(s > 0.0)) {
      fail = 1;
      break;
    }
    double d = sqrt(s);
    A[n * j + j] = d;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double t = A[n * i + j];
      const double* Li = A + n * i;
      const double* Lj = A + n * j;
      for (int64_t l = 0; l < j; ++l) t -= Li[l] * Lj[l];
      A[n * i + j] = t / d;
    }
  }
  return fail ? -1 : 0;
}

static void chol_dense_solve(const double* L, int64_t n, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = x[i];
    for (int64_t l = 0; l < i; ++l) s -= L[n * i + l] * x[l];
    x[i] = s / L[n * i + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t l = i + 1; l < n; ++l) s -= L[n * l + i] * x[l];
    x[i] = s / L[n * i + i];
  }
}

/* 3x3 SPD inverse through its Cholesky factor. */
static int inv3_spd(const double* A, double* Ainv) {
  double L[9];
  memcpy(L, A, sizeof L);
  if (chol_small(L, 3)) return -1;
  for (int j = 0; j < 3; ++j) {
    double e[3] = {0, 0, 0};
    e[j] = 1.0;
    chol_solve_small(L, 3, e);
    for (int i = 0; i < 3; ++i) Ainv[3 * i + j] = e[i];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Schur complement on the compacted unknowns (Sec. 4.2 step 2, Eq. LM)        */
/* ------------------------------------------------------------------------- */

/* Damped, inverted point blocks V*^-1 (zero for inactive points). */
static int damped_point_inverses(int64_t P, const double* V, const int32_t* pt_rank,
                                 double lambda, double* Vinv) {
  int fail = 0;
#pragma omp parallel for schedule(static) reduction(| : fail)
  for (int64_t p = 0; p < P; ++p) {
    double* Vi = Vinv + 9 * p;
    if (pt_rank[p] < 0) {
      memset(Vi, 0, sizeof(double) * 9);
      continue;
    }
    double A[9];
    memcpy(A, V + 9 * p, sizeof A);
    for (int a = 0; a < 3; ++a) A[4 * a] += lambda * damp_diag(V[9 * p + 4 * a]);
    if (inv3_spd(A, Vi)) fail |= 1;
  }
  return fail ? -1 : 0;
}

void oracle_schur_dense(const oracle_problem* pb, const double* U, const double* V,
                        const double* W, const double* gc, const double* gp,
                        const uint8_t* obs_mask, const int32_t* cam_rank, const int32_t* pt_rank,
                        int64_t n_cam_free, double lambda, double* S, double* b) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  int64_t n = 9 * n_cam_free;
  double* Vinv = (double*)malloc(sizeof(double) * 9 * (size_t)(P > 0 ? P : 1));
  damped_point_inverses(P, V, pt_rank, lambda, Vinv);
  csr_t byc = build_csr(C, N, pb->obs_cam);
  csr_t byp = build_csr(P, N, pb->obs_pt);
  memset(S, 0, sizeof(double) * (size_t)(n * n));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < C; ++c) {
    int32_t a = cam_rank[c];
    if (a < 0) continue;
    /* diagonal block: damped U */
    for (int i = 0; i < 9; ++i) {
      for (int j = 0; j < 9; ++j) S[(9 * a + i) * n + 9 * a + j] = U[81 * c + 9 * i + j];
      S[(9 * a + i) * n + 9 * a + i] += lambda * damp_diag(U[81 * c + 10 * i]);
      b[9 * a + i] = -gc[9 * c + i];
    }
    for (int64_t q = byc.off[c]; q < byc.off[c + 1]; ++q) {
      int64_t k = byc.idx[q];
      if (!obs_mask[k]) continue;
      int32_t p = pb->obs_pt[k];
      const double* Wk = W + 27 * k;
      const double* Vi = Vinv + 9 * (int64_t)p;
      double Y[27]; /* W_k V*^-1 */
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0;
          for (int l = 0; l < 3; ++l) s += Wk[3 * i + l] * Vi[3 * l + j];
          Y[3 * i + j] = s;
        }
      /* b += W V^-1 g_p */
      for (int i = 0; i < 9; ++i) {
        double s = 0;
        for (int l = 0; l < 3; ++l) s += Y[3 * i + l] * gp[3 * (int64_t)p + l];
        b[9 * a + i] += s;
      }
      /* S row block a -= W_k V^-1 W_k'^T for every active observation k' of p */
      for (int64_t q2 = byp.off[p]; q2 < byp.off[p + 1]; ++q2) {
        int64_t k2 = byp.idx[q2];
        if (!obs_mask[k2]) continue;
        int32_t bcol = cam_rank[pb->obs_cam[k2]];
        if (bcol < 0) continue;
        const double* W2 = W + 27 * k2;
        for (int i = 0; i < 9; ++i)
          for (int j = 0; j < 9; ++j) {
            double s = 0;
            for (int l = 0; l < 3; ++l) s += Y[3 * i + l] * W2[3 * j + l];
            S[(9 * a + i) * n + 9 * bcol + j] -= s;
          }
      }
    }
  }
  free_csr(&byc);
  free_csr(&byp);
  free(Vinv);
}

/* ------------------------------------------------------------------------- */
/* LM step solve (Eq. LM) with scatter back to full arrays (Sec. 4.2 step 3)  */
/* ------------------------------------------------------------------------- */

typedef struct {
  const oracle_problem* pb;
  const double *U, *W, *Vinv;
  const uint8_t* obs_mask;
  const int32_t* cam_rank;
  csr_t byc, byp;
  double lambda;
  int64_t nf;
} schur_op;

/* y = S x with S applied implicitly: U* x - W V*^-1 (W^T x). */
static void schur_apply(const schur_op* s, const double* x, double* y, double* tp) {
  const oracle_problem* pb = s->pb;
  int64_t C = pb->n_cams, P = pb->n_pts;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < P; ++p) {
    double t[3] = {0, 0, 0};
    for (int64_t q = s->byp.off[p]; q < s->byp.off[p + 1]; ++q) {
      int64_t k = s->byp.idx[q];
      if (!s->obs_mask[k]) continue;
      int32_t a = s->cam_rank[pb->obs_cam[k]];
      if (a < 0) continue;
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 9; ++i) t[j] += s->W[27 * k + 3 * i + j] * x[9 * a + i];
    }
    const double* Vi = s->Vinv + 9 * p;
    for (int i = 0; i < 3; ++i) tp[3 * p + i] = Vi[3 * i] * t[0] + Vi[3 * i + 1] * t[1] + Vi[3 * i + 2] * t[2];
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < C; ++c) {
    int32_t a = s->cam_rank[c];
    if (a < 0) continue;
    const double* Uc = s->U + 81 * c;
    for (int i = 0; i < 9; ++i) {
      double acc = 0;
      for (int j = 0; j < 9; ++j) acc += Uc[9 * i + j] * x[9 * a + j];
      acc += s->lambda * damp_diag(Uc[10 * i]) * x[9 * a + i];
      y[9 * a + i] = acc;
    }
    for (int64_t q = s->byc.off[c]; q < s->byc.off[c + 1]; ++q) {
      int64_t k = s->byc.idx[q];
      if (!s->obs_mask[k]) continue;
      int32_t p = pb->obs_pt[k];
      for (int i = 0; i < 9; ++i) {
        double acc = 0;
        for (int j = 0; j < 3; ++j) acc += s->W[27 * k + 3 * i + j] * tp[3 * (int64_t)p + j];
        y[9 * a + i] -= acc;
      }
    }
  }
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Block-Jacobi preconditioned CG on S x = b, x0 = 0, stop when |r| <= tol |b|.
 * Blocks are the 9x9 diagonal blocks of S. */
static int pcg(const schur_op* s, const oracle_opts* o, const double* b, double* x,
               double* rel_res) {
  const oracle_problem* pb = s->pb;
  int64_t C = pb->n_cams, P = pb->n_pts, nf = s->nf;
  int64_t n = 9 * nf;
  /* preconditioner blocks: D_a = U*_c - sum_{k in c} W_k V*^-1 W_k^T */
  double* Dl = (double*)malloc(sizeof(double) * 81 * (size_t)(nf > 0 ? nf : 1));
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
  for (int64_t c = 0; c < C; ++c) {
    int32_t a = s->cam_rank[c];
    if (a < 0) continue;
    double* D = Dl + 81 * (int64_t)a;
    for (int i = 0; i < 81; ++i) D[i] = s->U[81 * c + i];
    for (int i = 0; i < 9; ++i) D[10 * i] += s->lambda * damp_diag(s->U[81 * c + 10 * i]);
    for (int64_t q = s->byc.off[c]; q < s->byc.off[c + 1]; ++q) {
      int64_t k = s->byc.idx[q];
      if (!s->obs_mask[k]) continue;
      const double* Wk = s->W + 27 * k;
      const double* Vi = s->Vinv + 9 * (int64_t)pb->obs_pt[k];
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
          double acc = 0;
          for (int l = 0; l < 3; ++l)
            for (int m = 0; m < 3; ++m) acc += Wk[3 * i + l] * Vi[3 * l + m] * Wk[3 * j + m];
          D[9 * i + j] -= acc;
        }
    }
    if (chol_small(D, 9)) fail |= 1;
  }
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* tp = (double*)malloc(sizeof(double) * 3 * (size_t)(P > 0 ? P : 1));
  int it = 0;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
  }
  double bn = sqrt(dot(b, b, n));
  *rel_res = 0.0;
  if (fail) {
    it = -1;
  } else if (bn > 0.0) {
    for (int64_t i = 0; i < n; ++i) z[i] = r[i];
    for (int64_t a = 0; a < nf; ++a) chol_solve_small(Dl + 81 * a, 9, z + 9 * a);
    memcpy(p, z, sizeof(double) * (size_t)n);
    double rz = dot(r, z, n);
    double rn = bn;
    while (it < o->pcg_max_iters) {
      schur_apply(s, p, q, tp);
      ++it;
      double alpha = rz / dot(p, q, n);
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      rn = sqrt(dot(r, r, n));
      if (rn <= o->pcg_rel_tol * bn) break;
      for (int64_t i = 0; i < n; ++i) z[i] = r[i];
      for (int64_t a = 0; a < nf; ++a) chol_solve_small(Dl + 81 * a, 9, z + 9 * a);
      double rz2 = dot(r, z, n);
      double beta = rz2 / rz;
      rz = rz2;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    *rel_res = rn / bn;
  }
  free(Dl);
  free(r);
  free(z);
  free(p);
  free(q);
  free(tp);
  return it;
}

int oracle_solve_step(const oracle_problem* pb, const oracle_opts* o, const double* U,
                      const double* V, const double* W, const double* gc, const double* gp,
                      const uint8_t* obs_mask, const int32_t* cam_rank, const int32_t* pt_rank,
                      int64_t n_cam_free, double lambda, double* dc, double* dp,
                      double* pred_decrease, double* pcg_rel_res) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  int64_t n = 9 * n_cam_free;
  double* Vinv = (double*)malloc(sizeof(double) * 9 * (size_t)(P > 0 ? P : 1));
  double* xc = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* b = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  int status = 0;
  double relres = 0.0;
  /* Camera model of Sec. 3.2 (centre, rotation, focal): slots 7 and 8 are not
   * parameters.  Their Jacobian columns and gradient entries are zero; the solve
   * holds them with a unit diagonal in U (before damping), which decouples them
   * exactly (their unknowns come out zero) and keeps the undamped system of the
   * adjoint nonsingular.  The other unknowns are those of the system without the
   * two slots. */
  double* Uk = NULL;
  if (o->camera_model == 1 && C > 0) {
    Uk = (double*)malloc(sizeof(double) * 81 * (size_t)C);
    memcpy(Uk, U, sizeof(double) * 81 * (size_t)C);
    for (int64_t c = 0; c < C; ++c)
      for (int i = 7; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
          Uk[81 * c + 9 * i + j] = i == j ? 1.0 : 0.0;
          Uk[81 * c + 9 * j + i] = i == j ? 1.0 : 0.0;
        }
    U = Uk;
  }
  if (damped_point_inverses(P, V, pt_rank, lambda, Vinv)) status = -1;
  csr_t byc = build_csr(C, N, pb->obs_cam);
  csr_t byp = build_csr(P, N, pb->obs_pt);
  if (status == 0) {
    if (o->solver == 0) {
      double* S = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
      oracle_schur_dense(pb, U, V, W, gc, gp, obs_mask, cam_rank, pt_rank, n_cam_free, lambda, S, b);
      if (chol_dense(S, n)) status = -1;
      else {
        memcpy(xc, b, sizeof(double) * (size_t)n);
        chol_dense_solve(S, n, xc);
      }
      free(S);
    } else {
      /* b = -g_c + W V*^-1 g_p */
      for (int64_t c = 0; c < C; ++c) {
        int32_t a = cam_rank[c];
        if (a < 0) continue;
        for (int i = 0; i < 9; ++i) b[9 * a + i] = -gc[9 * c + i];
        for (int64_t q = byc.off[c]; q < byc.off[c + 1]; ++q) {
          int64_t k = byc.idx[q];
          if (!obs_mask[k]) continue;
          int32_t p = pb->obs_pt[k];
          double z3[3];
          for (int i = 0; i < 3; ++i)
            z3[i] = Vinv[9 * (int64_t)p + 3 * i] * gp[3 * (int64_t)p] +
                    Vinv[9 * (int64_t)p + 3 * i + 1] * gp[3 * (int64_t)p + 1] +
                    Vinv[9 * (int64_t)p + 3 * i + 2] * gp[3 * (int64_t)p + 2];
          for (int i = 0; i < 9; ++i)
            b[9 * a + i] += W[27 * k + 3 * i] * z3[0] + W[27 * k + 3 * i + 1] * z3[1] +
                            W[27 * k + 3 * i + 2] * z3[2];
        }
      }
      schur_op s = {pb, U, W, Vinv, obs_mask, cam_rank, byc, byp, lambda, n_cam_free};
      int it = pcg(&s, o, b, xc, &relres);
      if (it < 0) status = -1;
      else status = it;
    }
  }
  /* scatter back: inactive / gauge cameras and inactive points stay unchanged */
  memset(dc, 0, sizeof(double) * 9 * (size_t)C);
  memset(dp, 0, sizeof(double) * 3 * (size_t)P);
  if (status >= 0) {
    for (int64_t c = 0; c < C; ++c)
      if (cam_rank[c] >= 0) memcpy(dc + 9 * c, xc + 9 * (int64_t)cam_rank[c], sizeof(double) * 9);
    /* back-substitution: dp = V*^-1 (-g_p - sum_k W_k^T dc_{c(k)}) */
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
      if (pt_rank[p] < 0) continue;
      double t[3] = {-gp[3 * p], -gp[3 * p + 1], -gp[3 * p + 2]};
      for (int64_t q = byp.off[p]; q < byp.off[p + 1]; ++q) {
        int64_t k = byp.idx[q];
        if (!obs_mask[k]) continue;
        int32_t c = pb->obs_cam[k];
        if (cam_rank[c] < 0) continue;
        for (int j = 0; j < 3; ++j)
          for (int i = 0; i < 9; ++i) t[j] -= W[27 * k + 3 * i + j] * dc[9 * (int64_t)c + i];
      }
      const double* Vi = Vinv + 9 * p;
      for (int i = 0; i < 3; ++i) dp[3 * p + i] = Vi[3 * i] * t[0] + Vi[3 * i + 1] * t[1] + Vi[3 * i + 2] * t[2];
    }
    /* predicted decrease 1/2 dx^T (lambda D dx - g) over the compacted unknowns */
    double L = 0.0;
    for (int64_t c = 0; c < C; ++c) {
      if (cam_rank[c] < 0) continue;
      for (int i = 0; i < 9; ++i) {
        double d = dc[9 * c + i];
        L += d * (lambda * damp_diag(U[81 * c + 10 * i]) * d - gc[9 * c + i]);
      }
    }
    for (int64_t p = 0; p < P; ++p) {
      if (pt_rank[p] < 0) continue;
      for (int i = 0; i < 3; ++i) {
        double d = dp[3 * p + i];
        L += d * (lambda * damp_diag(V[9 * p + 4 * i]) * d - gp[3 * p + i]);
      }
    }
    *pred_decrease = 0.5 * L;
  }
  if (pcg_rel_res) *pcg_rel_res = relres;
  free_csr(&byc);
  free_csr(&byp);
  free(Vinv);
  free(xc);
  free(b);
  free(Uk);
  return status;
}

void oracle_apply_step(int64_t n_cams, int64_t n_pts, const double* cams, const double* pts,
                       const double* dc, const double* dp, double* cams_out, double* pts_out) {
  for (int64_t c = 0; c < n_cams; ++c) {
    double w[3];
    oracle_rotvec_compose(dc + 9 * c, cams + 9 * c, w);
    cams_out[9 * c + 0] = w[0];
    cams_out[9 * c + 1] = w[1];
    cams_out[9 * c + 2] = w[2];
    for (int i = 3; i < 9; ++i) cams_out[9 * c + i] = cams[9 * c + i] + dc[9 * c + i];
  }
  for (int64_t i = 0; i < 3 * n_pts; ++i) pts_out[i] = pts[i] + dp[i];
}

/* ------------------------------------------------------------------------- */
/* LM loop (Sec. 3.3) with dynamic parameter extraction every iteration        */
/* ------------------------------------------------------------------------- */

/* Gain-ratio test of Sec. 3.3's LM loop.  The paper names Marquardt damping but
 * not its control; the reading is Nielsen's rule as given by Madsen, Nielsen and
 * Tingleff, "Methods for non-linear least squares problems" (2004), Sec. 3.2:
 * gain = (F(x) - F(x + h)) / (L(0) - L(h)); the step is taken when the gain is
 * positive; here "positive" is gain > 1e-3, and a non-finite candidate cost or
 * a non-positive predicted decrease rejects. */
int oracle_lm_accept(double F, double Fc, double pred) {
  double gain = (F - Fc) / pred;
  return isfinite(Fc) && isfinite(gain) && pred > 0.0 && gain > 1e-3;
}

/* Nielsen's damping update (same source, Eq. 2.21 and Algorithm 3.16):
 * accepted: mu <- mu * max(1/3, 1 - (2 gain - 1)^3), nu <- 2;
 * rejected: mu <- mu * nu, nu <- 2 nu. */
void oracle_lm_damping(int accepted, double gain, double* lambda, double* nu) {
  if (accepted) {
    double t = 2.0 * gain - 1.0;
    double f = 1.0 - t * t * t;
    *lambda *= f > 1.0 / 3.0 ? f : 1.0 / 3.0;
    *nu = 2.0;
  } else {
    *lambda *= *nu;
    *nu *= 2.0;
  }
}

int oracle_lm(const oracle_problem* pb, const oracle_opts* o, int max_iters, double* cams,
              double* pts, oracle_iter_log* log, uint8_t* alive_io) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  size_t n1 = (size_t)(N > 0 ? N : 1);
  uint8_t* alive = alive_io ? alive_io : (uint8_t*)malloc(n1);
  if (!alive_io) memset(alive, 1, n1);
  uint8_t* geom = (uint8_t*)malloc(n1);
  uint8_t* valid = (uint8_t*)malloc(n1);
  uint8_t* obs_mask = (uint8_t*)malloc(n1);
  double* res = (double*)malloc(sizeof(double) * n1);
  uint8_t* cam_mask = (uint8_t*)malloc((size_t)C + 1);
  uint8_t* pt_mask = (uint8_t*)malloc((size_t)P + 1);
  int32_t* cam_rank = (int32_t*)malloc(sizeof(int32_t) * ((size_t)C + 1));
  int32_t* pt_rank = (int32_t*)malloc(sizeof(int32_t) * ((size_t)P + 1));
  double* U = (double*)malloc(sizeof(double) * 81 * ((size_t)C + 1));
  double* V = (double*)malloc(sizeof(double) * 9 * ((size_t)P + 1));
  double* W = (double*)malloc(sizeof(double) * 27 * n1);
  double* gc = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* gp = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));
  double* dc = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* dp = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));
  double* cams2 = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* pts2 = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));

  double lambda = o->lambda0, nu = o->nu0 > 0.0 ? o->nu0 : 2.0;
  int state_changed = 1;
  int64_t n_cam_free = 0, n_pt_act = 0;
  double F = 0.0, rmse = 0.0;
  int it;
  for (it = 0; it < max_iters; ++it) {
    /* one-shot mode: validity, drop and peeling at the first iteration only,
     * the active set frozen afterwards (the static pruning Sec. 4.2 contrasts
     * with its per-iteration extraction) */
    int once = o->extract_mode == 1;
    int drop_now = !once && o->extract_every > 0 && o->drop_residual_px > 0.0 && it > 0 &&
                   it % o->extract_every == 0;
    int relin = state_changed || drop_now || it == 0;
    if (relin && (!once || it == 0)) {
      /* Sec. 4.2 step 1: re-evaluate validity with the current state */
      oracle_predicate(pb, o, cams, pts, geom, res);
      if (drop_now) /* reading: sticky residual drop of geometrically valid observations */
        for (int64_t k = 0; k < N; ++k)
          if (geom[k] && res[k] > o->drop_residual_px) alive[k] = 0;
      for (int64_t k = 0; k < N; ++k) valid[k] = (uint8_t)(alive[k] && geom[k]);
      /* step 2: active sets and ranks */
      oracle_extract(pb, o, valid, cam_mask, pt_mask, obs_mask, cam_rank, pt_rank, &n_cam_free,
                     &n_pt_act);
    }
    if (relin) {
      F = oracle_cost(pb, o, cams, pts, obs_mask, &rmse);
      oracle_normal_equations(pb, o, cams, pts, obs_mask, U, V, W, gc, gp);
    }
    double pred = 0.0, relres = 0.0;
    int st = oracle_solve_step(pb, o, U, V, W, gc, gp, obs_mask, cam_rank, pt_rank, n_cam_free,
                               lambda, dc, dp, &pred, &relres);
    double Fc = NAN, gain = NAN;
    int accepted = 0;
    if (st >= 0) {
      /* step 3: scatter back, inactive parameters unchanged */
      oracle_apply_step(C, P, cams, pts, dc, dp, cams2, pts2);
      Fc = oracle_cost(pb, o, cams2, pts2, obs_mask, NULL);
      gain = (F - Fc) / pred;
      accepted = oracle_lm_accept(F, Fc, pred);
    }
    if (log) {
      oracle_iter_log* L = log + it;
      int64_t na = 0;
      for (int64_t k = 0; k < N; ++k) na += obs_mask[k];
      int64_t nc = 0;
      for (int64_t c = 0; c < C; ++c) nc += cam_mask[c];
      L->cost = F;
      L->rmse_px = rmse;
      L->lambda = lambda;
      L->gain = gain;
      L->pred_decrease = pred;
      L->cand_cost = Fc;
      L->accepted = accepted;
      L->pcg_iters = st > 0 ? st : 0;
      L->pcg_rel_res = relres;
      L->n_cam_act = nc;
      L->n_pt_act = n_pt_act;
      L->n_obs_act = na;
    }
    oracle_lm_damping(accepted, gain, &lambda, &nu);
    if (accepted) {
      memcpy(cams, cams2, sizeof(double) * 9 * (size_t)C);
      memcpy(pts, pts2, sizeof(double) * 3 * (size_t)P);
      state_changed = 1;
    } else {
      state_changed = 0;
    }
  }
  if (!alive_io) free(alive);
  free(geom);
  free(valid);
  free(obs_mask);
  free(res);
  free(cam_mask);
  free(pt_mask);
  free(cam_rank);
  free(pt_rank);
  free(U);
  free(V);
  free(W);
  free(gc);
  free(gp);
  free(dc);
  free(dp);
  free(cams2);
  free(pts2);
  return it;
}

/* ------------------------------------------------------------------------- */
/* implicit adjoint                                                           */
/* ------------------------------------------------------------------------- */

/* At the optimum the robust gradient sum_k rho'_k J_k^T r_k vanishes.  Reading:
 * with IRLS weights and the active set frozen and the Gauss-Newton matrix H
 * standing in for the Hessian, the implicit function theorem gives
 * dL/dy = -mu^T dg/dy with H mu = dL/dtheta.  For the stacked residual,
 * dr/du_k = -e_0, dr/dv_k = -e_1, dr/dd_k = sqrt(w) m / d^2 e_2, hence
 * dL/du_k = rho'_k (J_k mu)_0, dL/dv_k = rho'_k (J_k mu)_1,
 * dL/dd_k = -rho'_k sqrt(w) m / d^2 (J_k mu)_2. */
/* Inverse left Jacobian of SO(3) at w: the LM update w <- Log(Exp(dw) Exp(w))
 * has d w / d dw = Jl(w)^-1 at dw = 0, with
 *   Jl^-1 = I - W/2 + (1/th^2 - (1 + cos th) / (2 th sin th)) W^2,  W = [w]x,
 * and the series 1/12 + th^2/720 of the last coefficient near th = 0. */
void oracle_so3_left_jacobian_inv(const double w[3], double J[9]) {
  double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double th = sqrt(th2);
  double c2 = th < 1e-4 ? 1.0 / 12.0 + th2 / 720.0 : 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
  double Wm[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double w2 = 0.0;
      for (int k = 0; k < 3; ++k) w2 += Wm[3 * i + k] * Wm[3 * k + j];
      J[3 * i + j] = (i == j ? 1.0 : 0.0) - 0.5 * Wm[3 * i + j] + c2 * w2;
    }
}

int oracle_backward(const oracle_problem* pb, const oracle_opts* o, const double* cams,
                    const double* pts, const uint8_t* obs_mask, const int32_t* cam_rank,
                    const int32_t* pt_rank, int64_t n_cam_free, const double* dL_dcams,
                    const double* dL_dpts, double* dL_duv, double* dL_ddepth) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  size_t n1 = (size_t)(N > 0 ? N : 1);
  double* U = (double*)malloc(sizeof(double) * 81 * ((size_t)C + 1));
  double* V = (double*)malloc(sizeof(double) * 9 * ((size_t)P + 1));
  double* W = (double*)malloc(sizeof(double) * 27 * n1);
  double* gc = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* gp = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));
  double* mc = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* mp = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));
  oracle_normal_equations(pb, o, cams, pts, obs_mask, U, V, W, gc, gp);
  /* Solve the undamped system H mu = a with the Schur complement: the same
   * routine as the LM step with lambda = 0 and g := -a. */
  double* ac = (double*)malloc(sizeof(double) * 9 * ((size_t)C + 1));
  double* ap = (double*)malloc(sizeof(double) * 3 * ((size_t)P + 1));
  /* dL_dcams is the gradient in the stored parameters; the solve runs in the
   * update's coordinates, where the rotation block is Jl(w)^-T dL/dw. */
  for (int64_t c = 0; c < C; ++c) {
    double J[9];
    oracle_so3_left_jacobian_inv(cams + 9 * c, J);
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += J[3 * j + i] * dL_dcams[9 * c + j];
      ac[9 * c + i] = -acc;
    }
    for (int i = 3; i < 9; ++i) ac[9 * c + i] = -dL_dcams[9 * c + i];
    if (o->camera_model == 1) ac[9 * c + 7] = ac[9 * c + 8] = 0.0;  /* not parameters */
  }
  for (int64_t i = 0; i < 3 * P; ++i) ap[i] = -dL_dpts[i];
  oracle_opts od = *o;
  od.solver = 0;
  double pred, rr;
  int st = oracle_solve_step(pb, &od, U, V, W, ac, ap, obs_mask, cam_rank, pt_rank, n_cam_free,
                             0.0, mc, mp, &pred, &rr);
  if (st >= 0) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k) {
      dL_duv[2 * k] = 0.0;
      dL_duv[2 * k + 1] = 0.0;
      dL_ddepth[k] = 0.0;
      if (!obs_mask[k]) continue;
      int c = pb->obs_cam[k], p = pb->obs_pt[k];
      double d = pb->depth[k];
      double r[3], Jc[27], Jp[9];
      double wt = depth_wt(o, d);
      oracle_observe_model(o->camera_model, cams + 9 * (int64_t)c, pts + 3 * (int64_t)p, pb->obs_uv + 2 * k,
                     depth_tau(d), wt, o->cx, o->cy, r, Jc, Jp, NULL, NULL);
      double s = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      double rw = huber_w(s, o->huber_delta);
      double Jm[3];
      for (int m = 0; m < 3; ++m) {
        double acc = 0;
        if (cam_rank[c] >= 0)
          for (int i = 0; i < 9; ++i) acc += Jc[9 * m + i] * mc[9 * (int64_t)c + i];
        for (int i = 0; i < 3; ++i) acc += Jp[3 * m + i] * mp[3 * (int64_t)p + i];
        Jm[m] = acc;
      }
      dL_duv[2 * k] = rw * Jm[0];
      dL_duv[2 * k + 1] = rw * Jm[1];
      if (has_prior(d)) dL_ddepth[k] = -rw * sqrt(wt) / (d * d) * Jm[2];
    }
  }
  free(U);
  free(V);
  free(W);
  free(gc);
  free(gp);
  free(mc);
  free(mp);
  free(ac);
  free(ap);
  return st < 0 ? -1 : 0;
}
