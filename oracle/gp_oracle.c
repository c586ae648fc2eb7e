/* gp_oracle.c -- plain FP64 reference of the depth-constrained global positioning
 * LM (Sec. 3.1 Eq. GP objective, Sec. 4.1 GP paragraph, Sec. 3.3 Eq. LM).
 * TEST INFRASTRUCTURE ONLY; see gp_oracle.h.
 *
 * Every step runs in the order the method states it: residuals and Jacobians,
 * robust-weighted normal equations, Marquardt damping of the full system, then
 * the exact solve of the damped system by eliminating the free scales (each
 * couples to one camera and one point only), then the points, leaving the dense
 * camera-centre system, factored by Cholesky; back-substitution; candidate; gain
 * ratio; damping update.  Sums run in a fixed order (observations ascending). */
#include "gp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int gp_has_prior(double d) { return d > 0.0 && isfinite(d); }

/* Huber on the squared norm, as in the BA oracle (reading: rho acts on |u|^2). */
static double gp_rho(double s, double delta) {
  if (delta <= 0.0 || s <= delta * delta) return s;
  return 2.0 * delta * sqrt(s) - delta * delta;
}
static double gp_w(double s, double delta) {
  if (delta <= 0.0 || s <= delta * delta) return 1.0;
  return delta / sqrt(s);
}

/* Marquardt diagonal, clamped as in the BA oracle. */
static double gp_clamp(double d) { return d < 1e-6 ? 1e-6 : (d > 1e32 ? 1e32 : d); }

void oracle_gp_residual(const double t[3], const double X[3], const double v[3], double s,
                        double u[3], double Jt[9], double JX[9], double Js[3]) {
  double e[3] = {X[0] - t[0], X[1] - t[1], X[2] - t[2]};
  for (int i = 0; i < 3; ++i) u[i] = v[i] - s * e[i];
  if (Jt)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Jt[3 * i + j] = i == j ? s : 0.0;
  if (JX)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) JX[3 * i + j] = i == j ? -s : 0.0;
  if (Js)
    for (int i = 0; i < 3; ++i) Js[i] = -e[i];
}

int64_t oracle_gp_free_set(const oracle_gp_problem* pb, int32_t* free_rank) {
  int64_t n = 0;
  for (int64_t k = 0; k < pb->n_obs; ++k) free_rank[k] = gp_has_prior(pb->depth[k]) ? -1 : (int32_t)n++;
  return n;
}

double oracle_gp_scale(const oracle_gp_problem* pb, const double* scales, int64_t k) {
  double d = pb->depth[k];
  return gp_has_prior(d) ? 1.0 / d : scales[k];
}

double oracle_gp_cost(const oracle_gp_problem* pb, const oracle_gp_opts* o, const double* centres,
                      const double* pts, const double* scales, double* rms) {
  double F = 0.0, E = 0.0;
  for (int64_t k = 0; k < pb->n_obs; ++k) {
    double u[3];
    oracle_gp_residual(centres + 3 * (int64_t)pb->obs_cam[k], pts + 3 * (int64_t)pb->obs_pt[k],
                       pb->rays + 3 * k, oracle_gp_scale(pb, scales, k), u, NULL, NULL, NULL);
    double s = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    F += gp_rho(s, o->huber_delta);
    E += s;
  }
  if (rms) *rms = pb->n_obs > 0 ? sqrt(E / (double)pb->n_obs) : 0.0;
  return 0.5 * F;
}

void oracle_gp_normal_equations(const oracle_gp_problem* pb, const oracle_gp_opts* o,
                                const double* centres, const double* pts, const double* scales,
                                double* U, double* V, double* W, double* Hts, double* HXs,
                                double* Q, double* gt, double* gX, double* gs) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  memset(U, 0, sizeof(double) * 9 * (size_t)C);
  memset(V, 0, sizeof(double) * 9 * (size_t)P);
  memset(gt, 0, sizeof(double) * 3 * (size_t)C);
  memset(gX, 0, sizeof(double) * 3 * (size_t)P);
  for (int64_t k = 0; k < N; ++k) {
    int c = pb->obs_cam[k], p = pb->obs_pt[k];
    int pinned = gp_has_prior(pb->depth[k]);
    double u[3], Jt[9], JX[9], Js[3];
    oracle_gp_residual(centres + 3 * (int64_t)c, pts + 3 * (int64_t)p, pb->rays + 3 * k,
                       oracle_gp_scale(pb, scales, k), u, Jt, JX, Js);
    double w = gp_w(u[0] * u[0] + u[1] * u[1] + u[2] * u[2], o->huber_delta);
    /* J^T w J and J^T w u, block by block (J rows are the 3 residual components) */
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) {
        double utt = 0.0, uxx = 0.0, utx = 0.0;
        for (int m = 0; m < 3; ++m) {
          utt += Jt[3 * m + a] * w * Jt[3 * m + b];
          uxx += JX[3 * m + a] * w * JX[3 * m + b];
          utx += Jt[3 * m + a] * w * JX[3 * m + b];
        }
        U[9 * (int64_t)c + 3 * a + b] += utt;
        V[9 * (int64_t)p + 3 * a + b] += uxx;
        W[9 * k + 3 * a + b] = utx;
      }
      double g1 = 0.0, g2 = 0.0, h1 = 0.0, h2 = 0.0;
      for (int m = 0; m < 3; ++m) {
        g1 += Jt[3 * m + a] * w * u[m];
        g2 += JX[3 * m + a] * w * u[m];
        h1 += Jt[3 * m + a] * w * Js[m];
        h2 += JX[3 * m + a] * w * Js[m];
      }
      gt[3 * (int64_t)c + a] += g1;
      gX[3 * (int64_t)p + a] += g2;
      Hts[3 * k + a] = pinned ? 0.0 : h1;
      HXs[3 * k + a] = pinned ? 0.0 : h2;
    }
    double q = 0.0, g = 0.0;
    for (int m = 0; m < 3; ++m) {
      q += Js[m] * w * Js[m];
      g += Js[m] * w * u[m];
    }
    Q[k] = pinned ? 0.0 : q;
    gs[k] = pinned ? 0.0 : g;
  }
}

/* 3x3 inverse by the adjugate (symmetric positive definite input). */
static int inv3(const double A[9], double B[9]) {
  double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (!(det > 0.0) || !isfinite(det)) return -1;
  double id = 1.0 / det;
  B[0] = c00 * id;
  B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  B[3] = c01 * id;
  B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  B[6] = c02 * id;
  B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return 0;
}

/* In-place Cholesky A = L L^T (lower, row-major n x n) and solve L L^T x = b. */
static int chol_solve(double* A, int64_t n, double* b) {
  for (int64_t j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    A[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= A[i * n + k] * b[k];
    b[i] = s / A[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int64_t k = i + 1; k < n; ++k) s -= A[k * n + i] * b[k];
    b[i] = s / A[i * n + i];
  }
  return 0;
}

int oracle_gp_solve_step(const oracle_gp_problem* pb, const oracle_gp_opts* o, const double* centres,
                         const double* pts, const double* scales, double lambda, double* dt,
                         double* dX, double* ds, double* pred_decrease) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  size_t c1 = (size_t)C + 1, p1 = (size_t)P + 1, n1 = (size_t)N + 1;
  double* U = malloc(sizeof(double) * 9 * c1);
  double* V = malloc(sizeof(double) * 9 * p1);
  double* W = malloc(sizeof(double) * 9 * n1);
  double* Hts = malloc(sizeof(double) * 3 * n1);
  double* HXs = malloc(sizeof(double) * 3 * n1);
  double* Q = malloc(sizeof(double) * n1);
  double* gt = malloc(sizeof(double) * 3 * c1);
  double* gX = malloc(sizeof(double) * 3 * p1);
  double* gs = malloc(sizeof(double) * n1);
  oracle_gp_normal_equations(pb, o, centres, pts, scales, U, V, W, Hts, HXs, Q, gt, gX, gs);

  /* unknowns: centres of non-gauge cameras with observations, points with
   * observations, free scales */
  int32_t* cam_rank = malloc(sizeof(int32_t) * c1);
  int* cam_nobs = calloc(c1, sizeof(int));
  int* pt_nobs = calloc(p1, sizeof(int));
  for (int64_t k = 0; k < N; ++k) {
    cam_nobs[pb->obs_cam[k]]++;
    pt_nobs[pb->obs_pt[k]]++;
  }
  int64_t Cf = 0;
  for (int64_t c = 0; c < C; ++c) cam_rank[c] = (!pb->fixed[c] && cam_nobs[c] > 0) ? (int32_t)Cf++ : -1;

  /* Eq. LM: damped system H + lambda D, D = clamp(diag H) of the full system */
  double* Us = malloc(sizeof(double) * 9 * c1);
  double* Vs = malloc(sizeof(double) * 9 * p1);
  double* Ws = malloc(sizeof(double) * 9 * n1);
  double* Qs = malloc(sizeof(double) * n1);
  double* gtr = malloc(sizeof(double) * 3 * c1);
  double* gXr = malloc(sizeof(double) * 3 * p1);
  memcpy(Us, U, sizeof(double) * 9 * (size_t)C);
  memcpy(Vs, V, sizeof(double) * 9 * (size_t)P);
  memcpy(Ws, W, sizeof(double) * 9 * (size_t)N);
  memcpy(gtr, gt, sizeof(double) * 3 * (size_t)C);
  memcpy(gXr, gX, sizeof(double) * 3 * (size_t)P);
  for (int64_t c = 0; c < C; ++c)
    for (int i = 0; i < 3; ++i) Us[9 * c + 4 * i] += lambda * gp_clamp(U[9 * c + 4 * i]);
  for (int64_t p = 0; p < P; ++p)
    for (int i = 0; i < 3; ++i) Vs[9 * p + 4 * i] += lambda * gp_clamp(V[9 * p + 4 * i]);
  for (int64_t k = 0; k < N; ++k) Qs[k] = gp_has_prior(pb->depth[k]) ? 0.0 : Q[k] + lambda * gp_clamp(Q[k]);

  /* eliminate each free scale: it couples only to its camera and its point */
  for (int64_t k = 0; k < N; ++k) {
    if (gp_has_prior(pb->depth[k])) continue;
    int c = pb->obs_cam[k], p = pb->obs_pt[k];
    const double* a = Hts + 3 * k;
    const double* b = HXs + 3 * k;
    double q = Qs[k];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        Us[9 * (int64_t)c + 3 * i + j] -= a[i] * a[j] / q;
        Vs[9 * (int64_t)p + 3 * i + j] -= b[i] * b[j] / q;
        Ws[9 * k + 3 * i + j] -= a[i] * b[j] / q;
      }
      gtr[3 * (int64_t)c + i] -= a[i] * gs[k] / q;
      gXr[3 * (int64_t)p + i] -= b[i] * gs[k] / q;
    }
  }

  /* eliminate the points: S = Us - sum W Vs^-1 W^T, rhs = -gt + sum W Vs^-1 gX */
  int status = 0;
  double* Vinv = malloc(sizeof(double) * 9 * p1);
  for (int64_t p = 0; p < P; ++p) {
    if (pt_nobs[p] == 0) {
      memset(Vinv + 9 * p, 0, sizeof(double) * 9);
      continue;
    }
    if (inv3(Vs + 9 * p, Vinv + 9 * p) != 0) status = -1;
  }
  /* observations of each point, ascending */
  int64_t* off = calloc(p1 + 1, sizeof(int64_t));
  int64_t* byp = malloc(sizeof(int64_t) * n1);
  for (int64_t k = 0; k < N; ++k) off[pb->obs_pt[k] + 1]++;
  for (int64_t p = 0; p < P; ++p) off[p + 1] += off[p];
  int64_t* fill = malloc(sizeof(int64_t) * p1);
  for (int64_t p = 0; p < P; ++p) fill[p] = off[p];
  for (int64_t k = 0; k < N; ++k) byp[fill[pb->obs_pt[k]]++] = k;

  int64_t n = 3 * Cf;
  double* S = calloc((size_t)(n > 0 ? n * n : 1), sizeof(double));
  double* rhs = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int64_t c = 0; c < C; ++c) {
    int r = cam_rank[c];
    if (r < 0) continue;
    for (int i = 0; i < 3; ++i) {
      rhs[3 * r + i] = -gtr[3 * c + i];
      for (int j = 0; j < 3; ++j) S[(3 * r + i) * n + 3 * r + j] = Us[9 * c + 3 * i + j];
    }
  }
  for (int64_t p = 0; p < P && status == 0; ++p) {
    const double* Vi = Vinv + 9 * p;
    for (int64_t a = off[p]; a < off[p + 1]; ++a) {
      int64_t k = byp[a];
      int r = cam_rank[pb->obs_cam[k]];
      if (r < 0) continue;
      double WV[9];  /* W_k Vinv_p */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
          for (int m = 0; m < 3; ++m) s += Ws[9 * k + 3 * i + m] * Vi[3 * m + j];
          WV[3 * i + j] = s;
        }
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += WV[3 * i + m] * gXr[3 * p + m];
        rhs[3 * r + i] += s;
      }
      for (int64_t b2 = off[p]; b2 < off[p + 1]; ++b2) {
        int64_t k2 = byp[b2];
        int r2 = cam_rank[pb->obs_cam[k2]];
        if (r2 < 0) continue;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int m = 0; m < 3; ++m) s += WV[3 * i + m] * Ws[9 * k2 + 3 * j + m];
            S[(3 * r + i) * n + 3 * r2 + j] -= s;
          }
      }
    }
  }
  if (status == 0 && n > 0) status = chol_solve(S, n, rhs);

  memset(dt, 0, sizeof(double) * 3 * (size_t)C);
  memset(dX, 0, sizeof(double) * 3 * (size_t)P);
  memset(ds, 0, sizeof(double) * (size_t)N);
  double pred = 0.0;
  if (status == 0) {
    for (int64_t c = 0; c < C; ++c)
      if (cam_rank[c] >= 0)
        for (int i = 0; i < 3; ++i) dt[3 * c + i] = rhs[3 * cam_rank[c] + i];
    /* points: dX = Vs^-1 (-gX' - sum W^T dt) */
    for (int64_t p = 0; p < P; ++p) {
      if (pt_nobs[p] == 0) continue;
      double r[3] = {-gXr[3 * p], -gXr[3 * p + 1], -gXr[3 * p + 2]};
      for (int64_t a = off[p]; a < off[p + 1]; ++a) {
        int64_t k = byp[a];
        const double* d = dt + 3 * (int64_t)pb->obs_cam[k];
        for (int i = 0; i < 3; ++i)
          for (int m = 0; m < 3; ++m) r[i] -= Ws[9 * k + 3 * m + i] * d[m];
      }
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += Vinv[9 * p + 3 * i + m] * r[m];
        dX[3 * p + i] = s;
      }
    }
    /* free scales: ds = (-gs - Hts^T dt - HXs^T dX) / Qs */
    for (int64_t k = 0; k < N; ++k) {
      if (gp_has_prior(pb->depth[k])) continue;
      const double* d1 = dt + 3 * (int64_t)pb->obs_cam[k];
      const double* d2 = dX + 3 * (int64_t)pb->obs_pt[k];
      double s = -gs[k];
      for (int i = 0; i < 3; ++i) s -= Hts[3 * k + i] * d1[i] + HXs[3 * k + i] * d2[i];
      ds[k] = s / Qs[k];
    }
    /* predicted decrease 1/2 dx^T (lambda D dx - g) over every unknown */
    for (int64_t c = 0; c < C; ++c) {
      if (cam_rank[c] < 0) continue;
      for (int i = 0; i < 3; ++i)
        pred += 0.5 * dt[3 * c + i] * (lambda * gp_clamp(U[9 * c + 4 * i]) * dt[3 * c + i] - gt[3 * c + i]);
    }
    for (int64_t p = 0; p < P; ++p) {
      if (pt_nobs[p] == 0) continue;
      for (int i = 0; i < 3; ++i)
        pred += 0.5 * dX[3 * p + i] * (lambda * gp_clamp(V[9 * p + 4 * i]) * dX[3 * p + i] - gX[3 * p + i]);
    }
    for (int64_t k = 0; k < N; ++k) {
      if (gp_has_prior(pb->depth[k])) continue;
      pred += 0.5 * ds[k] * (lambda * gp_clamp(Q[k]) * ds[k] - gs[k]);
    }
  }
  if (pred_decrease) *pred_decrease = pred;
  free(U); free(V); free(W); free(Hts); free(HXs); free(Q); free(gt); free(gX); free(gs);
  free(cam_rank); free(cam_nobs); free(pt_nobs);
  free(Us); free(Vs); free(Ws); free(Qs); free(gtr); free(gXr); free(Vinv);
  free(off); free(byp); free(fill); free(S); free(rhs);
  return status;
}

int oracle_gp_lm(const oracle_gp_problem* pb, const oracle_gp_opts* o, int max_iters, double* centres,
                 double* pts, double* scales, oracle_iter_log* log) {
  int64_t C = pb->n_cams, P = pb->n_pts, N = pb->n_obs;
  size_t c1 = (size_t)C + 1, p1 = (size_t)P + 1, n1 = (size_t)N + 1;
  double* dt = malloc(sizeof(double) * 3 * c1);
  double* dX = malloc(sizeof(double) * 3 * p1);
  double* ds = malloc(sizeof(double) * n1);
  double* t2 = malloc(sizeof(double) * 3 * c1);
  double* X2 = malloc(sizeof(double) * 3 * p1);
  double* s2 = malloc(sizeof(double) * n1);
  int32_t* fr = malloc(sizeof(int32_t) * n1);
  int64_t n_free = oracle_gp_free_set(pb, fr);
  int64_t ncf = 0, npa = 0;
  {
    int* cn = calloc(c1, sizeof(int));
    int* pn = calloc(p1, sizeof(int));
    for (int64_t k = 0; k < N; ++k) {
      cn[pb->obs_cam[k]]++;
      pn[pb->obs_pt[k]]++;
    }
    for (int64_t c = 0; c < C; ++c) ncf += !pb->fixed[c] && cn[c] > 0;
    for (int64_t p = 0; p < P; ++p) npa += pn[p] > 0;
    free(cn);
    free(pn);
  }
  double lambda = o->lambda0, nu = 2.0;
  double rms = 0.0;
  double F = oracle_gp_cost(pb, o, centres, pts, scales, &rms);
  int it;
  for (it = 0; it < max_iters; ++it) {
    double pred = 0.0;
    int st = oracle_gp_solve_step(pb, o, centres, pts, scales, lambda, dt, dX, ds, &pred);
    double Fc = NAN, gain = NAN, rms_c = 0.0;
    int accepted = 0;
    if (st == 0) {
      for (int64_t i = 0; i < 3 * C; ++i) t2[i] = centres[i] + dt[i];
      for (int64_t i = 0; i < 3 * P; ++i) X2[i] = pts[i] + dX[i];
      for (int64_t k = 0; k < N; ++k) s2[k] = scales[k] + ds[k];
      Fc = oracle_gp_cost(pb, o, t2, X2, s2, &rms_c);
      gain = (F - Fc) / pred;
      accepted = oracle_lm_accept(F, Fc, pred);
    }
    if (log) {
      oracle_iter_log* L = log + it;
      memset(L, 0, sizeof *L);
      L->cost = F;
      L->rmse_px = rms;
      L->lambda = lambda;
      L->gain = gain;
      L->pred_decrease = pred;
      L->cand_cost = Fc;
      L->accepted = accepted;
      L->n_cam_act = ncf;
      L->n_pt_act = npa;
      L->n_obs_act = n_free;
    }
    oracle_lm_damping(accepted, gain, &lambda, &nu);
    if (accepted) {
      memcpy(centres, t2, sizeof(double) * 3 * (size_t)C);
      memcpy(pts, X2, sizeof(double) * 3 * (size_t)P);
      for (int64_t k = 0; k < N; ++k)
        if (fr[k] >= 0) scales[k] = s2[k];
      F = Fc;
      rms = rms_c;
    }
  }
  free(dt); free(dX); free(ds); free(t2); free(X2); free(s2); free(fr);
  return it;
}
