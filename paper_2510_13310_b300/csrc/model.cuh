// model.cuh -- device camera model: residuals and Jacobian blocks of one observation.
//
// Reprojection residual of Eq. (BA objective) (Sec. 3.2) with the 9-parameter
// radial camera, stacked with the inverse-depth residual of Sec. 4.1,
// r_d = 1/Depth - m/d, into r = [u^ - u, v^ - v, sqrt(w) r_d].  The camera block
// uses the left rotation increment: dP/d(dw) = -[R X]x, dP/dt = I; the point
// block is dP/dX = R.
//
// Camera models, both in the nine slots [w, t or c, f, k1, k2] of a camera and
// projected through one working record (R, t, f, k1, k2, model):
//   0 (radial):  P = R X + t, distortion 1 + k1 rr + k2 rr^2;
//   1 (Sec. 3.2's parameterisation: centre, rotation, focal length):
//                P = R (X - c), no distortion; the record holds t = -R c and
//                k1 = k2 = 0, the Jacobian has dP/d(dw) = -[P]x, dP/dc = -R and
//                no k1, k2 columns.
#pragma once
#include "common.cuh"

namespace bab {

template <typename T>
struct ObsLin {
  T r[3];
  T Jc[3][9];
  T Jp[3][3];
  T wrob;   // IRLS weight rho'(|r|^2) of the Huber loss
  // what both blocks are built from (the observation record of the explicit
  // system's formation): D = d r / d P (D10 = D01, D20 = D21 = 0), the point a the
  // rotation increment acts on, the normalised image point
  T D00, D01, D02, D11, D12, D22, a0, a1, a2, xn, yn;
};

// Huber weight on the squared norm s: 1 inside, delta / sqrt(s) outside.
template <typename T>
__device__ __forceinline__ T huber_weight(T s, T delta) {
  if (delta <= T(0) || s <= delta * delta) return T(1);
  return delta / sqrt(s);
}
// FP64 division and square root are scarce on B300 (a dependent DDIV costs
// ~400 cycles).  The FP64 evaluation therefore uses Newton-Raphson refinement of
// FP32 seeds: for 1/a, x <- x + x (1 - a x), each step doubling the correct
// bits (2^-23 -> 2^-46 -> rounding level); for 1/sqrt(s), y <- y (3 - s y^2) / 2
// twice, then sqrt(s) = s y with one Newton correction r <- r + (s - r^2) y / 2.
// Results are within a few ulp of the correctly rounded values.  Arguments
// outside the FP32 exponent range fall back to the FP64 operations.
// Comparisons on the integer pipe: for non-NaN doubles the IEEE order equals the
// signed order of dkey (+0 and -0 both map to 0).  A NaN gets a key beyond every
// finite value of its sign, so every predicate below that brackets a value from
// both sides (0 <= u < W) is false for it, as with IEEE comparisons.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFll);
}
// |a| within [2^-100, 2^100] (exponent field test, no FP64 instruction)
__device__ __forceinline__ bool fp32_range(double a) {
  const int e = (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF;
  return e >= 1023 - 100 && e <= 1023 + 100;
}

__device__ __forceinline__ double recip_nr(double a) {
  if (!fp32_range(a)) return 1.0 / a;
  double x = (double)__frcp_rn((float)a);
  x = fma(x, fma(-a, x, 1.0), x);
  x = fma(x, fma(-a, x, 1.0), x);
  return x;
}
__device__ __forceinline__ double sqrt_nr(double s) {
  if (__double_as_longlong(s) < 0 || !fp32_range(s)) return sqrt(s);
  double y = (double)rsqrtf((float)s);
  const double hs = 0.5 * s;
  y = y * fma(-hs * y, y, 1.5);
  y = y * fma(-hs * y, y, 1.5);
  const double r = s * y;
  return fma(fma(-r, r, s), 0.5 * y, r);
}

// Huber loss on the squared norm s (s >= 0 or NaN; the threshold test on the
// integer pipe).
__device__ __forceinline__ double huber_loss(double s, double delta) {
  if (delta <= 0.0 || dkey(s) <= dkey(delta * delta)) return s;
  return 2.0 * delta * sqrt_nr(s) - delta * delta;
}

// cw: working camera record (R row-major, t, f, k1, k2).
template <typename T>
__device__ __forceinline__ void linearize_obs(const T* __restrict__ cw, T X0, T X1, T X2, T u,
                                              T v, T tau, T sw, T cx, T cy, T delta,
                                              ObsLin<T>& o) {
  const T* R = cw;
  T a0 = R[0] * X0 + R[1] * X1 + R[2] * X2;  // a = R X
  T a1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
  T a2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
  T px = a0 + cw[9], py = a1 + cw[10], pz = a2 + cw[11];
  T f = cw[12], k1 = cw[13], k2 = cw[14];
  T iz = T(1) / pz;
  T xn = px * iz, yn = py * iz;
  T rr = xn * xn + yn * yn;
  T dist = T(1) + rr * (k1 + k2 * rr);
  T fd = f * dist;
  o.r[0] = fd * xn + cx - u;
  o.r[1] = fd * yn + cy - v;
  o.r[2] = sw * (iz - tau);
  T s = o.r[0] * o.r[0] + o.r[1] * o.r[1] + o.r[2] * o.r[2];
  o.wrob = huber_weight(s, delta);

  // D = d r / d P (rows u, v, depth)
  T g = T(2) * f * (k1 + T(2) * k2 * rr);  // f * d dist / d rr * 2
  T dxz = -xn * iz, dyz = -yn * iz;         // d xn / d pz, d yn / d pz
  // d rr / dP = 2 (xn iz, yn iz, -rr iz)
  T D00 = fd * iz + g * xn * xn * iz;
  T D01 = g * xn * yn * iz;
  T D02 = fd * dxz - g * xn * rr * iz;
  T D10 = D01;
  T D11 = fd * iz + g * yn * yn * iz;
  T D12 = fd * dyz - g * yn * rr * iz;
  T D22 = -sw * iz * iz;

  // model 1: the rotation increment acts on R (X - c) = P
  if (cw[15] != T(0)) a0 = px, a1 = py, a2 = pz;
  o.D00 = D00, o.D01 = D01, o.D02 = D02, o.D11 = D11, o.D12 = D12, o.D22 = D22;
  o.a0 = a0, o.a1 = a1, o.a2 = a2, o.xn = xn, o.yn = yn;
  // rotation columns: D * (-[a]x) with -[a]x = [[0,a2,-a1],[-a2,0,a0],[a1,-a0,0]]
  o.Jc[0][0] = -D01 * a2 + D02 * a1;
  o.Jc[0][1] = D00 * a2 - D02 * a0;
  o.Jc[0][2] = -D00 * a1 + D01 * a0;
  o.Jc[1][0] = -D11 * a2 + D12 * a1;
  o.Jc[1][1] = D10 * a2 - D12 * a0;
  o.Jc[1][2] = -D10 * a1 + D11 * a0;
  o.Jc[2][0] = D22 * a1;
  o.Jc[2][1] = -D22 * a0;
  o.Jc[2][2] = T(0);
  // translation columns: D
  o.Jc[0][3] = D00; o.Jc[0][4] = D01; o.Jc[0][5] = D02;
  o.Jc[1][3] = D10; o.Jc[1][4] = D11; o.Jc[1][5] = D12;
  o.Jc[2][3] = T(0); o.Jc[2][4] = T(0); o.Jc[2][5] = D22;
  // intrinsics f, k1, k2
  o.Jc[0][6] = dist * xn; o.Jc[0][7] = f * xn * rr; o.Jc[0][8] = f * xn * rr * rr;
  o.Jc[1][6] = dist * yn; o.Jc[1][7] = f * yn * rr; o.Jc[1][8] = f * yn * rr * rr;
  o.Jc[2][6] = T(0); o.Jc[2][7] = T(0); o.Jc[2][8] = T(0);
  // point block: D * R
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    o.Jp[0][j] = D00 * R[j] + D01 * R[3 + j] + D02 * R[6 + j];
    o.Jp[1][j] = D10 * R[j] + D11 * R[3 + j] + D12 * R[6 + j];
    o.Jp[2][j] = D22 * R[6 + j];
  }
  if (cw[15] != T(0)) {
    // model 1: centre columns -D R, no distortion columns
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
      for (int j = 0; j < 3; ++j) o.Jc[m][3 + j] = -o.Jp[m][j];
      o.Jc[m][7] = T(0);
      o.Jc[m][8] = T(0);
    }
  }
}

// FP64 evaluation of one observation: residual, camera-frame depth and pixel.
struct Eval64 {
  double r0, r1, r2, z, uh, vh;
};

__device__ __forceinline__ Eval64 eval_obs64(const double* __restrict__ cw, double X0, double X1,
                                             double X2, double u, double v, double tau, double sw,
                                             double cx, double cy) {
  const double* R = cw;
  double px = fma(R[0], X0, fma(R[1], X1, fma(R[2], X2, cw[9])));
  double py = fma(R[3], X0, fma(R[4], X1, fma(R[5], X2, cw[10])));
  double pz = fma(R[6], X0, fma(R[7], X1, fma(R[8], X2, cw[11])));
  const double iz = recip_nr(pz);
  double xn = px * iz, yn = py * iz;
  double rr = xn * xn + yn * yn;
  double fd = cw[12] * (1.0 + rr * (cw[13] + cw[14] * rr));
  Eval64 e;
  e.uh = fd * xn + cx;
  e.vh = fd * yn + cy;
  e.z = pz;
  e.r0 = e.uh - u;
  e.r1 = e.vh - v;
  e.r2 = sw * (iz - tau);
  return e;
}

// Rotation matrix of an axis-angle vector: cos(th) I + sin(th) [k]x + (1 - cos(th)) k k^T,
// with the series of sin(th)/th and (1 - cos(th))/th^2 near zero.
__device__ __forceinline__ void rotvec_matrix(const double w[3], double R[9]) {
  double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double c, sa, cb;  // cos th, sin th / th, (1 - cos th) / th^2
  if (t2 < 1e-16) {
    c = 1.0 - 0.5 * t2;
    sa = 1.0 - t2 / 6.0;
    cb = 0.5 - t2 / 24.0;
  } else {
    double th = sqrt(t2);
    double sn, cs;
    sincos(th, &sn, &cs);
    c = cs;
    sa = sn / th;
    cb = (1.0 - cs) / t2;
  }
  R[0] = c + cb * w[0] * w[0];
  R[1] = cb * w[0] * w[1] - sa * w[2];
  R[2] = cb * w[0] * w[2] + sa * w[1];
  R[3] = cb * w[1] * w[0] + sa * w[2];
  R[4] = c + cb * w[1] * w[1];
  R[5] = cb * w[1] * w[2] - sa * w[0];
  R[6] = cb * w[2] * w[0] - sa * w[1];
  R[7] = cb * w[2] * w[1] + sa * w[0];
  R[8] = c + cb * w[2] * w[2];
}

// Working record of a camera's nine parameters (see the camera models above):
// R (9), t (3), f, k1, k2, model.
__device__ __forceinline__ void cam_record(const double* __restrict__ p, int model, double rec[16]) {
  const double w[3] = {p[0], p[1], p[2]};
  double R[9];
  rotvec_matrix(w, R);
  for (int i = 0; i < 9; ++i) rec[i] = R[i];
  if (model == 1) {
    for (int i = 0; i < 3; ++i) rec[9 + i] = -(R[3 * i] * p[3] + R[3 * i + 1] * p[4] + R[3 * i + 2] * p[5]);
    rec[12] = p[6];
    rec[13] = 0.0;
    rec[14] = 0.0;
    rec[15] = 1.0;
  } else {
    for (int i = 0; i < 6; ++i) rec[9 + i] = p[3 + i];
    rec[15] = 0.0;
  }
}

// Left composition of rotations in axis-angle form, Log(Exp(a) Exp(b)), through
// unit quaternions (Hamilton product), result angle in [0, pi].
__device__ __forceinline__ void rotvec_left_compose(const double a[3], const double b[3],
                                                    double out[3]) {
  double qa[4], qb[4];
  const double* ws[2] = {a, b};
  double* qs[2] = {qa, qb};
  for (int i = 0; i < 2; ++i) {
    const double* w = ws[i];
    double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double hc, hs;  // cos(th/2), sin(th/2)/th
    if (t2 < 1e-16) {
      hc = 1.0 - t2 / 8.0;
      hs = 0.5 - t2 / 48.0;
    } else {
      double th = sqrt(t2), sn, cs;
      sincos(0.5 * th, &sn, &cs);
      hc = cs;
      hs = sn / th;
    }
    qs[i][0] = hc;
    qs[i][1] = hs * w[0];
    qs[i][2] = hs * w[1];
    qs[i][3] = hs * w[2];
  }
  double s = qa[0] * qb[0] - (qa[1] * qb[1] + qa[2] * qb[2] + qa[3] * qb[3]);
  double v0 = qa[0] * qb[1] + qb[0] * qa[1] + (qa[2] * qb[3] - qa[3] * qb[2]);
  double v1 = qa[0] * qb[2] + qb[0] * qa[2] + (qa[3] * qb[1] - qa[1] * qb[3]);
  double v2 = qa[0] * qb[3] + qb[0] * qa[3] + (qa[1] * qb[2] - qa[2] * qb[1]);
  if (s < 0.0) { s = -s; v0 = -v0; v1 = -v1; v2 = -v2; }
  double vn = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
  double k = vn < 1e-12 ? 2.0 / s : 2.0 * atan2(vn, s) / vn;
  out[0] = k * v0;
  out[1] = k * v1;
  out[2] = k * v2;
}

}  // namespace bab
