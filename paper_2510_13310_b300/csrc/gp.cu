// gp.cu -- depth-constrained global positioning (GP) on the device, and its C ABI.
//
// The objective of Sec. 3.1 (Eq. GP objective): sum_k rho(|u_k|^2) with
// u_k = v_k - s_k (X_j - t_i) for observation k of point j in camera i, v_k the
// unit ray from the camera centre t_i toward the feature in the world frame
// (rotations are known and held), s_k a per-observation scale and rho Huber.
// Sec. 4.1 pins the scale of every observation with a metric depth d_k
// (s_k = 1/d_k, removed from the unknowns); the other scales stay free and are
// compacted by their rank among the free observations (a prefix scan over the
// free flags, the same scan as the BA extraction's ranks).
//
// The LM step of Sec. 3.3 (Eq. LM, Marquardt damping of the full system) is
// solved exactly by elimination: each free scale couples one centre and one
// point, so it is eliminated per observation, which leaves per observation a
// symmetric 3x3 block M_k = w s^2 I - (w s)^2 e e^T / Q*_k (e = X - t, Q*_k the
// damped scale curvature) that is at once the centre block, the point block
// and, negated, the centre-point coupling.  Eliminating the points (3x3 V*_j)
// leaves the centre system S (3 C_f): its diagonal blocks are summed over each
// camera's observations (camera-order chunks, fixed order), its off-diagonal
// blocks S_ij = -sum_p M_k V*_p^-1 M_k' over the co-visibility runs of camera
// pairs.  The centre system of these scenes is dense, so it is Jacobi-scaled and
// solved by the tensor-core Cholesky-preconditioned CG of dense_tc.cu.  Points
// and free scales follow by back-substitution.  FP32 hot path; the cost, the
// predicted decrease and the gain ratio in FP64; every reduction in a fixed order.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ba_b300.h"
#include "internal.h"
#include "layout_dev.h"

namespace bab {
namespace gpk {

constexpr int kThreads = 128;
constexpr int kPartStride = 24;  // floats per camera-chunk partial (22 used)

__device__ __forceinline__ float huber_w32(float n2, float delta) {
  return (delta <= 0.f || n2 <= delta * delta) ? 1.f : delta * rsqrtf(n2);
}
__device__ __forceinline__ double clampd(double a) { return fmin(fmax(a, 1e-6), 1e32); }
__device__ __forceinline__ float clampf(float a) { return fminf(fmaxf(a, 1e-6f), 1e32f); }

// per point-order observation, 5 float4:
//  r0 (M00 M01 M02 M11)  r1 (M12 M22 q0 q1)  r2 (q2 d gu0 gu1)  r3 (gu2 gs Qs ws)  r4 (Dq . . .)
// M: reduced 3x3 block; q: reduced centre gradient (the point's is -q);
// d = w s^2 (diagonal of the unreduced centre and point blocks); gu = w s u (the
// unreduced centre gradient); gs, Qs, Dq: scale gradient, damped curvature and
// its clamped diagonal (free scales only); ws = w s.
constexpr int kRec = 5;
// per point, 4 float4: p0 (Vi00 Vi01 Vi02 Vi11) p1 (Vi12 Vi22 DV nobs) p2 (gXr, .) p3 (gXu, .)
constexpr int kPtRec = 4;

// Steps (a)+(b), point side, at damping lambda: per observation M_k, q_k, ...;
// per point V*_j^-1 (FP64 adjugate), reduced and unreduced gradients; then
// Y_k = M_k V*_j^-1 per observation.  One thread per point, observations in order.
__global__ void __launch_bounds__(kThreads) k_gp_point(int P, const int* __restrict__ pt_off,
                                                       const int* __restrict__ po_cam,
                                                       const int* __restrict__ po_sidx,
                                                       const float4* __restrict__ ray4,
                                                       const float4* __restrict__ cw, const float4* __restrict__ pw,
                                                       const float* __restrict__ sw, float lambda, float huber,
                                                       float4* __restrict__ rec, float4* __restrict__ Y,
                                                       float4* __restrict__ ptrec) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  const int kb = pt_off[j], ke = pt_off[j + 1];
  const float4 Xw = pw[j];
  float V[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gr[3] = {0.f, 0.f, 0.f}, gu[3] = {0.f, 0.f, 0.f}, DV = 0.f;
  for (int k = kb; k < ke; ++k) {
    const float4 rv = ray4[k];
    const float4 tw = cw[po_cam[k]];
    const int si = po_sidx[k];
    const float s = si >= 0 ? sw[si] : rv.w;
    const float e0 = Xw.x - tw.x, e1 = Xw.y - tw.y, e2 = Xw.z - tw.z;
    const float u0 = fmaf(-s, e0, rv.x), u1 = fmaf(-s, e1, rv.y), u2 = fmaf(-s, e2, rv.z);
    const float w = huber_w32(u0 * u0 + u1 * u1 + u2 * u2, huber);
    const float ws = w * s, d = ws * s;
    float M[6] = {d, 0.f, 0.f, d, 0.f, d};
    float q0 = ws * u0, q1 = ws * u1, q2 = ws * u2;
    const float g0 = q0, g1 = q1, g2 = q2;
    float gs = 0.f, Qs = 0.f, Dq = 0.f;
    if (si >= 0) {
      const float Qr = w * (e0 * e0 + e1 * e1 + e2 * e2);
      Dq = clampf(Qr);
      Qs = fmaf(lambda, Dq, Qr);
      gs = -w * (e0 * u0 + e1 * u1 + e2 * u2);
      const float c1 = ws * ws / Qs, c2 = ws * gs / Qs;
      M[0] -= c1 * e0 * e0;
      M[1] -= c1 * e0 * e1;
      M[2] -= c1 * e0 * e2;
      M[3] -= c1 * e1 * e1;
      M[4] -= c1 * e1 * e2;
      M[5] -= c1 * e2 * e2;
      q0 = fmaf(c2, e0, q0);
      q1 = fmaf(c2, e1, q1);
      q2 = fmaf(c2, e2, q2);
    }
    float4* r = rec + (size_t)kRec * k;
    r[0] = make_float4(M[0], M[1], M[2], M[3]);
    r[1] = make_float4(M[4], M[5], q0, q1);
    r[2] = make_float4(q2, d, g0, g1);
    r[3] = make_float4(g2, gs, Qs, ws);
    r[4] = make_float4(Dq, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 6; ++i) V[i] += M[i];
    gr[0] -= q0, gr[1] -= q1, gr[2] -= q2;
    gu[0] -= g0, gu[1] -= g1, gu[2] -= g2;
    DV += d;
  }
  // V* = V + lambda clamp(DV) I and its inverse (adjugate, FP64: a 3x3 per point)
  double Vi[6] = {0, 0, 0, 0, 0, 0};
  if (ke > kb) {
    const double dl = (double)lambda * clampd((double)DV);
    const double a = V[0] + dl, b = V[1], c = V[2], dd = V[3] + dl, e = V[4], f = V[5] + dl;
    const double A0 = dd * f - e * e, A1 = c * e - b * f, A2 = b * e - c * dd;
    const double det = a * A0 + b * A1 + c * A2;
    const double id = 1.0 / det;
    Vi[0] = A0 * id;
    Vi[1] = A1 * id;
    Vi[2] = A2 * id;
    Vi[3] = (a * f - c * c) * id;
    Vi[4] = (b * c - a * e) * id;
    Vi[5] = (a * dd - b * b) * id;
  }
  float4* pr = ptrec + (size_t)kPtRec * j;
  pr[0] = make_float4((float)Vi[0], (float)Vi[1], (float)Vi[2], (float)Vi[3]);
  pr[1] = make_float4((float)Vi[4], (float)Vi[5], DV, (float)(ke - kb));
  pr[2] = make_float4(gr[0], gr[1], gr[2], 0.f);
  pr[3] = make_float4(gu[0], gu[1], gu[2], 0.f);
  const float W00 = (float)Vi[0], W01 = (float)Vi[1], W02 = (float)Vi[2], W11 = (float)Vi[3], W12 = (float)Vi[4],
              W22 = (float)Vi[5];
  for (int k = kb; k < ke; ++k) {
    const float4 a = rec[(size_t)kRec * k], b = rec[(size_t)kRec * k + 1];
    const float m00 = a.x, m01 = a.y, m02 = a.z, m11 = a.w, m12 = b.x, m22 = b.y;
    float4* y = Y + 3 * (size_t)k;
    // Y = M V*^-1, row-major 3x3 padded to 12
    y[0] = make_float4(m00 * W00 + m01 * W01 + m02 * W02, m00 * W01 + m01 * W11 + m02 * W12,
                       m00 * W02 + m01 * W12 + m02 * W22, m01 * W00 + m11 * W01 + m12 * W02);
    y[1] = make_float4(m01 * W01 + m11 * W11 + m12 * W12, m01 * W02 + m11 * W12 + m12 * W22,
                       m02 * W00 + m12 * W01 + m22 * W02, m02 * W01 + m12 * W11 + m22 * W12);
    y[2] = make_float4(m02 * W02 + m12 * W12 + m22 * W22, 0.f, 0.f, 0.f);
  }
}

// Camera side: per camera-order chunk (one camera, <= 1024 observations), sums
// of U (6), the reduced and unreduced gradients (3 + 3), DU, sum Y_k M_k (6) and
// sum Y_k gXr_p (3), in one fixed order (strided per thread, then a fixed tree).
__global__ void __launch_bounds__(kThreads) k_gp_cam_chunk(const int* __restrict__ chunk_obs,
                                                           const int* __restrict__ chunk_cam,
                                                           const int* __restrict__ crank,
                                                           const int* __restrict__ co_po,
                                                           const int* __restrict__ po_pt,
                                                           const float4* __restrict__ rec,
                                                           const float4* __restrict__ Y,
                                                           const float4* __restrict__ ptrec,
                                                           float* __restrict__ part) {
  __shared__ float red[kThreads / 32][22];
  const int q = blockIdx.x;
  float* out = part + (size_t)kPartStride * q;
  if (crank[chunk_cam[q]] < 0) {
    if (threadIdx.x < kPartStride) out[threadIdx.x] = 0.f;
    return;
  }
  float acc[22];
#pragma unroll
  for (int i = 0; i < 22; ++i) acc[i] = 0.f;
  for (int kc = chunk_obs[q] + threadIdx.x; kc < chunk_obs[q + 1]; kc += blockDim.x) {
    const int k = co_po[kc];
    const float4* r = rec + (size_t)kRec * k;
    const float4 a = r[0], b = r[1], c = r[2], d = r[3];
    const float M[9] = {a.x, a.y, a.z, a.y, a.w, b.x, a.z, b.x, b.y};
    const float4 y0 = Y[3 * (size_t)k], y1 = Y[3 * (size_t)k + 1], y2 = Y[3 * (size_t)k + 2];
    const float Yk[9] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w, y2.x};
    const float4 g = ptrec[(size_t)kPtRec * po_pt[k] + 2];
    acc[0] += a.x, acc[1] += a.y, acc[2] += a.z, acc[3] += a.w, acc[4] += b.x, acc[5] += b.y;
    acc[6] += b.z, acc[7] += b.w, acc[8] += c.x;   // reduced gradient q
    acc[9] += c.z, acc[10] += c.w, acc[11] += d.x;  // unreduced gradient gu
    acc[12] += c.y;                                 // DU
    // Y M (symmetric: M V^-1 M), upper triangle
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int t = 0; t < 6; ++t)
      acc[13 + t] += Yk[3 * ii[t]] * M[jj[t]] + Yk[3 * ii[t] + 1] * M[3 + jj[t]] + Yk[3 * ii[t] + 2] * M[6 + jj[t]];
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[19 + i] += Yk[3 * i] * g.x + Yk[3 * i + 1] * g.y + Yk[3 * i + 2] * g.z;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 22; ++i) {
    float v = acc[i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 22) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Per free camera (rank r): the chunk partials summed in order (FP64), damping,
// the diagonal block S_rr = U* - sum Y M, the right-hand side b_r = -(q + Y g),
// the Jacobi scale 1/sqrt(S_aa) and the record used by the predicted decrease.
__global__ void k_gp_cam_finish(int Cf, const int* __restrict__ cam_map, const int* __restrict__ cam_chunk,
                                const float* __restrict__ part, float lambda, float* __restrict__ Sdiag,
                                float* __restrict__ b, float* __restrict__ dsc, float4* __restrict__ camrec,
                                int* __restrict__ err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Cf) return;
  const int c = cam_map[r];
  double a[22];
  for (int i = 0; i < 22; ++i) a[i] = 0.0;
  for (int q = cam_chunk[c]; q < cam_chunk[c + 1]; ++q)
    for (int i = 0; i < 22; ++i) a[i] += (double)part[(size_t)kPartStride * q + i];
  const double dl = (double)lambda * clampd(a[12]);
  double S[6];
  for (int t = 0; t < 6; ++t) S[t] = a[t] - a[13 + t];
  S[0] += dl, S[3] += dl, S[5] += dl;
  for (int t = 0; t < 6; ++t) Sdiag[6 * (size_t)r + t] = (float)S[t];
  const double dg[3] = {S[0], S[3], S[5]};
  for (int i = 0; i < 3; ++i) {
    b[3 * (size_t)r + i] = (float)(-(a[6 + i] + a[19 + i]));
    if (!(dg[i] > 0.0)) atomicOr(err, 4);
    dsc[3 * (size_t)r + i] = dg[i] > 0.0 ? (float)(1.0 / sqrt(dg[i])) : 1.f;
  }
  camrec[r] = make_float4((float)a[12], (float)a[9], (float)a[10], (float)a[11]);
}

// Scaled diagonal blocks of the centre system: S^ = diag(d) S diag(d).
__global__ void k_gp_S_diag(int Cf, const float* __restrict__ Sdiag, const float* __restrict__ dsc, float* Sh,
                            long long ld) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Cf) return;
  const int sy[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Sh[(size_t)(3 * r + i) * ld + 3 * r + j] = Sdiag[6 * (size_t)r + sy[3 * i + j]] * dsc[3 * r + i] * dsc[3 * r + j];
}

// Off-diagonal blocks: one warp per co-visibility run (cameras i < j, pairs
// (k in i, k2 in j) of their shared points, ascending): S_ij = -sum Y_k M_k2,
// scaled, written at (i, j) and transposed at (j, i).
__global__ void __launch_bounds__(kThreads) k_gp_form_S(int n_runs, const int4* __restrict__ runs,
                                                        const int2* __restrict__ pairs,
                                                        const int* __restrict__ crank,
                                                        const float4* __restrict__ rec,
                                                        const float4* __restrict__ Y,
                                                        const float* __restrict__ dsc, float* Sh, long long ld) {
  const int lane = threadIdx.x & 31;
  for (int run = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; run < n_runs;
       run += (gridDim.x * blockDim.x) >> 5) {
    const int4 R = runs[run];
    const int ri = crank[R.x], rj = crank[R.y];
    if (ri < 0 || rj < 0) continue;
    float acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = 0.f;
    for (int t = lane; t < R.w; t += 32) {
      const int2 pr = pairs[R.z + t];
      const float4 y0 = Y[3 * (size_t)pr.x], y1 = Y[3 * (size_t)pr.x + 1], y2 = Y[3 * (size_t)pr.x + 2];
      const float Yk[9] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w, y2.x};
      const float4 a = rec[(size_t)kRec * pr.y], b = rec[(size_t)kRec * pr.y + 1];
      const float M[9] = {a.x, a.y, a.z, a.y, a.w, b.x, a.z, b.x, b.y};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jx = 0; jx < 3; ++jx)
          acc[3 * i + jx] += Yk[3 * i] * M[jx] + Yk[3 * i + 1] * M[3 + jx] + Yk[3 * i + 2] * M[6 + jx];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], m);
    }
    if (lane < 9) {
      const int i = lane / 3, jx = lane % 3;
      float v = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t)
        if (t == lane) v = acc[t];
      const float sv = -v * dsc[3 * ri + i] * dsc[3 * rj + jx];
      Sh[(size_t)(3 * ri + i) * ld + 3 * rj + jx] = sv;
      Sh[(size_t)(3 * rj + jx) * ld + 3 * ri + i] = sv;
    }
  }
}

// Identity rows of the padding that makes the centre system a whole number of
// 9-unknown super-blocks (three cameras each) for the block-Jacobi PCG.
__global__ void k_gp_pad(int n, int n_pad, float* Sh, long long ld) {
  const int r = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_pad) Sh[(size_t)r * ld + r] = 1.f;
}

// Block-Jacobi preconditioner of the scaled centre system: the inverse of each
// 9x9 diagonal super-block by Cholesky factorisation (FP32), one warp per block:
// lane i holds row i during the right-looking factorisation, then lane c solves
// for column c of the inverse from the factor in shared memory.  A block that
// fails to factor falls back to its inverse diagonal.
constexpr int kSbWarps = 4;
__global__ void __launch_bounds__(32 * kSbWarps) k_gp_superblock_inv(int Cs, const float* __restrict__ Sh, long long ld,
                                                                      float* __restrict__ Dinv) {
  __shared__ float Ls[kSbWarps][81];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int sb = blockIdx.x * kSbWarps + wl;
  if (sb >= Cs) return;  // whole warps leave together
  float row[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) row[j] = lane < 9 ? Sh[(size_t)(9 * sb + lane) * ld + 9 * sb + j] : 0.f;
  const float diag = lane < 9 ? row[lane < 9 ? lane : 0] : 1.f;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float akk = __shfl_sync(0xffffffffu, row[k], k);
    ok = ok && akk > 0.f;
    const float dk = sqrtf(fmaxf(akk, 1e-30f));
    // column k of L: L[i][k] = A[i][k] / d for i > k, d on the diagonal
    const float lik = lane == k ? dk : (lane > k ? row[k] / dk : 0.f);
    row[k] = lik;
#pragma unroll
    for (int j = k + 1; j < 9; ++j) {
      const float ljk = __shfl_sync(0xffffffffu, lik, j);
      if (lane > k && j <= lane) row[j] -= lik * ljk;
    }
  }
  if (lane < 9)
#pragma unroll
    for (int j = 0; j < 9; ++j) Ls[wl][9 * lane + j] = j <= lane ? row[j] : 0.f;
  __syncwarp();
  float inv[9];
  if (ok && lane < 9) {
    // column c = lane: L y = e_c, then L^T x = y
    float y[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float v = i == lane ? 1.f : 0.f;
#pragma unroll
      for (int k2 = 0; k2 < i; ++k2) v -= Ls[wl][9 * i + k2] * y[k2];
      y[i] = v / Ls[wl][9 * i + i];
    }
#pragma unroll
    for (int i = 8; i >= 0; --i) {
      float v = y[i];
#pragma unroll
      for (int k2 = i + 1; k2 < 9; ++k2) v -= Ls[wl][9 * k2 + i] * inv[k2];
      inv[i] = v / Ls[wl][9 * i + i];
    }
  }
  if (lane < 9)
#pragma unroll
    for (int i = 0; i < 9; ++i)
      Dinv[81 * (size_t)sb + 9 * i + lane] = ok ? inv[i] : (i == lane ? (diag > 0.f ? 1.f / diag : 1.f) : 0.f);
}

__global__ void k_gp_ones(int n, double* __restrict__ dscale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    dscale[i] = 1.0;
    reinterpret_cast<float*>(dscale + n)[i] = 1.f;
  }
}

__global__ void k_gp_scale(int n, const float* __restrict__ a, const float* __restrict__ d, float* __restrict__ o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] * d[i];
}

// Back-substitution: dX_j = V*^-1 (-g_X'_j + sum_k M_k dt_c) (the coupling
// block of observation k is -M_k), then each free scale ds = (-gs + ws e.(dt - dX)) / Qs;
// per block, the points' and scales' share of the predicted decrease
// 1/2 dx^T (lambda D dx - g) (FP64).
__global__ void __launch_bounds__(kThreads) k_gp_backsub(int P, const int* __restrict__ pt_off,
                                                         const int* __restrict__ po_cam,
                                                         const int* __restrict__ po_sidx,
                                                         const int* __restrict__ crank,
                                                         const float4* __restrict__ cw,
                                                         const float4* __restrict__ pw,
                                                         const float4* __restrict__ rec,
                                                         const float4* __restrict__ ptrec,
                                                         const float* __restrict__ dt, float lambda,
                                                         float4* __restrict__ dX, float* __restrict__ ds,
                                                         double* __restrict__ pred_parts) {
  __shared__ double red[32];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double pred = 0.0;
  if (j < P) {
    const int kb = pt_off[j], ke = pt_off[j + 1];
    const float4* pr = ptrec + (size_t)kPtRec * j;
    const float4 p0 = pr[0], p1 = pr[1], p2 = pr[2], p3 = pr[3];
    // p2 holds the reduced point gradient g_X' (= -sum q); the coupling block is -M_k
    float r0 = -p2.x, r1 = -p2.y, r2 = -p2.z;
    for (int k = kb; k < ke; ++k) {
      const int rc = crank[po_cam[k]];
      if (rc < 0) continue;
      const float4 a = rec[(size_t)kRec * k], b = rec[(size_t)kRec * k + 1];
      const float t0 = dt[3 * rc], t1 = dt[3 * rc + 1], t2 = dt[3 * rc + 2];
      r0 += a.x * t0 + a.y * t1 + a.z * t2;
      r1 += a.y * t0 + a.w * t1 + b.x * t2;
      r2 += a.z * t0 + b.x * t1 + b.y * t2;
    }
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (ke > kb) {
      x0 = p0.x * r0 + p0.y * r1 + p0.z * r2;
      x1 = p0.y * r0 + p0.w * r1 + p1.x * r2;
      x2 = p0.z * r0 + p1.x * r1 + p1.y * r2;
      const double dv = (double)lambda * clampd((double)p1.z);
      pred += 0.5 * ((double)x0 * (dv * x0 - p3.x) + (double)x1 * (dv * x1 - p3.y) + (double)x2 * (dv * x2 - p3.z));
    }
    dX[j] = make_float4(x0, x1, x2, 0.f);
    const float4 Xw = pw[j];
    for (int k = kb; k < ke; ++k) {
      const int si = po_sidx[k];
      if (si < 0) continue;
      const int c = po_cam[k], rc = crank[c];
      const float4 tw = cw[c];
      const float e0 = Xw.x - tw.x, e1 = Xw.y - tw.y, e2 = Xw.z - tw.z;
      float d0 = -x0, d1 = -x1, d2 = -x2;
      if (rc >= 0) d0 += dt[3 * rc], d1 += dt[3 * rc + 1], d2 += dt[3 * rc + 2];
      const float4 r3 = rec[(size_t)kRec * k + 3], r4 = rec[(size_t)kRec * k + 4];
      const float gs = r3.y, Qs = r3.z, ws = r3.w, Dq = r4.x;
      const float dsk = (-gs + ws * (e0 * d0 + e1 * d1 + e2 * d2)) / Qs;
      ds[si] = dsk;
      pred += 0.5 * (double)dsk * ((double)lambda * Dq * dsk - gs);
    }
  }
  const double s = block_sum(pred, red);
  if (threadIdx.x == 0) pred_parts[blockIdx.x] = s;
}

// The centres' share of the predicted decrease, then the fixed-order total.
__global__ void k_gp_pred_cams(int Cf, const float* __restrict__ dt, const float4* __restrict__ camrec,
                               float lambda, const double* __restrict__ parts, int n_parts,
                               Scalars* __restrict__ sc) {
  __shared__ double red[32];
  double v = 0.0;
  for (int r = threadIdx.x; r < Cf; r += blockDim.x) {
    const float4 cr = camrec[r];
    const double dl = (double)lambda * clampd((double)cr.x);
    const double g[3] = {cr.y, cr.z, cr.w};
    for (int i = 0; i < 3; ++i) {
      const double x = dt[3 * r + i];
      v += 0.5 * x * (dl * x - g[i]);
    }
  }
  for (int i = threadIdx.x; i < n_parts; i += blockDim.x) v += parts[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) sc->pred = v;
}

// Candidate x + dx into state slot d: FP64 masters and FP32 working copies.
__global__ void k_gp_candidate(int C, int P, int F, const int* __restrict__ crank, const float* __restrict__ dt,
                               const float4* __restrict__ dX, const float* __restrict__ ds,
                               const double* __restrict__ t_in, const double* __restrict__ X_in,
                               const double* __restrict__ s_in, double* __restrict__ t_out,
                               double* __restrict__ X_out, double* __restrict__ s_out, float4* __restrict__ cw_out,
                               float4* __restrict__ pw_out, float* __restrict__ sw_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C) {
    const int r = crank[i];
    double t[3];
    for (int a = 0; a < 3; ++a) t[a] = t_in[3 * (size_t)i + a] + (r >= 0 ? (double)dt[3 * r + a] : 0.0);
    for (int a = 0; a < 3; ++a) t_out[3 * (size_t)i + a] = t[a];
    cw_out[i] = make_float4((float)t[0], (float)t[1], (float)t[2], 0.f);
  }
  if (i < P) {
    const float4 d = dX[i];
    const double X[3] = {X_in[3 * (size_t)i] + d.x, X_in[3 * (size_t)i + 1] + d.y, X_in[3 * (size_t)i + 2] + d.z};
    for (int a = 0; a < 3; ++a) X_out[3 * (size_t)i + a] = X[a];
    pw_out[i] = make_float4((float)X[0], (float)X[1], (float)X[2], 0.f);
  }
  if (i < F) {
    const double s = s_in[i] + (double)ds[i];
    s_out[i] = s;
    sw_out[i] = (float)s;
  }
}

// FP64 cost of a state slot: F = 1/2 sum rho(|u|^2) and sum |u|^2, per block,
// then the last block to finish adds the partials in block order.
__global__ void __launch_bounds__(256) k_gp_eval(int N, const int* __restrict__ po_cam, const int* __restrict__ po_pt,
                                                 const int* __restrict__ po_sidx, const double4* __restrict__ ray64,
                                                 const double* __restrict__ t64, const double* __restrict__ X64,
                                                 const double* __restrict__ s64, double huber,
                                                 double* __restrict__ parts, Scalars* __restrict__ sc, int slot) {
  __shared__ double red[32];
  double F = 0.0, E = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const double4 rv = ray64[k];
    const int c = po_cam[k], p = po_pt[k], si = po_sidx[k];
    const double s = si >= 0 ? s64[si] : rv.w;
    const double u0 = rv.x - s * (X64[3 * (size_t)p] - t64[3 * (size_t)c]);
    const double u1 = rv.y - s * (X64[3 * (size_t)p + 1] - t64[3 * (size_t)c + 1]);
    const double u2 = rv.z - s * (X64[3 * (size_t)p + 2] - t64[3 * (size_t)c + 2]);
    const double n2 = u0 * u0 + u1 * u1 + u2 * u2;
    F += (huber <= 0.0 || n2 <= huber * huber) ? n2 : 2.0 * huber * sqrt(n2) - huber * huber;
    E += n2;
  }
  const double sF = block_sum(F, red);
  const double sE = block_sum(E, red);
  if (threadIdx.x == 0) {
    parts[2 * blockIdx.x] = sF;
    parts[2 * blockIdx.x + 1] = sE;
  }
  if (last_block_done(&sc->done_eval)) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      a += __ldcg(parts + 2 * i);
      b += __ldcg(parts + 2 * i + 1);
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
      sc->cost[slot] = 0.5 * a;
      sc->rmse_sum[slot] = b;
      sc->done_eval = 0;
    }
  }
}

// ---- set-up kernels ----
__global__ void k_gp_check(const double* __restrict__ v, long long n, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) atomicOr(bad, 1);
}
__global__ void k_gp_free_flags(int N, const double* __restrict__ depth, uint8_t* __restrict__ flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    const double d = depth[k];
    flags[k] = (d > 0.0 && isfinite(d)) ? 0 : 1;
  }
}
// point-order copies of the rays, pinned targets and free-scale ranks
__global__ void k_gp_obs(int N, const int* __restrict__ po, const double* __restrict__ rays,
                         const double* __restrict__ depth, const int* __restrict__ free_rank,
                         float4* __restrict__ ray4, double4* __restrict__ ray64, int* __restrict__ po_sidx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int o = po[k];
  const double d = depth[o];
  const bool pin = d > 0.0 && isfinite(d);
  const double tau = pin ? 1.0 / d : 0.0;
  const double v0 = rays[3 * (size_t)o], v1 = rays[3 * (size_t)o + 1], v2 = rays[3 * (size_t)o + 2];
  ray64[k] = make_double4(v0, v1, v2, tau);
  ray4[k] = make_float4((float)v0, (float)v1, (float)v2, (float)tau);
  po_sidx[k] = free_rank[o];
}
__global__ void k_gp_gather_scales(int F, const int* __restrict__ free_map, const double* __restrict__ scales0,
                                   double* __restrict__ s64, float* __restrict__ sw) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double s = scales0 ? scales0[free_map[f]] : 1.0;
  s64[f] = s;
  sw[f] = (float)s;
}
__global__ void k_gp_prep(int C, int P, const double* __restrict__ t64, const double* __restrict__ X64,
                          float4* __restrict__ cw, float4* __restrict__ pw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C) cw[i] = make_float4((float)t64[3 * (size_t)i], (float)t64[3 * (size_t)i + 1], (float)t64[3 * (size_t)i + 2], 0.f);
  if (i < P) pw[i] = make_float4((float)X64[3 * (size_t)i], (float)X64[3 * (size_t)i + 1], (float)X64[3 * (size_t)i + 2], 0.f);
}
// full-index outputs: scales in input order (pinned: 1/d), steps
__global__ void k_gp_scales_out(int N, const double* __restrict__ depth, const int* __restrict__ free_rank,
                                const double* __restrict__ s64, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int f = free_rank[k];
  out[k] = f >= 0 ? s64[f] : 1.0 / depth[k];
}
__global__ void k_gp_steps_out(int C, int P, int N, const int* __restrict__ crank, const int* __restrict__ free_rank,
                               const float* __restrict__ dt, const float4* __restrict__ dX,
                               const float* __restrict__ ds, double* __restrict__ o_dt, double* __restrict__ o_dX,
                               double* __restrict__ o_ds) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C)
    for (int a = 0; a < 3; ++a) o_dt[3 * (size_t)i + a] = crank[i] >= 0 ? (double)dt[3 * crank[i] + a] : 0.0;
  if (i < P) {
    const float4 d = dX[i];
    o_dX[3 * (size_t)i] = d.x, o_dX[3 * (size_t)i + 1] = d.y, o_dX[3 * (size_t)i + 2] = d.z;
  }
  if (i < N) o_ds[i] = free_rank[i] >= 0 ? (double)ds[free_rank[i]] : 0.0;
}

inline int blocks(long long n, int t) { return (int)std::max<long long>(1, (n + t - 1) / t); }

}  // namespace gpk
}  // namespace bab

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

using namespace bab;

struct ba_gp_problem {
  ba_gp_options opt{};
  std::vector<int32_t> fixed_list;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  int C = 0, P = 0, N = 0, F = 0, Cf = 0, n = 0;
  long long ld = 0;
  std::vector<void*> allocs;
  int64_t launches = 0;
  // layout
  int *po = nullptr, *po_cam = nullptr, *po_pt = nullptr, *pt_off = nullptr, *co_po = nullptr;
  int *chunk_obs = nullptr, *chunk_cam = nullptr, *cam_chunk = nullptr;
  int n_chunks = 0;
  int4* runs = nullptr;
  int2* pairs = nullptr;
  int n_runs = 0;
  // static per observation (point order) and the free-scale compaction
  float4* ray4 = nullptr;
  double4* ray64 = nullptr;
  int *po_sidx = nullptr, *free_rank = nullptr, *free_map = nullptr;
  double* depth_in = nullptr;  // input order, for the scale output
  int *crank = nullptr, *cam_map = nullptr;
  // state slots
  double *t64[2] = {}, *X64[2] = {}, *s64[2] = {};
  float4 *cw[2] = {}, *pw[2] = {};
  float* sw[2] = {};
  int cur = 0;
  bool cost_valid = false;
  // linearisation and solve
  float4 *rec = nullptr, *Y = nullptr, *ptrec = nullptr, *camrec = nullptr, *dX = nullptr;
  float *part = nullptr, *Sdiag = nullptr, *b = nullptr, *bh = nullptr, *dsc = nullptr, *Sh = nullptr;
  float *xh = nullptr, *dt = nullptr, *ds = nullptr;
  double *pred_parts = nullptr, *eval_parts = nullptr, *scales_out = nullptr, *steps_out = nullptr;
  int bs_grid = 1, eval_grid = 1;
  // centre-system solver: block-Jacobi PCG on 9-unknown super-blocks (three
  // cameras) with the explicit PCG kernel, or the tensor-core dense solve
  bool use_dense = false;
  int Cs = 0, n_pad = 0;
  float* Dinv = nullptr;         // [Cs][81] inverses of the diagonal super-blocks
  double* dscale = nullptr;      // unit scaling for the PCG kernel (the system is scaled already)
  float *pcg_scratch = nullptr, *pcg_M = nullptr;
  size_t pcg_scratch_stride = 0, pcg_smem = 0;
  int pcg_grid = 1, pcg_rows_in_smem = 1, pcg_vecs_in_smem = 1;
  unsigned long long* words = nullptr;
  unsigned tag = 1;
  DenseWork dw;
  unsigned dense_epoch = 0;
  Scalars* sc = nullptr;
  Scalars* h_sc = nullptr;
  int* err = nullptr;
  double lambda = 1e-4, nu = 2.0;
  int iter = 0;
  cudaEvent_t ev[6] = {};
};

namespace {

thread_local std::string g_gp_err;

void gp_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_gp_err = buf;
  set_last_error_message(buf);
}

#define GCU(expr)                                                                              \
  do {                                                                                         \
    cudaError_t _e = (expr);                                                                   \
    if (_e != cudaSuccess) {                                                                   \
      cudaGetLastError(); /* reported here: not left for the caller's next check */            \
      gp_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__);    \
      return _e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA;                       \
    }                                                                                          \
  } while (0)
#define GST(expr)                \
  do {                           \
    ba_status _s = (expr);       \
    if (_s != BA_OK) return _s;  \
  } while (0)
#define GLAUNCH(pb, cnt, ...)        \
  do {                               \
    __VA_ARGS__;                     \
    (pb)->launches += (cnt);         \
    GCU(cudaGetLastError());         \
  } while (0)

template <typename X>
ba_status galloc(ba_gp_problem* pb, X** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    gp_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return BA_ERR_OOM;
  }
  pb->allocs.push_back(q);
  *p = static_cast<X*>(q);
  return BA_OK;
}

void gp_free(ba_gp_problem* pb) {
  if (!pb) return;
  if (pb->stream) cudaStreamSynchronize(pb->stream);
  for (void* q : pb->allocs) cudaFree(q);
  if (pb->h_sc) cudaFreeHost(pb->h_sc);
  for (auto& e : pb->ev)
    if (e) cudaEventDestroy(e);
  delete pb;
}

ba_status gp_sync(ba_gp_problem* pb) {
  GCU(cudaStreamSynchronize(pb->stream));
  return BA_OK;
}

bool gp_opts_ok(const ba_gp_options* o) {
  return std::isfinite(o->huber_delta) && std::isfinite(o->lambda0) && o->lambda0 > 0 &&
         std::isfinite(o->pcg_rel_tol) && o->pcg_rel_tol > 0 && o->pcg_max_iters > 0;
}

// Uploads (or copies, for device pointers) n values into a new device buffer.
template <typename X>
ba_status gp_input(ba_gp_problem* pb, const X* src, size_t n, X** out) {
  GST(galloc(pb, out, n));
  if (n) GCU(cudaMemcpyAsync(*out, src, sizeof(X) * n, cudaMemcpyDefault, pb->stream));
  return BA_OK;
}

ba_status gp_create_impl(const ba_gp_options* opts, void* stream, int64_t n_cams, const double* centres,
                         int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                         const int32_t* obs_pt, const double* rays, const double* depth, const double* scales0,
                         ba_gp_problem* pb) {
  if (!opts || !gp_opts_ok(opts)) {
    gp_error("invalid GP options");
    return BA_ERR_INVALID_ARG;
  }
  if (n_cams < 0 || n_pts < 0 || n_obs < 0 || n_cams >= (1LL << 24) || n_pts >= (1LL << 30) ||
      n_obs >= (1LL << 30)) {
    gp_error("sizes out of range");
    return BA_ERR_INVALID_ARG;
  }
  if ((n_cams && !centres) || (n_pts && !pts) || (n_obs && (!obs_cam || !obs_pt || !rays || !depth))) {
    gp_error("null input array");
    return BA_ERR_INVALID_ARG;
  }
  pb->opt = *opts;
  pb->fixed_list.assign(opts->fixed_cams, opts->fixed_cams + (opts->fixed_cams ? opts->n_fixed : 0));
  pb->opt.fixed_cams = nullptr;
  pb->stream = (cudaStream_t)stream;
  pb->lambda = opts->lambda0;
  const int C = (int)n_cams, P = (int)n_pts, N = (int)n_obs;
  pb->C = C, pb->P = P, pb->N = N;
  GCU(cudaGetDevice(&pb->device));
  GCU(cudaDeviceGetAttribute(&pb->num_sms, cudaDevAttrMultiProcessorCount, pb->device));
  for (int32_t f : pb->fixed_list)
    if (f < 0 || f >= C) {
      gp_error("fixed camera %d out of range", f);
      return BA_ERR_INVALID_ARG;
    }

  // inputs on the device
  int32_t *d_oc = nullptr, *d_op = nullptr;
  double *d_t = nullptr, *d_X = nullptr, *d_rays = nullptr, *d_s0 = nullptr;
  GST(gp_input(pb, obs_cam, (size_t)N, &d_oc));
  GST(gp_input(pb, obs_pt, (size_t)N, &d_op));
  GST(gp_input(pb, centres, (size_t)3 * C, &d_t));
  GST(gp_input(pb, pts, (size_t)3 * P, &d_X));
  GST(gp_input(pb, rays, (size_t)3 * N, &d_rays));
  GST(gp_input(pb, depth, (size_t)N, &pb->depth_in));
  if (scales0) GST(gp_input(pb, scales0, (size_t)N, &d_s0));
  GST(galloc(pb, &pb->err, 1));
  GCU(cudaMemsetAsync(pb->err, 0, sizeof(int), pb->stream));
  GLAUNCH(pb, 1, gpk::k_gp_check<<<gpk::blocks(3LL * C, 256), 256, 0, pb->stream>>>(d_t, 3LL * C, pb->err));
  GLAUNCH(pb, 1, gpk::k_gp_check<<<gpk::blocks(3LL * P, 256), 256, 0, pb->stream>>>(d_X, 3LL * P, pb->err));
  GLAUNCH(pb, 1, gpk::k_gp_check<<<gpk::blocks(3LL * N, 256), 256, 0, pb->stream>>>(d_rays, 3LL * N, pb->err));
  if (d_s0) GLAUNCH(pb, 1, gpk::k_gp_check<<<gpk::blocks(N, 256), 256, 0, pb->stream>>>(d_s0, N, pb->err));
  {
    int bad = 0;
    GCU(cudaMemcpyAsync(&bad, pb->err, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
    GST(gp_sync(pb));
    if (bad) {
      gp_error("non-finite centre, point, ray or scale");
      return BA_ERR_INVALID_ARG;
    }
  }
  // observation layout (point order, camera-order chunks) and co-visibility runs
  auto dev_alloc = [pb](size_t bytes) -> void* {
    void* q = nullptr;
    return galloc(pb, reinterpret_cast<char**>(&q), bytes) == BA_OK ? q : nullptr;
  };
  DevLayout dl;
  {
    std::string msg;
    const int rc = build_obs_layout_dev_indices(C, P, N, d_oc, d_op, dev_alloc, pb->stream, &dl, &msg);
    if (rc) {
      gp_error("%s", msg.c_str());
      return rc == 1 ? BA_ERR_INVALID_ARG : rc == 3 ? BA_ERR_OOM : BA_ERR_CUDA;
    }
  }
  pb->po = dl.po;
  pb->po_cam = dl.po_cam;
  pb->po_pt = dl.po_pt;
  pb->pt_off = dl.pt_off;
  pb->co_po = dl.co_po;
  pb->chunk_obs = dl.chunk_obs;
  pb->chunk_cam = dl.chunk_cam;
  pb->cam_chunk = dl.cam_chunk;
  pb->n_chunks = dl.n_chunks;
  {
    DevCovis cv;
    std::string msg;
    const int rc = build_covis_runs_dev(dl, C, N, dev_alloc, pb->stream, &cv, &msg);
    if (rc) {
      gp_error("%s", msg.c_str());
      return rc == 1 ? BA_ERR_INVALID_ARG : rc == 3 ? BA_ERR_OOM : BA_ERR_CUDA;
    }
    pb->runs = cv.runs;
    pb->pairs = cv.pairs;
    pb->n_runs = cv.n_runs;
  }
  // free centres: not a gauge camera and at least one observation (ranks on the host)
  {
    std::vector<uint8_t> fixed((size_t)C, 0);
    for (int32_t f : pb->fixed_list) fixed[f] = 1;
    std::vector<int> rank((size_t)C, -1), map;
    for (int c = 0; c < C; ++c)
      if (!fixed[c] && dl.h_cam_off[c + 1] > dl.h_cam_off[c]) {
        rank[c] = (int)map.size();
        map.push_back(c);
      }
    pb->Cf = (int)map.size();
    pb->n = 3 * pb->Cf;
    // the block-Jacobi PCG takes the centre system in 9-unknown super-blocks of
    // three cameras: order padded to 9 ceil(Cf / 3) with identity rows
    pb->Cs = (pb->Cf + 2) / 3;
    pb->n_pad = 9 * pb->Cs;
    GST(galloc(pb, &pb->crank, (size_t)C));
    GST(galloc(pb, &pb->cam_map, (size_t)pb->Cf));
    if (C) GCU(cudaMemcpyAsync(pb->crank, rank.data(), sizeof(int) * C, cudaMemcpyHostToDevice, pb->stream));
    if (pb->Cf) GCU(cudaMemcpyAsync(pb->cam_map, map.data(), sizeof(int) * pb->Cf, cudaMemcpyHostToDevice, pb->stream));
    GST(gp_sync(pb));
  }
  // Sec. 4.1 partition: free flags, their ascending ranks (prefix scan) and the map back
  {
    uint8_t* flags = nullptr;
    GST(galloc(pb, &flags, (size_t)N));
    GST(galloc(pb, &pb->free_rank, (size_t)N));
    GST(galloc(pb, &pb->free_map, (size_t)N));
    int* d_count = nullptr;
    GST(galloc(pb, &d_count, 1));
    const int nb = rank_blocks(N) + 1;
    int* tmp = nullptr;
    GST(galloc(pb, &tmp, (size_t)nb));
    if (N) GLAUNCH(pb, 1, gpk::k_gp_free_flags<<<gpk::blocks(N, 256), 256, 0, pb->stream>>>(N, pb->depth_in, flags));
    GCU(launch_rank(flags, N, pb->free_rank, pb->free_map, d_count, tmp, nb, pb->stream));
    pb->launches += 3;
    int h = 0;
    GCU(cudaMemcpyAsync(&h, d_count, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
    GST(gp_sync(pb));
    pb->F = h;
  }
  GST(galloc(pb, &pb->ray4, (size_t)N));
  GST(galloc(pb, &pb->ray64, (size_t)N));
  GST(galloc(pb, &pb->po_sidx, (size_t)N));
  if (N)
    GLAUNCH(pb, 1, gpk::k_gp_obs<<<gpk::blocks(N, 256), 256, 0, pb->stream>>>(
                       N, pb->po, d_rays, pb->depth_in, pb->free_rank, pb->ray4, pb->ray64, pb->po_sidx));
  for (int s = 0; s < 2; ++s) {
    GST(galloc(pb, &pb->t64[s], (size_t)3 * C));
    GST(galloc(pb, &pb->X64[s], (size_t)3 * P));
    GST(galloc(pb, &pb->s64[s], (size_t)pb->F));
    GST(galloc(pb, &pb->cw[s], (size_t)C));
    GST(galloc(pb, &pb->pw[s], (size_t)P));
    GST(galloc(pb, &pb->sw[s], (size_t)pb->F));
  }
  if (C) GCU(cudaMemcpyAsync(pb->t64[0], d_t, sizeof(double) * 3 * C, cudaMemcpyDeviceToDevice, pb->stream));
  if (P) GCU(cudaMemcpyAsync(pb->X64[0], d_X, sizeof(double) * 3 * P, cudaMemcpyDeviceToDevice, pb->stream));
  if (pb->F)
    GLAUNCH(pb, 1, gpk::k_gp_gather_scales<<<gpk::blocks(pb->F, 256), 256, 0, pb->stream>>>(
                       pb->F, pb->free_map, d_s0, pb->s64[0], pb->sw[0]));
  GLAUNCH(pb, 1, gpk::k_gp_prep<<<gpk::blocks(std::max(C, P), 256), 256, 0, pb->stream>>>(C, P, pb->t64[0], pb->X64[0],
                                                                                         pb->cw[0], pb->pw[0]));
  // working arrays
  GST(galloc(pb, &pb->rec, (size_t)gpk::kRec * N));
  GST(galloc(pb, &pb->Y, (size_t)3 * N));
  GST(galloc(pb, &pb->ptrec, (size_t)gpk::kPtRec * P));
  GST(galloc(pb, &pb->part, (size_t)gpk::kPartStride * std::max(1, pb->n_chunks)));
  GST(galloc(pb, &pb->Sdiag, (size_t)6 * pb->Cf));
  GST(galloc(pb, &pb->camrec, (size_t)pb->Cf));
  GST(galloc(pb, &pb->b, (size_t)pb->n));
  GST(galloc(pb, &pb->bh, (size_t)std::max(pb->n_pad, pb->n)));
  GST(galloc(pb, &pb->xh, (size_t)std::max(pb->n_pad, pb->n)));
  GST(galloc(pb, &pb->dt, (size_t)pb->n));
  GST(galloc(pb, &pb->dsc, (size_t)pb->n));
  GST(galloc(pb, &pb->dX, (size_t)P));
  GST(galloc(pb, &pb->ds, (size_t)pb->F));
  pb->use_dense = opts->solver == BA_SOLVER_DENSE;
  if (opts->solver != BA_SOLVER_AUTO && opts->solver != BA_SOLVER_EXPLICIT && opts->solver != BA_SOLVER_DENSE) {
    gp_error("GP solver must be BA_SOLVER_AUTO, BA_SOLVER_EXPLICIT or BA_SOLVER_DENSE");
    return BA_ERR_INVALID_ARG;
  }
  pb->ld = spcg_row_stride<float>(std::max(pb->n_pad, 1));
  if ((size_t)pb->n_pad * pb->ld * 4 > ((size_t)16 << 30)) {
    gp_error("centre system of order %d is too large for the explicit solve", pb->n);
    return BA_ERR_INVALID_ARG;
  }
  GST(galloc(pb, &pb->Sh, (size_t)std::max(pb->n_pad, 1) * pb->ld));
  if (!pb->use_dense && pb->Cf > 0) {
    const int n = pb->n_pad;
    GST(galloc(pb, &pb->Dinv, (size_t)81 * pb->Cs));
    GST(galloc(pb, &pb->dscale, (size_t)2 * n));
    GLAUNCH(pb, 1, gpk::k_gp_ones<<<gpk::blocks(n, 256), 256, 0, pb->stream>>>(n, pb->dscale));
    const size_t nw = (size_t)2 * n * spcg_words_per_value(false);
    GST(galloc(pb, &pb->words, nw));
    GCU(cudaMemsetAsync(pb->words, 0, sizeof(unsigned long long) * nw, pb->stream));
    int optin = 0;
    GCU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pb->device));
    pb->pcg_grid = std::max(1, std::min(pb->num_sms, (n + 7) / 8));
    const int rows_max = std::max(8, (n + pb->pcg_grid - 1) / pb->pcg_grid);
    auto bytes = [&](int ri, int vi) { return spcg_smem_bytes<float>(n, rows_max, ri, vi, pb->Cs); };
    if (bytes(1, 1) > (size_t)optin) pb->pcg_rows_in_smem = 0;
    if (!pb->pcg_rows_in_smem && bytes(0, 1) > (size_t)optin) pb->pcg_vecs_in_smem = 0;
    pb->pcg_smem = bytes(pb->pcg_rows_in_smem, pb->pcg_vecs_in_smem);
    if (pb->pcg_smem > (size_t)optin) {
      gp_error("centre system PCG of order %d needs %zu B of shared memory per block", n, pb->pcg_smem);
      return BA_ERR_INVALID_ARG;
    }
    if (!pb->pcg_vecs_in_smem) {
      pb->pcg_scratch_stride = (size_t)4 * spcg_row_stride<float>(n);
      GST(galloc(pb, &pb->pcg_scratch, pb->pcg_scratch_stride * pb->pcg_grid));
      GST(galloc(pb, &pb->pcg_M, (size_t)kSpcgMStride * pb->Cs));
    }
    const void* fn = spcg_kernel_ptr<float>(pb->pcg_rows_in_smem != 0);
    GCU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pb->pcg_smem));
    int per = 0;
    GCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, spcg_threads(), pb->pcg_smem));
    if (per < 1 || pb->pcg_grid > per * pb->num_sms) {
      gp_error("centre system PCG kernel cannot be resident");
      return BA_ERR_INVALID_ARG;
    }
  }
  if (pb->use_dense) {
    const size_t np = ((size_t)pb->n + 127) / 128 * 128;
    GST(galloc(pb, &pb->dw.A, np * np));
    GST(galloc(pb, &pb->dw.Linv, np * 128));
    GST(galloc(pb, &pb->dw.vec, 4 * np));
    GST(galloc(pb, &pb->dw.part, (size_t)256));
    GST(galloc(pb, &pb->dw.scal, (size_t)8));
    GST(galloc(pb, &pb->dw.flags, np / 128 + 1));
    GCU(cudaMemsetAsync(pb->dw.flags, 0, sizeof(unsigned) * (np / 128 + 1), pb->stream));
    GST(galloc(pb, &pb->dw.err, (size_t)1));
    pb->dw.epoch = &pb->dense_epoch;
  }
  pb->bs_grid = gpk::blocks(P, gpk::kThreads);
  GST(galloc(pb, &pb->pred_parts, (size_t)pb->bs_grid));
  pb->eval_grid = std::max(1, std::min(pb->num_sms * 8, gpk::blocks(N, 256)));
  GST(galloc(pb, &pb->eval_parts, (size_t)2 * pb->eval_grid));
  GST(galloc(pb, &pb->scales_out, (size_t)N));
  GST(galloc(pb, &pb->steps_out, (size_t)3 * C + 3 * (size_t)P + N));
  GST(galloc(pb, &pb->sc, 1));
  GCU(cudaMemsetAsync(pb->sc, 0, sizeof(Scalars), pb->stream));
  GCU(cudaMallocHost(&pb->h_sc, sizeof(Scalars)));
  memset(pb->h_sc, 0, sizeof(Scalars));
  for (auto& e : pb->ev) GCU(cudaEventCreate(&e));
  GST(gp_sync(pb));
  return BA_OK;
}

ba_status gp_eval(ba_gp_problem* pb, int slot) {
  GLAUNCH(pb, 1, gpk::k_gp_eval<<<pb->eval_grid, 256, 0, pb->stream>>>(
                     pb->N, pb->po_cam, pb->po_pt, pb->po_sidx, pb->ray64, pb->t64[slot], pb->X64[slot],
                     pb->s64[slot], pb->opt.huber_delta, pb->eval_parts, pb->sc, slot));
  return BA_OK;
}

// Steps (a)-(d) at damping lambda: linearisation with the scales eliminated,
// the centre system, its tensor-core solve and the back-substitution; leaves
// dt (rank order), dX, ds and sc->pred.
ba_status gp_solve_damped(ba_gp_problem* pb, double lambda, DenseResult* dres) {
  const int s = pb->cur, P = pb->P, Cf = pb->Cf, n = pb->n;
  const float lam = (float)lambda;
  GCU(cudaMemsetAsync(pb->err, 0, sizeof(int), pb->stream));
  GCU(cudaEventRecord(pb->ev[0], pb->stream));
  if (P)
    GLAUNCH(pb, 1, gpk::k_gp_point<<<gpk::blocks(P, gpk::kThreads), gpk::kThreads, 0, pb->stream>>>(
                       P, pb->pt_off, pb->po_cam, pb->po_sidx, pb->ray4, pb->cw[s], pb->pw[s], pb->sw[s], lam,
                       (float)pb->opt.huber_delta, pb->rec, pb->Y, pb->ptrec));
  if (pb->n_chunks)
    GLAUNCH(pb, 1, gpk::k_gp_cam_chunk<<<pb->n_chunks, gpk::kThreads, 0, pb->stream>>>(
                       pb->chunk_obs, pb->chunk_cam, pb->crank, pb->co_po, pb->po_pt, pb->rec, pb->Y, pb->ptrec,
                       pb->part));
  GCU(cudaEventRecord(pb->ev[1], pb->stream));
  *dres = DenseResult{};
  if (Cf) {
    GLAUNCH(pb, 1, gpk::k_gp_cam_finish<<<gpk::blocks(Cf, 128), 128, 0, pb->stream>>>(
                       Cf, pb->cam_map, pb->cam_chunk, pb->part, lam, pb->Sdiag, pb->b, pb->dsc, pb->camrec, pb->err));
    GCU(cudaMemsetAsync(pb->Sh, 0, sizeof(float) * (size_t)pb->n_pad * pb->ld, pb->stream));
    if (pb->n_pad > n)
      GLAUNCH(pb, 1, gpk::k_gp_pad<<<1, 32, 0, pb->stream>>>(n, pb->n_pad, pb->Sh, pb->ld));
    GLAUNCH(pb, 1, gpk::k_gp_S_diag<<<gpk::blocks(Cf, 128), 128, 0, pb->stream>>>(Cf, pb->Sdiag, pb->dsc, pb->Sh, pb->ld));
    if (pb->n_runs)
      GLAUNCH(pb, 1, gpk::k_gp_form_S<<<std::min(gpk::blocks(pb->n_runs, 4), 32 * pb->num_sms), gpk::kThreads, 0,
                                        pb->stream>>>(pb->n_runs, pb->runs, pb->pairs, pb->crank, pb->rec, pb->Y,
                                                      pb->dsc, pb->Sh, pb->ld));
    if (pb->n_pad > n) GCU(cudaMemsetAsync(pb->bh + n, 0, sizeof(float) * (pb->n_pad - n), pb->stream));
    GLAUNCH(pb, 1, gpk::k_gp_scale<<<gpk::blocks(n, 256), 256, 0, pb->stream>>>(n, pb->b, pb->dsc, pb->bh));
    GCU(cudaEventRecord(pb->ev[2], pb->stream));
    if (pb->use_dense) {
      GCU(dense_spd_solve(pb->dw, pb->Sh, pb->ld, n, pb->bh, pb->xh, pb->opt.pcg_rel_tol, pb->opt.pcg_max_iters,
                          pb->num_sms, pb->stream, dres));
      pb->launches += dres->launches;
    } else {
      // block-Jacobi PCG on the scaled system with the explicit PCG kernel: three
      // cameras form one of its 9-unknown blocks; unit scaling (already scaled)
      GLAUNCH(pb, 1, gpk::k_gp_superblock_inv<<<gpk::blocks(pb->Cs, gpk::kSbWarps), 32 * gpk::kSbWarps, 0,
                                                pb->stream>>>(pb->Cs, pb->Sh, pb->ld, pb->Dinv));
      SpcgArgs<float> a{};
      a.Shat = pb->Sh;
      a.Dinv = pb->Dinv;
      a.dscale = pb->dscale;
      a.b = pb->bh;
      a.Cf = pb->Cs;
      a.n = pb->n_pad;
      a.rows_in_smem = pb->pcg_rows_in_smem;
      a.vecs_in_smem = pb->pcg_vecs_in_smem;
      a.scratch = pb->pcg_scratch;
      a.scratch_stride = pb->pcg_scratch_stride;
      a.Mshared = nullptr;
      if (pb->pcg_M) {
        GCU(launch_spcg_precond<float>(pb->Cs, pb->Dinv, pb->dscale, pb->pcg_M, pb->stream));
        pb->launches += 1;
        a.Mshared = pb->pcg_M;
      }
      a.x = pb->xh;
      a.words = pb->words;
      a.err = pb->err;
      a.sc = pb->sc;
      a.tol = pb->opt.pcg_rel_tol;
      a.max_iters = pb->opt.pcg_max_iters;
      a.timeout_ns = 2000000000LL;
      const unsigned span = (unsigned)a.max_iters + 2u;
      if (pb->tag == 0 || pb->tag > 0xFFFFFFFFu - span) {
        GCU(cudaMemsetAsync(pb->words, 0, sizeof(unsigned long long) * 2 * (size_t)pb->n_pad *
                                              spcg_words_per_value(false), pb->stream));
        pb->tag = 1;
      }
      a.tag_base = pb->tag;
      pb->tag += span;
      GCU(launch_spcg<float>(a, pb->pcg_grid, pb->pcg_smem, pb->stream));
      pb->launches += 1;
      dres->iters = -1;  // read back with the scalars
    }
    GLAUNCH(pb, 1, gpk::k_gp_scale<<<gpk::blocks(n, 256), 256, 0, pb->stream>>>(n, pb->xh, pb->dsc, pb->dt));
  } else {
    GCU(cudaEventRecord(pb->ev[2], pb->stream));
  }
  GCU(cudaEventRecord(pb->ev[3], pb->stream));
  GLAUNCH(pb, 1, gpk::k_gp_backsub<<<pb->bs_grid, gpk::kThreads, 0, pb->stream>>>(
                     P, pb->pt_off, pb->po_cam, pb->po_sidx, pb->crank, pb->cw[s], pb->pw[s], pb->rec, pb->ptrec,
                     pb->dt, lam, pb->dX, pb->ds, pb->pred_parts));
  GLAUNCH(pb, 1, gpk::k_gp_pred_cams<<<1, 256, 0, pb->stream>>>(Cf, pb->dt, pb->camrec, lam, pb->pred_parts,
                                                                 P ? pb->bs_grid : 0, pb->sc));
  return BA_OK;
}

ba_status gp_lm_step(ba_gp_problem* pb, ba_iter_info* info) {
  if (!pb->cost_valid) {
    GST(gp_eval(pb, pb->cur));
    pb->cost_valid = true;
  }
  const double lambda = pb->lambda;
  DenseResult dres;
  GST(gp_solve_damped(pb, lambda, &dres));
  const int s = pb->cur, d = 1 - pb->cur;
  GLAUNCH(pb, 1, gpk::k_gp_candidate<<<gpk::blocks(std::max(std::max(pb->C, pb->P), pb->F), 256), 256, 0, pb->stream>>>(
                     pb->C, pb->P, pb->F, pb->crank, pb->dt, pb->dX, pb->ds, pb->t64[s], pb->X64[s], pb->s64[s],
                     pb->t64[d], pb->X64[d], pb->s64[d], pb->cw[d], pb->pw[d], pb->sw[d]));
  GST(gp_eval(pb, d));
  GCU(cudaEventRecord(pb->ev[4], pb->stream));
  GCU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  int h_err = 0;
  GCU(cudaMemcpyAsync(&h_err, pb->err, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
  GST(gp_sync(pb));
  const Scalars& sc = *pb->h_sc;
  if (dres.iters < 0) {  // the PCG kernel's own count and residual
    dres.iters = sc.pcg_iters;
    dres.rel_res = sc.pcg_rel_res;
  }
  const double F = sc.cost[s], Fc = sc.cost[d], pred = sc.pred;
  const double gain = (F - Fc) / pred;
  const bool timeout = (dres.flags & 16) != 0 || (h_err & 1) != 0;
  const bool ok = std::isfinite(Fc) && std::isfinite(gain) && pred > 0.0 && !timeout && !(h_err & 4);
  const bool accept = ok && gain > 1e-3;
  if (info) {
    memset(info, 0, sizeof *info);
    info->cost = F;
    info->rmse_px = pb->N > 0 ? std::sqrt(sc.rmse_sum[s] / pb->N) : 0.0;
    info->lambda = lambda;
    info->gain = gain;
    info->pred_decrease = pred;
    info->cand_cost = Fc;
    info->accepted = accept ? 1 : 0;
    info->pcg_iters = dres.iters;
    info->pcg_rel_res = dres.rel_res;
    info->n_cam_act = pb->Cf;
    info->n_pt_act = pb->P;
    info->n_obs_act = pb->F;
    cudaEventElapsedTime(&info->ms[0], pb->ev[0], pb->ev[1]);
    cudaEventElapsedTime(&info->ms[1], pb->ev[1], pb->ev[2]);
    cudaEventElapsedTime(&info->ms[2], pb->ev[2], pb->ev[3]);
    cudaEventElapsedTime(&info->ms[3], pb->ev[3], pb->ev[4]);
    cudaEventElapsedTime(&info->ms[6], pb->ev[0], pb->ev[4]);
  }
  if (accept) {
    pb->cur = d;
    const double t = 2.0 * gain - 1.0;
    pb->lambda = lambda * std::max(1.0 / 3.0, 1.0 - t * t * t);
    pb->nu = 2.0;
  } else {
    pb->lambda = lambda * pb->nu;
    pb->nu *= 2.0;
  }
  pb->iter++;
  if (timeout) {
    gp_error("dense solve pipeline timed out");
    return BA_ERR_TIMEOUT;
  }
  if (!ok) return BA_ERR_NONFINITE;
  if (dres.iters >= pb->opt.pcg_max_iters && dres.rel_res > pb->opt.pcg_rel_tol) return BA_ERR_NOT_CONVERGED;
  return BA_OK;
}

}  // namespace

extern "C" {

void ba_gp_default_options(ba_gp_options* o) {
  static const int32_t kGauge[1] = {0};
  memset(o, 0, sizeof *o);
  o->huber_delta = 0.1;
  o->lambda0 = 1e-4;
  o->pcg_rel_tol = 1e-6;
  o->pcg_max_iters = 500;
  o->fixed_cams = kGauge;
  o->n_fixed = 1;
  o->solver = BA_SOLVER_AUTO;
}

ba_status ba_gp_create(const ba_gp_options* opts, void* stream, int64_t n_cams, const double* centres,
                       int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                       const int32_t* obs_pt, const double* rays, const double* depth, const double* scales0,
                       ba_gp_problem** out) {
  if (!out) {
    gp_error("null output handle");
    return BA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  ba_gp_problem* pb = new ba_gp_problem();
  ba_status st = gp_create_impl(opts, stream, n_cams, centres, n_pts, pts, n_obs, obs_cam, obs_pt, rays, depth,
                                scales0, pb);
  if (st != BA_OK) {
    gp_free(pb);
    return st;
  }
  *out = pb;
  return BA_OK;
}

ba_status ba_gp_lm_step(ba_gp_problem* pb, ba_iter_info* info) {
  if (!pb) return BA_ERR_INVALID_ARG;
  return gp_lm_step(pb, info);
}

ba_status ba_gp_solve(ba_gp_problem* pb, int max_iters, ba_iter_info* log, int* n_done) {
  if (!pb || max_iters < 0) return BA_ERR_INVALID_ARG;
  ba_status last = BA_OK;
  int i = 0;
  for (; i < max_iters; ++i) {
    ba_status st = gp_lm_step(pb, log ? log + i : nullptr);
    if (st != BA_OK && st != BA_ERR_NOT_CONVERGED && st != BA_ERR_NONFINITE) {
      if (n_done) *n_done = i + 1;
      return st;
    }
    if (st != BA_OK) last = st;
  }
  if (n_done) *n_done = i;
  return last == BA_ERR_NONFINITE ? BA_OK : last;
}

ba_status ba_gp_get_params(ba_gp_problem* pb, double* centres, double* pts, double* scales) {
  if (!pb) return BA_ERR_INVALID_ARG;
  const int s = pb->cur;
  if (centres && pb->C)
    GCU(cudaMemcpyAsync(centres, pb->t64[s], sizeof(double) * 3 * pb->C, cudaMemcpyDefault, pb->stream));
  if (pts && pb->P) GCU(cudaMemcpyAsync(pts, pb->X64[s], sizeof(double) * 3 * pb->P, cudaMemcpyDefault, pb->stream));
  if (scales && pb->N) {
    GLAUNCH(pb, 1, gpk::k_gp_scales_out<<<gpk::blocks(pb->N, 256), 256, 0, pb->stream>>>(
                       pb->N, pb->depth_in, pb->free_rank, pb->s64[s], pb->scales_out));
    GCU(cudaMemcpyAsync(scales, pb->scales_out, sizeof(double) * pb->N, cudaMemcpyDefault, pb->stream));
  }
  return gp_sync(pb);
}

ba_status ba_gp_get_free(ba_gp_problem* pb, int32_t* free_rank, int64_t* n_free) {
  if (!pb) return BA_ERR_INVALID_ARG;
  if (free_rank && pb->N)
    GCU(cudaMemcpyAsync(free_rank, pb->free_rank, sizeof(int32_t) * pb->N, cudaMemcpyDefault, pb->stream));
  if (n_free) *n_free = pb->F;
  return gp_sync(pb);
}

ba_status ba_gp_solve_damped(ba_gp_problem* pb, double lambda, double* dt, double* dX, double* ds,
                             ba_iter_info* info) {
  if (!pb || !(lambda >= 0.0) || !std::isfinite(lambda)) return BA_ERR_INVALID_ARG;
  DenseResult dres;
  GST(gp_solve_damped(pb, lambda, &dres));
  double* o = pb->steps_out;
  const int m = std::max(std::max(pb->C, pb->P), pb->N);
  GLAUNCH(pb, 1, gpk::k_gp_steps_out<<<gpk::blocks(m, 256), 256, 0, pb->stream>>>(
                     pb->C, pb->P, pb->N, pb->crank, pb->free_rank, pb->dt, pb->dX, pb->ds, o, o + 3 * (size_t)pb->C,
                     o + 3 * (size_t)pb->C + 3 * (size_t)pb->P));
  if (dt && pb->C) GCU(cudaMemcpyAsync(dt, o, sizeof(double) * 3 * pb->C, cudaMemcpyDefault, pb->stream));
  if (dX && pb->P)
    GCU(cudaMemcpyAsync(dX, o + 3 * (size_t)pb->C, sizeof(double) * 3 * pb->P, cudaMemcpyDefault, pb->stream));
  if (ds && pb->N)
    GCU(cudaMemcpyAsync(ds, o + 3 * (size_t)pb->C + 3 * (size_t)pb->P, sizeof(double) * pb->N, cudaMemcpyDefault,
                        pb->stream));
  GCU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  GST(gp_sync(pb));
  if (info) {
    memset(info, 0, sizeof *info);
    info->lambda = lambda;
    info->pred_decrease = pb->h_sc->pred;
    info->pcg_iters = dres.iters < 0 ? pb->h_sc->pcg_iters : dres.iters;
    info->pcg_rel_res = dres.iters < 0 ? pb->h_sc->pcg_rel_res : dres.rel_res;
  }
  return BA_OK;
}

ba_status ba_gp_eval_cost(ba_gp_problem* pb, double* cost, double* rms) {
  if (!pb) return BA_ERR_INVALID_ARG;
  GST(gp_eval(pb, pb->cur));
  GCU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  GST(gp_sync(pb));
  if (cost) *cost = pb->h_sc->cost[pb->cur];
  if (rms) *rms = pb->N > 0 ? std::sqrt(pb->h_sc->rmse_sum[pb->cur] / pb->N) : 0.0;
  return BA_OK;
}

int64_t ba_gp_kernel_launches(const ba_gp_problem* pb) { return pb ? pb->launches : 0; }

void ba_gp_destroy(ba_gp_problem* pb) { gp_free(pb); }

}  // extern "C"
