// schur_explicit.cu -- step (b)/(d) on an explicit reduced camera system.
//
// When the free cameras are few enough for the Schur complement
//   S = U* - sum_p sum_{k,k' in p} W_k V*_p^-1 W_k'^T          (Eq. LM, Schur form)
// to be held densely, it is formed once per damping value and the PCG runs on
// it directly: each block keeps its rows of S in shared memory, so a matvec is
// a dense row-block product with no cross-block partial sums.
//
// S is formed Jacobi-scaled, S^ = D^-1 S D^-1 with D = sqrt(diag U*), so every
// entry is of order one.  Off-diagonal blocks S_ij (i < j) are sums over the
// points both cameras see; those pairs of observations are listed once at set-up
// (the co-visibility runs), so each block is summed by one warp (or, with very
// many short runs, one lane) in registers in a fixed order: no atomics,
// bit-reproducible.  The diagonal blocks come from the block-Jacobi pass
// (U* - sum W V*^-1 W^T) and the lower triangle is mirrored.  The same blocks feed
// the block-sparse storage and its partitioned PCG further down.
#include <cuda/atomic>
#include <type_traits>

#include "df.cuh"
#include "internal.h"
#include "model.cuh"

namespace bab {


template <typename T>
__device__ __forceinline__ void load_cam_rec(const T* __restrict__ camw, int c, T cw[kCamStride]) {
#pragma unroll
  for (int q = 0; q < kCamStride; ++q) cw[q] = camw[kCamStride * (size_t)c + q];
}

// W = rho' Jc^T Jp of one observation, 9x3 row-major.
template <typename T>
__device__ __forceinline__ void obs_W(const T* cw, const T* X, T u, T v, T tau, const ModelParams& mp,
                                      T W[27]) {
  T sw = tau > T(0) ? (T)mp.sw_valid : (T)mp.sw_invalid;
  ObsLin<T> o;
  linearize_obs<T>(cw, X[0], X[1], X[2], u, v, tau, sw, (T)mp.cx, (T)mp.cy, (T)mp.huber, o);
#pragma unroll
  for (int a = 0; a < 9; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      W[3 * a + b] = o.wrob * (o.Jc[0][a] * o.Jp[0][b] + o.Jc[1][a] * o.Jp[1][b] + o.Jc[2][a] * o.Jp[2][b]);
}

// Per point-order observation k (camera a, point p): Y^_k = D_a^-1 W_k M_p with
// M_p M_p^T = V*_p^-1 (3x3 Cholesky), so that W_k V*_p^-1 W_k'^T scaled by the
// Jacobi factors is the plain product Y^_k Y^_k'^T.  A block takes 128
// consecutive rows: W rows are brought into shared memory with 16-byte
// coalesced loads, transformed in place one row per thread, and stored back the
// same way.  Rows of observations of cameras that are not free are zero (their
// blocks are never formed); an inactive observation has W = 0 and gets Y^ = 0.
constexpr int kYRows = 128;

template <typename T>
__global__ void __launch_bounds__(kYRows) k_form_Y(int N, int C, int P, const int* __restrict__ po_cam,
                                                  const int* __restrict__ po_pt, const T* __restrict__ W,
                                                  const T* __restrict__ Vinv, const int* __restrict__ crank,
                                                  const double* __restrict__ dscale, int Cf,
                                                  T* __restrict__ Y, const int* __restrict__ dst_row) {
  __shared__ __align__(16) T buf[kYRows * kWStride];
  constexpr int kVec = (int)(kWStride * sizeof(T) / 16);  // 16-byte words per row
  const int k0 = blockIdx.x * kYRows;
  const int rows = min(kYRows, N - k0);
  const uint4* src = reinterpret_cast<const uint4*>(W + kWStride * (size_t)k0);
  uint4* sb = reinterpret_cast<uint4*>(buf);
  for (int i = threadIdx.x; i < rows * kVec; i += kYRows) sb[i] = src[i];
  __syncthreads();
  const int t = threadIdx.x;
  if (t < rows) {
    const int k = k0 + t;
    T* y = buf + kWStride * t;
    const int a = crank[bidx(po_cam[k], C, 10)];
    if (a < 0) {
#pragma unroll
      for (int q = 0; q < 27; ++q) y[q] = T(0);
    } else {
      const T* dinv = reinterpret_cast<const T*>(dscale + 9 * Cf) + 9 * a;
      const T* vi = Vinv + 6 * (size_t)bidx(po_pt[k], P, 11);
      const T v00 = vi[0], v01 = vi[1], v02 = vi[2], v11 = vi[3], v12 = vi[4], v22 = vi[5];
      T l00 = T(0), l10 = T(0), l20 = T(0), l11 = T(0), l21 = T(0), l22 = T(0);
      if (v00 > T(0)) {
        l00 = sqrt(v00);
        const T r0 = T(1) / l00;
        l10 = v01 * r0;
        l20 = v02 * r0;
        const T d1 = v11 - l10 * l10;
        if (d1 > T(0)) {
          l11 = sqrt(d1);
          l21 = (v12 - l20 * l10) / l11;
        }
        const T d2 = v22 - l20 * l20 - l21 * l21;
        l22 = d2 > T(0) ? sqrt(d2) : T(0);
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const T w0 = y[3 * r], w1 = y[3 * r + 1], w2 = y[3 * r + 2], sc = dinv[r];
        y[3 * r] = sc * (w0 * l00 + w1 * l10 + w2 * l20);
        y[3 * r + 1] = sc * (w1 * l11 + w2 * l21);
        y[3 * r + 2] = sc * (w2 * l22);
      }
    }
  }
  __syncthreads();
  if (dst_row) {
    // camera-order rows: consecutive lanes store consecutive 16-byte words of a row
    for (int i = threadIdx.x; i < rows * kVec; i += kYRows) {
      const int r = i / kVec;
      reinterpret_cast<uint4*>(Y + kWStride * (size_t)dst_row[k0 + r])[i - r * kVec] = sb[i];
    }
  } else {
    uint4* dst = reinterpret_cast<uint4*>(Y + kWStride * (size_t)k0);
    for (int i = threadIdx.x; i < rows * kVec; i += kYRows) dst[i] = sb[i];
  }
}

template <typename T>
__device__ __forceinline__ void load_row27(const T* __restrict__ p, T v[27]);
template <>
__device__ __forceinline__ void load_row27<float>(const float* __restrict__ p, float v[27]) {
  const float4* q = reinterpret_cast<const float4*>(p);  // rows are 112-byte aligned
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float4 t = q[i];
    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
  }
  const float4 t = q[6];
  v[24] = t.x; v[25] = t.y; v[26] = t.z;
}
template <>
__device__ __forceinline__ void load_row27<double>(const double* __restrict__ p, double v[27]) {
  const double2* q = reinterpret_cast<const double2*>(p);  // rows are 224-byte aligned
#pragma unroll
  for (int i = 0; i < 13; ++i) {
    const double2 t = q[i];
    v[2 * i] = t.x; v[2 * i + 1] = t.y;
  }
  v[26] = p[26];
}

// One round of a warp reduce-scatter on a per-lane vector of length M (the
// first M entries of v): the lane keeps the half selected by bit r of its lane
// id, sends the other half to lane ^ 2^r and adds what that lane sends back.
// After the rounds for M = 96, 48, 24, 12, 6 lane L holds the full warp sums of
// entries 48 b0 + 24 b1 + 12 b2 + 6 b3 + 3 b4 + (0, 1, 2) of the original
// vector (b_r = bit r of L), in v[0..2]; the order of additions is fixed.
template <typename T, int M>
__device__ __forceinline__ void rs_round(T (&v)[96], int lane, int r) {
  constexpr int H = M / 2;
  const bool hi = (lane >> r) & 1;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const T send = hi ? v[i] : v[H + i];
    const T keep = hi ? v[H + i] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << r);
  }
}

// Off-diagonal blocks from the static co-visibility runs: run = every point seen
// by both cameras i < j, as pairs (k, k2) of point-order observations, ascending
// in point.  One warp per run: each lane sums Y^_k Y^_k2^T over its subset of the
// run in registers, then the lanes are reduced in a fixed order
// (deterministic).  Inactive observations have Y^ = 0 and add nothing; runs whose
// cameras are not both free are skipped.
// Three 128-thread blocks per SM: 81 accumulators and two 27-entry rows per lane
// fit without spilling (four blocks force 128 registers and spill: 19% slower).
// kSparse: Shat is the block storage of the block-sparse system: run r's block
// goes to slot 2 r and its transpose to slot 2 r + 1 (kBlkStride entries each).
template <typename T, bool kSparse>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 1)
    k_form_S_runs(int n_runs, const int4* __restrict__ runs, const int2* __restrict__ pairs,
                  const T* __restrict__ Y, const int* __restrict__ crank, int Cf, T* __restrict__ Shat, int C,
                  int N) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int ld = spcg_row_stride<T>(9 * Cf);
  for (int ri = gw; ri < n_runs; ri += nw) {
    const int4 rn = runs[ri];  // (camera i, camera j, first pair, pair count)
    const int a = crank[bidx(rn.x, C, 12)], b = crank[bidx(rn.y, C, 12)];
    if (a < 0 || b < 0) continue;
    T acc[81];
#pragma unroll
    for (int q = 0; q < 81; ++q) acc[q] = T(0);
    const int qe = rn.z + rn.w;
    int q = rn.z + lane;
    int2 nxt = q < qe ? pairs[q] : make_int2(0, 0);
    for (; q < qe; q += 32) {
      const int2 pr = nxt;
      if (q + 32 < qe) nxt = pairs[q + 32];  // next pair's indices in flight during this one
      T y1[27], y2[27];
      load_row27<T>(Y + kWStride * (size_t)bidx(pr.x, N, 13), y1);
      load_row27<T>(Y + kWStride * (size_t)bidx(pr.y, N, 13), y2);
#pragma unroll
      for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int s2 = 0; s2 < 9; ++s2)
          acc[9 * r + s2] += y1[3 * r] * y2[3 * s2] + y1[3 * r + 1] * y2[3 * s2 + 1] + y1[3 * r + 2] * y2[3 * s2 + 2];
    }
    // warp reduce-scatter of the 81 sums (padded to 96): lane keeps three finished sums
    T v[96];
#pragma unroll
    for (int t = 0; t < 96; ++t) v[t] = t < 81 ? acc[t] : T(0);
    rs_round<T, 96>(v, lane, 0);
    rs_round<T, 48>(v, lane, 1);
    rs_round<T, 24>(v, lane, 2);
    rs_round<T, 12>(v, lane, 3);
    rs_round<T, 6>(v, lane, 4);
    const int base = 48 * (lane & 1) + 24 * ((lane >> 1) & 1) + 12 * ((lane >> 2) & 1) + 6 * ((lane >> 3) & 1) +
                     3 * ((lane >> 4) & 1);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int t = base + j;
      if (t < 81) {
        const int r = t / 9, s2 = t - 9 * r;
        if constexpr (kSparse) {
          Shat[(size_t)kBlkStride * (2 * (size_t)ri) + 9 * r + s2] = -v[j];
          Shat[(size_t)kBlkStride * (2 * (size_t)ri + 1) + 9 * s2 + r] = -v[j];
        } else {
          Shat[(size_t)(9 * a + r) * ld + 9 * b + s2] = -v[j];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same blocks from observation records (FP32, warp per run).  With D the
// derivative of the residual in the camera frame (model.cuh), the camera Jacobian
// factors as Jc = [D N | D T | e g^T]: N = -[a]x (a = R X, or R X + t for the
// centre model), T = I (or -R for the centre model's centre columns), e = (xn, yn,
// 0) and g = (dist, f rr, f rr^2) (or (dist, 0, 0) for the centre model, whose
// dist is 1); the point Jacobian is Jp = D R and W = w Jc^T Jp.  The pair term
// W_k V*_p^-1 W_k2^T then needs, per observation, G = w D^T D, u = w D^T e, g and a
// (the record, 64 B, written by the point-side linearisation and independent of
// the damping) and, per pair,
//   M = R_i V*_p^-1 R_j^T,  L = G M G2,  h = G M u2,  h2 = G2 M^T u,  c = u . M u2:
//   rot-rot [a]x L N2, rot-trans [a]x L T2, trans-rot T^T L N2, trans-trans T^T L T2,
//   rot-intr ([a]x h) g2^T, trans-intr (T^T h) g2^T, intr-rot g (a2 x h2)^T,
//   intr-trans g (T2^T h2)^T, intr-intr c g g2^T.
// A pair reads two observation records and the point's record (V*^-1, 32 B,
// written with V*^-1 by the point damping): 160 B in five 32-byte loads, against
// two 112-byte rows of Y^ = D^-1 W M_p, and no Y^ pass runs.  The latency of these
// scattered gathers is what limits this kernel (12 resident warps per SM at 168
// registers); the 32-byte loads and the stored a and g keep the loads and the
// per-pair arithmetic few.  The Jacobi
// scaling is applied to the summed block.  Each lane sums its pairs in order (the
// intrinsic rows' 27 sums in shared memory, the other 54 in registers) and the
// lanes are reduced in a fixed butterfly (deterministic).
// ---------------------------------------------------------------------------
// one 32-byte read-only load (32-byte aligned address)
__device__ __forceinline__ void ld_nc_v8(const float* __restrict__ p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}
// observation record [16]: G00 G01 G02 G11 G12 G22 u0 u1 | u2 g0 g1 g2 a0 a1 a2 0
struct ObsRec {
  float g00, g01, g02, g11, g12, g22, u0, u1, u2, gi0, gi1, gi2, a0, a1, a2;
};
__device__ __forceinline__ ObsRec load_rec(const float* __restrict__ rec, int k) {
  float x[8], y[8];
  ld_nc_v8(rec + 16 * (size_t)k, x);
  ld_nc_v8(rec + 16 * (size_t)k + 8, y);
  return ObsRec{x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], y[0], y[1], y[2], y[3], y[4], y[5], y[6]};
}
// symmetric 3 x 3 G of a record times a general 3 x 3 B (rows r of G B)
__device__ __forceinline__ void rec_gmul(const ObsRec& r, const float (&B)[3][3], float (&out)[3][3]) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    out[0][t] = r.g00 * B[0][t] + r.g01 * B[1][t] + r.g02 * B[2][t];
    out[1][t] = r.g01 * B[0][t] + r.g11 * B[1][t] + r.g12 * B[2][t];
    out[2][t] = r.g02 * B[0][t] + r.g12 * B[1][t] + r.g22 * B[2][t];
  }
}
__device__ __forceinline__ void rec_gvec(const ObsRec& r, const float (&v)[3], float (&out)[3]) {
  out[0] = r.g00 * v[0] + r.g01 * v[1] + r.g02 * v[2];
  out[1] = r.g01 * v[0] + r.g11 * v[1] + r.g12 * v[2];
  out[2] = r.g02 * v[0] + r.g12 * v[1] + r.g22 * v[2];
}

// Z N2 added into rows r0.. of acc at column 0 (N2 = -[a2]x)
template <int K>
__device__ __forceinline__ void acc_times_n(float (&acc)[K], int row0, const float (&Z)[3][3], const float (&a2)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    acc[9 * (row0 + r) + 0] += -Z[r][1] * a2[2] + Z[r][2] * a2[1];
    acc[9 * (row0 + r) + 1] += Z[r][0] * a2[2] - Z[r][2] * a2[0];
    acc[9 * (row0 + r) + 2] += -Z[r][0] * a2[1] + Z[r][1] * a2[0];
  }
}
// Z T2 added into rows row0.. at columns 3-5 (T2 = I, or -R_j for the centre model)
template <bool kCentre, int K>
__device__ __forceinline__ void acc_times_t(float (&acc)[K], int row0, const float (&Z)[3][3], const float* Rj) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int t = 0; t < 3; ++t)
      acc[9 * (row0 + r) + 3 + t] +=
          kCentre ? -(Z[r][0] * Rj[t] + Z[r][1] * Rj[3 + t] + Z[r][2] * Rj[6 + t]) : Z[r][t];
}

template <bool kSparse, bool kCentre>
__global__ void __launch_bounds__(128, 3)
    k_form_S_rec(int n_runs, const int4* __restrict__ runs, const int2* __restrict__ pairs,
                 const int* __restrict__ pair_pt, const float* __restrict__ orec, const float* __restrict__ prec,
                 const float* __restrict__ camw, const double* __restrict__ dscale,
                 const int* __restrict__ crank, int Cf, float* __restrict__ Shat, int C, int N, int P) {
  __shared__ float cam_s[4][32];
  __shared__ float sacc_s[4][27 * 32];  // the intrinsic rows' sums, entry t of lane l at 32 t + l
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* sacc = sacc_s[wib] + lane;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int ld = spcg_row_stride<float>(9 * Cf);
  const float* dinv = reinterpret_cast<const float*>(dscale + 9 * (size_t)Cf);
  for (int ri = gw; ri < n_runs; ri += nw) {
    const int4 rn = runs[ri];  // (camera i, camera j, first pair, pair count)
    const int ci_ = bidx(rn.x, C, 39), cj_ = bidx(rn.y, C, 39);
    const int a = crank[ci_], b = crank[cj_];
    if (a < 0 || b < 0) continue;
    // the two cameras' rotations (the first 9 entries of the working records)
    __syncwarp();
    if (lane < 9) cam_s[wib][lane] = camw[kCamStride * (size_t)ci_ + lane];
    else if (lane >= 16 && lane < 25) cam_s[wib][lane] = camw[kCamStride * (size_t)cj_ + lane - 16];
    __syncwarp();
    const float* ci = cam_s[wib];
    const float* cj = cam_s[wib] + 16;
    float acc[54];  // rows 0-5 (rotation, translation); rows 6-8 in sacc
#pragma unroll
    for (int q = 0; q < 54; ++q) acc[q] = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) sacc[32 * t] = 0.f;
    const int qe = rn.z + rn.w;
    int q = rn.z + lane;
    int2 nxt = q < qe ? pairs[q] : make_int2(0, 0);
    int npt = q < qe ? pair_pt[q] : 0;
    for (; q < qe; q += 32) {
      const int2 pr = nxt;
      const int p = bidx(npt, P, 40);
      if (q + 32 < qe) nxt = pairs[q + 32], npt = pair_pt[q + 32];  // next pair's indices in flight
      const ObsRec r1 = load_rec(orec, bidx(pr.x, N, 41)), r2 = load_rec(orec, bidx(pr.y, N, 41));
      float pv[8];  // the point record: V*^-1 (v00 v01 v02 v11 v12 v22), 0, 0
      ld_nc_v8(prec + 8 * (size_t)p, pv);
      const float V[3][3] = {{pv[0], pv[1], pv[2]}, {pv[1], pv[3], pv[4]}, {pv[2], pv[4], pv[5]}};
      const float a1[3] = {r1.a0, r1.a1, r1.a2}, a2[3] = {r2.a0, r2.a1, r2.a2};
      // M = R_i V R_j^T
      float T0[3][3], M[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) T0[r][t] = ci[3 * r] * V[0][t] + ci[3 * r + 1] * V[1][t] + ci[3 * r + 2] * V[2][t];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) M[r][t] = T0[r][0] * cj[3 * t] + T0[r][1] * cj[3 * t + 1] + T0[r][2] * cj[3 * t + 2];
      // L = G M G2, h = G M u2, h2 = G2 M^T u, c = u . M u2
      const float u1[3] = {r1.u0, r1.u1, r1.u2}, u2[3] = {r2.u0, r2.u1, r2.u2};
      float Mu2[3], Mtu1[3], h1[3], h2[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        Mu2[r] = M[r][0] * u2[0] + M[r][1] * u2[1] + M[r][2] * u2[2];
        Mtu1[r] = M[0][r] * u1[0] + M[1][r] * u1[1] + M[2][r] * u1[2];
      }
      rec_gvec(r1, Mu2, h1);
      rec_gvec(r2, Mtu1, h2);
      const float c = u1[0] * Mu2[0] + u1[1] * Mu2[1] + u1[2] * Mu2[2];
      const float g1[3] = {r1.gi0, r1.gi1, r1.gi2}, g2[3] = {r2.gi0, r2.gi1, r2.gi2};
      // intrinsic rows first (shared memory): g (a2 x h2)^T, g (T2^T h2)^T, c g g2^T
      {
        float ah2[3], th2[3];
        ah2[0] = a2[1] * h2[2] - a2[2] * h2[1], ah2[1] = a2[2] * h2[0] - a2[0] * h2[2], ah2[2] = a2[0] * h2[1] - a2[1] * h2[0];
#pragma unroll
        for (int r = 0; r < 3; ++r) th2[r] = kCentre ? -(cj[r] * h2[0] + cj[3 + r] * h2[1] + cj[6 + r] * h2[2]) : h2[r];
#pragma unroll
        for (int t = 0; t < 3; ++t)
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            sacc[32 * (9 * t + r)] += g1[t] * ah2[r];
            sacc[32 * (9 * t + 3 + r)] += g1[t] * th2[r];
            sacc[32 * (9 * t + 6 + r)] += c * g1[t] * g2[r];
          }
      }
      rec_gmul(r1, M, T0);  // T0 = G M
      float L[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        L[r][0] = T0[r][0] * r2.g00 + T0[r][1] * r2.g01 + T0[r][2] * r2.g02;
        L[r][1] = T0[r][0] * r2.g01 + T0[r][1] * r2.g11 + T0[r][2] * r2.g12;
        L[r][2] = T0[r][0] * r2.g02 + T0[r][1] * r2.g12 + T0[r][2] * r2.g22;
      }
      // rotation rows: [a1]x L (T0 reused), then times N2 and T2
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        T0[0][t] = a1[1] * L[2][t] - a1[2] * L[1][t];
        T0[1][t] = a1[2] * L[0][t] - a1[0] * L[2][t];
        T0[2][t] = a1[0] * L[1][t] - a1[1] * L[0][t];
      }
      acc_times_n(acc, 0, T0, a2);
      acc_times_t<kCentre>(acc, 0, T0, cj);
      // translation rows: T1^T L (L itself, or -R_i^T L), then times N2 and T2
      if (kCentre) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int t = 0; t < 3; ++t) T0[r][t] = -(ci[r] * L[0][t] + ci[3 + r] * L[1][t] + ci[6 + r] * L[2][t]);
      } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int t = 0; t < 3; ++t) T0[r][t] = L[r][t];
      }
      acc_times_n(acc, 3, T0, a2);
      acc_times_t<kCentre>(acc, 3, T0, cj);
      // the intrinsic columns of rows 0-5: ([a1]x h) g2^T, (T1^T h) g2^T
      float ah1[3], th1[3];
      ah1[0] = a1[1] * h1[2] - a1[2] * h1[1], ah1[1] = a1[2] * h1[0] - a1[0] * h1[2], ah1[2] = a1[0] * h1[1] - a1[1] * h1[0];
#pragma unroll
      for (int r = 0; r < 3; ++r) th1[r] = kCentre ? -(ci[r] * h1[0] + ci[3 + r] * h1[1] + ci[6 + r] * h1[2]) : h1[r];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          acc[9 * r + 6 + t] += ah1[r] * g2[t];
          acc[9 * (3 + r) + 6 + t] += th1[r] * g2[t];
        }
    }
    // warp reduce-scatter of the 81 sums (padded to 96), then the Jacobi scaling
    float v[96];
#pragma unroll
    for (int t = 0; t < 96; ++t) v[t] = t < 54 ? acc[t] : t < 81 ? sacc[32 * (t - 54)] : 0.f;
    rs_round<float, 96>(v, lane, 0);
    rs_round<float, 48>(v, lane, 1);
    rs_round<float, 24>(v, lane, 2);
    rs_round<float, 12>(v, lane, 3);
    rs_round<float, 6>(v, lane, 4);
    const int base = 48 * (lane & 1) + 24 * ((lane >> 1) & 1) + 12 * ((lane >> 2) & 1) + 6 * ((lane >> 3) & 1) +
                     3 * ((lane >> 4) & 1);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int t = base + j;
      if (t < 81) {
        const int r = t / 9, s2 = t - 9 * r;
        const float val = -(v[j] * dinv[9 * a + r]) * dinv[9 * b + s2];
        if constexpr (kSparse) {
          Shat[(size_t)kBlkStride * (2 * (size_t)ri) + 9 * r + s2] = val;
          Shat[(size_t)kBlkStride * (2 * (size_t)ri + 1) + 9 * s2 + r] = val;
        } else {
          Shat[(size_t)(9 * a + r) * ld + 9 * b + s2] = val;
        }
      }
    }
  }
}

__global__ void k_pair_pt(size_t npairs, const int2* __restrict__ pairs, const int* __restrict__ po_pt,
                          int* __restrict__ pair_pt) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q < npairs) pair_pt[q] = po_pt[pairs[q].x];
}

cudaError_t launch_pair_pt(size_t npairs, const int2* pairs, const int* po_pt, int* pair_pt, cudaStream_t s) {
  if (npairs) k_pair_pt<<<(unsigned)((npairs + 255) / 256), 256, 0, s>>>(npairs, pairs, po_pt, pair_pt);
  return cudaGetLastError();
}

// The same blocks with one lane per run, for scenes with very many short runs
// (every camera pair sharing a few dozen points): each lane accumulates its run
// in registers and writes the 81 entries itself, so no cross-lane reduction is
// needed; lanes of a warp take consecutive runs of similar length.
template <typename T, bool kSparse>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1)
    k_form_S_lanes(int n_runs, const int4* __restrict__ runs, const int2* __restrict__ pairs,
                   const T* __restrict__ Y, const int* __restrict__ crank, int Cf, T* __restrict__ Shat, int C,
                   int N) {
  const int ld = spcg_row_stride<T>(9 * Cf);
  for (int ri = blockIdx.x * blockDim.x + threadIdx.x; ri < n_runs; ri += gridDim.x * blockDim.x) {
    const int4 rn = runs[ri];
    const int a = crank[bidx(rn.x, C, 14)], b = crank[bidx(rn.y, C, 14)];
    if (a < 0 || b < 0) continue;
    T acc[81];
#pragma unroll
    for (int q = 0; q < 81; ++q) acc[q] = T(0);
    const int qe = rn.z + rn.w;
    int2 nxt = pairs[rn.z];
    for (int q = rn.z; q < qe; ++q) {
      const int2 pr = nxt;
      if (q + 1 < qe) nxt = pairs[q + 1];
      T y2[27];
      load_row27<T>(Y + kWStride * (size_t)bidx(pr.y, N, 15), y2);
      const T* y1 = Y + kWStride * (size_t)bidx(pr.x, N, 15);
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const T a0 = y1[3 * r], a1 = y1[3 * r + 1], a2 = y1[3 * r + 2];
#pragma unroll
        for (int s2 = 0; s2 < 9; ++s2)
          acc[9 * r + s2] += a0 * y2[3 * s2] + a1 * y2[3 * s2 + 1] + a2 * y2[3 * s2 + 2];
      }
    }
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int s2 = 0; s2 < 9; ++s2) {
        if constexpr (kSparse) {
          Shat[(size_t)kBlkStride * (2 * (size_t)ri) + 9 * r + s2] = -acc[9 * r + s2];
          Shat[(size_t)kBlkStride * (2 * (size_t)ri + 1) + 9 * s2 + r] = -acc[9 * r + s2];
        } else {
          Shat[(size_t)(9 * a + r) * ld + 9 * b + s2] = -acc[9 * r + s2];
        }
      }
  }
}

// ---------------------------------------------------------------------------
// Camera-owned formation (FP32).  The kernels above read both Y^ rows of every
// pair from L2 or device memory.  Here run (i, j) is summed by one owner camera
// (run_owner_first: i when i + j is even, else j; about half of each camera's
// runs), and a block takes up to 128 runs of one owner, one lane per run: the
// block stages the owner's Y^ rows (camera order, ascending in point) in shared
// memory kCfRows at a time, and each lane adds, for its run's pairs within the
// staged rows, the owner row from shared memory times the other camera's row
// from device memory.  The owner's rows cross into the SM once per block
// instead of once per pair.  Each lane sums its run in pair order (fixed), so
// the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kCfThreads = 128;
constexpr int kCfRows = 384;  // staged rows per chunk: 384 x 112 B = 42 KB

__global__ void k_po_co(int N, const int* __restrict__ co_po, int* __restrict__ po_co) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) po_co[co_po[j]] = j;
}

// pairs of run r, in place: point-order (k in i, k2 in j) -> camera-order
// (owner's row, other's row)
__global__ void k_owner_pairs(int n_runs, const int4* __restrict__ runs, const int* __restrict__ po_co,
                              int2* __restrict__ pairs) {
  const int r = blockIdx.x;
  if (r >= n_runs) return;
  const int4 rn = runs[r];
  const bool first = run_owner_first(rn.x, rn.y);
  for (int q = rn.z + threadIdx.x; q < rn.z + rn.w; q += blockDim.x) {
    const int2 pr = pairs[q];
    const int a = po_co[pr.x], b = po_co[pr.y];
    pairs[q] = first ? make_int2(a, b) : make_int2(b, a);
  }
}

cudaError_t launch_owner_pairs(int N, const int* co_po, int* po_co, int n_runs, const int4* runs, int2* pairs,
                               cudaStream_t s) {
  if (N > 0) k_po_co<<<(N + 255) / 256, 256, 0, s>>>(N, co_po, po_co);
  if (n_runs > 0) k_owner_pairs<<<n_runs, 128, 0, s>>>(n_runs, runs, po_co, pairs);
  return cudaGetLastError();
}

// the run's block S_ij (i < j) from acc = sum Y_owner Y_other^T (S_ij itself when
// the owner is i, its transpose when the owner is j), negated, into the dense
// system or the block storage
template <bool kSparse>
__device__ __forceinline__ void store_run_block(const float (&acc)[81], bool owner_first, int ri, int a, int b,
                                                int ld, float* __restrict__ Shat) {
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const float v = -(owner_first ? acc[9 * r + c] : acc[9 * c + r]);  // S_ij[r][c]
      if constexpr (kSparse) {
        Shat[(size_t)kBlkStride * (2 * (size_t)ri) + 9 * r + c] = v;
        Shat[(size_t)kBlkStride * (2 * (size_t)ri + 1) + 9 * c + r] = v;
      } else {
        Shat[(size_t)(9 * a + r) * ld + 9 * b + c] = v;
      }
    }
}

template <bool kSparse>
__global__ void __launch_bounds__(kCfThreads, 4)
    k_form_S_cam(const int4* __restrict__ blocks, const int* __restrict__ own_run, const int4* __restrict__ runs,
                 const int2* __restrict__ pairs, const int* __restrict__ cam_off, const float* __restrict__ Y,
                 const int* __restrict__ crank, int Cf, float* __restrict__ Shat, int n_runs, int C, int N) {
  __shared__ __align__(16) uint4 stage[kCfRows * 7];
  const int4 bd = blocks[blockIdx.x];  // (owner camera, first own_run index, runs, unused)
  const int cam = bidx(bd.x, C, 30);
  const int t = threadIdx.x;
  const int lo = cam_off[cam], hi = cam_off[cam + 1];  // the owner camera's rows
  int ri = -1, a = -1, b = -1, cur = 0, end = 0;
  bool first = true;
  if (t < bd.z) {
    ri = bidx(own_run[bd.y + t], n_runs, 31);
    const int4 rn = runs[ri];
    a = crank[bidx(rn.x, C, 32)];
    b = crank[bidx(rn.y, C, 32)];
    first = run_owner_first(rn.x, rn.y);
    cur = rn.z;
    end = rn.z + rn.w;
  }
  const bool live = t < bd.z && a >= 0 && b >= 0;
  int2 pr = live && cur < end ? pairs[cur] : make_int2(0x7fffffff, 0);  // the lane's next pair
  float acc[81];
#pragma unroll
  for (int q = 0; q < 81; ++q) acc[q] = 0.f;
  const uint4* Y4 = reinterpret_cast<const uint4*>(Y);
  for (int s0 = lo; s0 < hi; s0 += kCfRows) {
    const int n = min(kCfRows, hi - s0);
    __syncthreads();  // the previous chunk's rows are no longer read
    for (int i = t; i < n * 7; i += kCfThreads) stage[i] = Y4[(size_t)7 * s0 + i];
    __syncthreads();
    if (!live) continue;
    const int s1 = s0 + n;
    while (cur < end && pr.x < s1) {
      const int2 nx = cur + 1 < end ? pairs[cur + 1] : make_int2(0x7fffffff, 0);  // in flight meanwhile
      float y2[27];
      load_row27<float>(Y + kWStride * (size_t)bidx(pr.y, N, 33), y2);
      const float* y1 = reinterpret_cast<const float*>(stage + 7 * bidx(pr.x - s0, n, 34));
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const float a0 = y1[3 * r], a1 = y1[3 * r + 1], a2 = y1[3 * r + 2];
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[9 * r + c] += a0 * y2[3 * c] + a1 * y2[3 * c + 1] + a2 * y2[3 * c + 2];
      }
      pr = nx;
      ++cur;
    }
  }
  if (live) store_run_block<kSparse>(acc, first, ri, a, b, spcg_row_stride<float>(9 * Cf), Shat);
}

// Diagonal blocks of the block-sparse system, scaled: slot 2 n_runs + c for the
// camera c of rank f, from the packed block-Jacobi block D_f.
template <typename T>
__global__ void k_S_diag_blocks(int Cf, const int* __restrict__ cam_map, const T* __restrict__ Dblk,
                                const double* __restrict__ dscale, int n_runs, T* __restrict__ Bs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 81 * Cf) return;
  const int f = e / 81, t = e - 81 * f, r = t / 9, c = t - 9 * r;
  const T* di = reinterpret_cast<const T*>(dscale + 9 * (size_t)Cf);
  Bs[(size_t)kBlkStride * (2 * (size_t)n_runs + cam_map[f]) + t] =
      Dblk[45 * (size_t)f + sym9(r, c)] * di[9 * f + r] * di[9 * f + c];
}

// Diagonal blocks from the block-Jacobi blocks D_a = U*_a - sum W V*^-1 W^T (packed),
// scaled; and the lower triangle mirrored from the upper one.
template <typename T>
__global__ void k_S_finalize(int Cf, const T* __restrict__ Dblk, const double* __restrict__ dscale,
                             T* __restrict__ Shat) {
  __shared__ T tile[32][33];
  const int n = 9 * Cf, ld = spcg_row_stride<T>(n);
  const int bx = blockIdx.x, by = blockIdx.y;  // tile column, tile row
  // tiles on or below the diagonal, and the first tile above it (a 9 x 9 camera
  // block can straddle two 32-tiles: its upper entries there are written too)
  if (bx > by + 1) return;
  const bool mirror = bx <= by;
  if (mirror) {
    // read the transposed tile (upper triangle source)
    int r0 = bx * 32, c0 = by * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      int r = r0 + i, c = c0 + threadIdx.x;
      tile[i][threadIdx.x] = (r < n && c < n) ? Shat[(size_t)r * ld + c] : T(0);
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int r = by * 32 + i, c = bx * 32 + threadIdx.x;
    if (r >= n || c >= n) continue;
    int fr = r / 9, fc = c / 9;
    if (fr == fc) {
      int ir = r - 9 * fr, ic = c - 9 * fc;
      const T* di = reinterpret_cast<const T*>(dscale + n);
      Shat[(size_t)r * ld + c] = Dblk[45 * (size_t)fr + sym9(ir, ic)] * di[r] * di[c];
    } else if (mirror && c < r) {
      Shat[(size_t)r * ld + c] = tile[threadIdx.x][i];
    }
  }
}

// Jacobi scaling of the explicit system from the damped U blocks alone:
// D = sqrt(diag U*) in FP64 and 1/D in the working precision (dscale + 9 Cf), with
// U*_ii = U_ii + lambda clamp(U_ii) rounded to T exactly as the Schur-diagonal
// kernel stores it
template <typename T>
__global__ void k_dscale(int Cf, const int* __restrict__ cam_map, const T* __restrict__ Ug, double lambda,
                         double* __restrict__ dscale, int kfix) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 9 * Cf) return;
  const int f = e / 9, i = e - 9 * f;
  // kfix: slots 7 and 8 held by a unit diagonal (as in the Schur-diagonal kernel)
  double u = kfix && i >= 7 ? 1.0 : (double)Ug[54 * (size_t)cam_map[f] + sym9(i, i)];
  u += lambda * fmin(fmax(u, 1e-6), 1e32);
  const double d = (double)(T)u;
  const double sd = sqrt(d > 0.0 ? d : 1e-30);
  dscale[e] = sd;
  reinterpret_cast<T*>(dscale + 9 * (size_t)Cf)[e] = (T)(1.0 / sd);
}

template <typename T>
cudaError_t launch_dscale(int Cf, const int* cam_map, const T* Ug, double lambda, double* dscale, cudaStream_t s,
                          int kfix) {
  if (Cf > 0) k_dscale<T><<<(9 * Cf + 255) / 256, 256, 0, s>>>(Cf, cam_map, Ug, lambda, dscale, kfix);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_form_S(const Layout& L, int n_runs, const int4* runs, const int2* pairs, const T* W,
                          const T* Vinv, const int* crank, const T* Ud, const T* Dblk, double* dscale,
                          int Cf, T* Y, T* Shat, bool lanes, int num_sms, cudaEvent_t ev0, cudaEvent_t ev1,
                          cudaEvent_t join, cudaStream_t s, const int* cam_map, bool sparse, const CamForm* cf,
                          const FormRec* fr) {
  if (sizeof(T) != 4) cf = nullptr, fr = nullptr;  // FP64 keeps point-order rows and the pair kernels
  if (cf || lanes) fr = nullptr;  // records serve the warp-per-run kernel
  if (Cf <= 0) return cudaSuccess;
  const int n = 9 * Cf;
  // dscale (D and 1/D) was written by the Schur-diagonal kernel
  if (L.N > 0 && !fr)
    k_form_Y<T><<<(L.N + kYRows - 1) / kYRows, kYRows, 0, s>>>(L.N, L.C, L.P, L.po_cam, L.po_pt, W, Vinv, crank,
                                                               dscale, Cf, Y, cf ? cf->po_co : nullptr);
  cudaError_t e = cudaSuccess;
  // the dense system is cleared (blocks of pairs that share no point stay zero);
  // the block-sparse one stores only written blocks (the matvec skips blocks
  // whose cameras are not both free)
  if (!sparse && (e = cudaMemsetAsync(Shat, 0, sizeof(T) * (size_t)n * spcg_row_stride<T>(n), s)) != cudaSuccess)
    return e;
  // events (nullable) around the co-visibility product kernel
  if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
  if (n_runs > 0 && cf) {
    if constexpr (sizeof(T) == 4) {
      if (sparse)
        k_form_S_cam<true><<<cf->n_blocks, kCfThreads, 0, s>>>(cf->blocks, cf->own_run, runs, pairs, cf->cam_off, Y,
                                                               crank, Cf, Shat, n_runs, L.C, L.N);
      else
        k_form_S_cam<false><<<cf->n_blocks, kCfThreads, 0, s>>>(cf->blocks, cf->own_run, runs, pairs, cf->cam_off, Y,
                                                                crank, Cf, Shat, n_runs, L.C, L.N);
    }
  } else if (n_runs > 0) {
    const int wpb = 4;  // warps per 128-thread block
    if (lanes) {
      // many short runs: one lane per run
      int grid = (n_runs + 127) / 128;
      if (grid > 16 * num_sms) grid = 16 * num_sms;  // (a resident-only grid measured slower here)
      if (sparse) k_form_S_lanes<T, true><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat, L.C, L.N);
      else k_form_S_lanes<T, false><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat, L.C, L.N);
    } else {
      // resident blocks only (three per SM in FP32), striding over the runs: no
      // partly filled last wave
      int grid = (n_runs + wpb - 1) / wpb;
      const int resident = (sizeof(T) == 4 ? 3 : 1) * num_sms;
      if (grid > resident) grid = resident;
      if constexpr (sizeof(T) == 4) {
        if (fr) {
          // one block per four runs (no resident-only grid): blocks retire as they
          // finish, so the side stream's Schur-diagonal chain, which the diagonal
          // blocks wait for, is scheduled alongside instead of after the formation
          grid = (n_runs + wpb - 1) / wpb;
          const float* Cw = reinterpret_cast<const float*>(fr->camw);
          auto* kern = sparse ? (fr->centre ? k_form_S_rec<true, true> : k_form_S_rec<true, false>)
                              : (fr->centre ? k_form_S_rec<false, true> : k_form_S_rec<false, false>);
          kern<<<grid, 128, 0, s>>>(n_runs, runs, pairs, fr->pair_pt, fr->rec, fr->prec, Cw, dscale, crank, Cf,
                                    (float*)Shat, L.C, L.N, L.P);
        }
      }
      if (!fr) {
        if (sparse) k_form_S_runs<T, true><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat, L.C, L.N);
        else k_form_S_runs<T, false><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat, L.C, L.N);
      }
    }
  }
  if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return e;
  // the diagonal blocks come from the Schur-diagonal kernel (on another stream when `join`)
  if (join && (e = cudaStreamWaitEvent(s, join, 0)) != cudaSuccess) return e;
  if (sparse) {
    k_S_diag_blocks<T><<<(81 * Cf + 255) / 256, 256, 0, s>>>(Cf, cam_map, Dblk, dscale, n_runs, Shat);
    return cudaGetLastError();
  }
  int nt = (n + 31) / 32;
  k_S_finalize<T><<<dim3(nt, nt), dim3(32, 8), 0, s>>>(Cf, Dblk, dscale, Shat);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// PCG on the scaled explicit system S^ x^ = b^ (b^ = D^-1 b, x = D^-1 x^) with the
// block-Jacobi preconditioner of S^ (Sec. 4.2 step 3).
//
// The vectors are short (n = 9 Cf <= 4608), so every block keeps all of them
// (p, r, z, q, x) and updates them redundantly; the only distributed work is
// the matvec.  Block b owns rows [n b / G, n (b+1) / G) of S^ (in shared memory
// when they fit), computes those entries of q = S^ p and publishes them; every
// block then gathers the whole q.  With q, p and r identical in every block,
// each block forms p^T q, alpha, r^T r, r^T z and beta itself, in the same
// order, hence to the same bits: one exchange per iteration and no grid-wide
// reduction or barrier.
//
// Exchange words: each 32-bit chunk of a published value travels in a 64-bit
// word whose high half is the iteration's tag; a 64-bit store and load are
// single-copy atomic, so a word carrying the expected tag is the published
// value, with no fence.  Tags are distinct across iterations and launches
// (tag_base advances by max_iters + 2 per launch).  Iteration i writes word set
// i & 1: a block publishes iteration i + 2 only after gathering all of
// iteration i + 1, which every block published only after gathering all of
// iteration i, so no word is overwritten before every block has read it.
// ---------------------------------------------------------------------------

constexpr int kSpcgThreads = 512;
// copies of every exchange word: block b polls copy b % kSpcgReplicas, which
// spreads the polling of all blocks over several L2 lines per word (8 copies
// measured 13% faster than one on the 1,791-unknown system)
constexpr int kSpcgReplicas = 8;

// asynchronous global -> shared copy of one 4- or 8-byte element (cp.async)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <typename T>
constexpr int spcg_words() {
  return sizeof(T) / 4;  // 32-bit chunks per value
}

template <typename T>
__device__ __forceinline__ void spcg_publish(unsigned long long* w, T v, unsigned tag) {
  const unsigned long long hi = (unsigned long long)tag << 32;
  if constexpr (sizeof(T) == 4) {
    st_relaxed_u64(w, hi | __float_as_uint(v));
  } else {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    st_relaxed_u64(w, hi | (bits & 0xFFFFFFFFull));
    st_relaxed_u64(w + 1, hi | (bits >> 32));
  }
}

template <typename T>
__device__ __forceinline__ T spcg_unpack(const unsigned long long* v) {
  if constexpr (sizeof(T) == 4) return __uint_as_float((unsigned)v[0]);
  else return __longlong_as_double((long long)((v[0] & 0xFFFFFFFFull) | (v[1] << 32)));
}


// Preconditioner block of one camera, symmetric 9x9 stored in full: rows 0-4 at
// 9 i, rows 5-8 from entry 48 on (each half starts on a 16-byte boundary), 84
// entries per camera
constexpr int kMStride = kSpcgMStride;
__host__ __device__ constexpr int mrow(int i) { return 9 * i + (i >= 5 ? 3 : 0); }

constexpr int kSpcgRedStride = 64;  // warp sums of one block reduction (K x 16, K <= 4)
// two alternating block-sum buffers, then the matvec's per-warp row partials (16 x 16 FP32)
constexpr size_t kSpcgSumBytes = sizeof(double) * 2 * kSpcgRedStride;
constexpr size_t kSpcgRedBytes = kSpcgSumBytes + sizeof(float) * 16 * 16;

// One step of a transposing butterfly: CNT values per lane become CNT / 2, each
// the sum of this lane's and lane ^ M's values for the half of the rows this
// lane keeps (the lower half when bit M of the lane is clear).
template <int M, int CNT>
__device__ __forceinline__ void tstep(float (&v)[16], int lane) {
  const bool up = lane & M;
#pragma unroll
  for (int i = 0; i < CNT / 2; ++i) {
    const float snd = up ? v[i] : v[i + CNT / 2];
    const float kp = up ? v[i + CNT / 2] : v[i];
    v[i] = kp + __shfl_xor_sync(0xffffffffu, snd, M);
  }
}

// per-block vector storage other than p: r, z, q, x (full length) and the
// preconditioner blocks (kMStride each), in T elements
template <typename T>
__host__ __device__ size_t spcg_vec_elems(int n, int Cf) {
  return (size_t)4 * spcg_row_stride<T>(n) + (size_t)kMStride * Cf;
}

template <typename T>
size_t spcg_smem_bytes(int n, int rows, int rows_in_smem, int vecs_in_smem, int Cf) {
  const int ns = spcg_row_stride<T>(n);
  size_t b = kSpcgRedBytes;
  b += rows_in_smem ? sizeof(T) * (size_t)rows * ns : 0;  // owned rows of S^
  b += sizeof(T) * (size_t)ns;                             // p (full length)
  b += vecs_in_smem ? sizeof(T) * spcg_vec_elems<T>(n, Cf) : 0;
  return (b + 15) & ~size_t(15);
}

// PCG dot products and their scalars.  FP64 problems sum in FP64.  FP32 problems
// keep FP64-level accuracy on the FP32 pipe (B300 issues FP64 at 1/64 of the FP32
// rate, so 512 threads spending one FP64 instruction each would cost ~0.1 us):
// every product a b enters as its exact TwoProduct pair, every addition is a
// TwoSum whose exact error joins a low-order word, and alpha = (r, z) / (p, q),
// beta = (r, z)' / (r, z) are double-float quotients rounded once to FP32.
// The accumulated dot agrees with the exact dot of the FP32 vectors to ~2^-44
// relative (the low word's own rounding); the sums are of products of FP32
// vectors, so this is what FP64 dots of the same vectors deliver.
template <typename T>
struct DotT;
template <>
struct DotT<double> {
  using type = double;
};
template <>
struct DotT<float> {
  using type = F2;  // unevaluated hi + lo, lo not renormalised until read
};
template <typename T>
using Dot = typename DotT<T>::type;

__device__ __forceinline__ void dot_zero(double& d) { d = 0.0; }
__device__ __forceinline__ void dot_zero(F2& d) { d = F2{0.f, 0.f}; }
__device__ __forceinline__ void dot_fma(double& d, double a, double b) { d = fma(a, b, d); }
__device__ __forceinline__ void dot_fma(F2& d, float a, float b) {
  const float pr = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -pr);  // a b = pr + pe exactly
  const F2 t = two_sum(d.h, pr);
  d.h = t.h;
  d.l = __fadd_rn(d.l, __fadd_rn(t.l, pe));
}
// a + b with the same bits whichever operand comes first (TwoSum's error is exact)
__device__ __forceinline__ double dot_add(double a, double b) { return a + b; }
__device__ __forceinline__ F2 dot_add(F2 a, F2 b) {
  const F2 t = two_sum(a.h, b.h);
  return F2{t.h, __fadd_rn(__fadd_rn(a.l, b.l), t.l)};
}
__device__ __forceinline__ double dot_shfl(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ F2 dot_shfl(F2 v, int m) {
  return F2{__shfl_xor_sync(0xffffffffu, v.h, m), __shfl_xor_sync(0xffffffffu, v.l, m)};
}
__device__ __forceinline__ double dot_norm(double v) { return v; }
__device__ __forceinline__ F2 dot_norm(F2 v) { return fast_two_sum(v.h, v.l); }
__device__ __forceinline__ double dot_value(double v) { return v; }
__device__ __forceinline__ double dot_value(F2 v) { return f2_to_double(v); }
// a / b in the working precision
__device__ __forceinline__ double dot_div(double a, double b) { return a / b; }
__device__ __forceinline__ float dot_div(F2 a, F2 b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const F2 r = f2_sub(a, f2_mul(F2{q1, 0.f}, b));  // a - q1 b, small
  return __fadd_rn(q1, __fdiv_rn(r.h, b.h));
}
__device__ __forceinline__ bool dot_le(double a, double b) { return a <= b; }
__device__ __forceinline__ bool dot_le(F2 a, F2 b) { return a.h < b.h || (a.h == b.h && a.l <= b.l); }
__device__ __forceinline__ bool dot_nonzero(double a) { return a != 0.0; }
__device__ __forceinline__ bool dot_nonzero(F2 a) { return a.h != 0.f; }  // normalised: lo = 0 when hi = 0
__device__ __forceinline__ bool dot_pos_finite(double a) { return a > 0.0 && isfinite(a); }
__device__ __forceinline__ bool dot_pos_finite(F2 a) { return a.h > 0.f && f2_finite(a); }

// Block-wide sums of K dots: a butterfly within each warp, then in every warp
// lanes l and l + 16 take warp sum l and a second butterfly over 16 lanes adds
// them, so every thread holds the same bits (dot_add is commutative bit for bit;
// for FP32 problems, the normalised double-float).  The tree is the pairwise
// one (w_i + w_i+8, then + 4, + 2, + 1).  One barrier: callers alternate
// between two `red` buffers (kSpcgRedStride doubles each).  Returns the OR of
// `flag` over the block.
template <int K, typename D>
__device__ __forceinline__ int block_allsum_dot(D (&v)[K], void* red_raw, int flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kSpcgThreads / 32;
  static_assert(NW == 16, "the fixed summation tree is written for 16 warps");
  static_assert(K * NW * sizeof(D) <= kSpcgRedStride * sizeof(double), "reduction buffer");
  D* red = reinterpret_cast<D*>(red_raw);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    D s = v[k];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s = dot_add(s, dot_shfl(s, m));
    if (lane == 0) red[NW * k + warp] = s;
  }
  const int any = __syncthreads_or(flag);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    D s = red[NW * k + (lane & (NW - 1))];
#pragma unroll
    for (int m = NW / 2; m > 0; m >>= 1) s = dot_add(s, dot_shfl(s, m));
    v[k] = dot_norm(s);
  }
  return any;
}

// z_c = M^_c r_c for one camera
template <typename T>
__device__ __forceinline__ void spcg_precond(const T* __restrict__ M, const T* __restrict__ r, T* __restrict__ z) {
  T rv[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) rv[j] = r[j];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) acc += M[mrow(i) + j] * rv[j];
    z[i] = acc;
  }
}

// Preconditioner blocks of S^: M^_f = diag(d) M_f diag(d), symmetrised, in T
// (the same expression for (i, j) and (j, i), so M^_f is symmetric bit for bit),
// cameras f = t0, t0 + stride, ...
template <typename T>
__device__ __forceinline__ void spcg_build_precond(int Cf, const T* __restrict__ Dinv, const double* __restrict__ dscale,
                                                   T* __restrict__ M, int t0, int stride) {
  for (int f = t0; f < Cf; f += stride) {
    const T* Df = Dinv + 81 * (size_t)f;
    T d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = (T)dscale[9 * f + i];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int j = 0; j < 9; ++j) M[kMStride * f + mrow(i) + j] = (T(0.5) * (Df[9 * i + j] + Df[9 * j + i])) * (d[i] * d[j]);
  }
}

template <typename T>
__global__ void k_spcg_precond(int Cf, const T* __restrict__ Dinv, const double* __restrict__ dscale,
                               T* __restrict__ M) {
  spcg_build_precond<T>(Cf, Dinv, dscale, M, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
cudaError_t launch_spcg_precond(int Cf, const T* Dinv, const double* dscale, T* M, cudaStream_t s) {
  if (Cf > 0) k_spcg_precond<T><<<(Cf + 127) / 128, 128, 0, s>>>(Cf, Dinv, dscale, M);
  return cudaGetLastError();
}

// Persistent PCG: standard preconditioned CG (x0 = 0, block-Jacobi M^).  Thread
// t handles the vector entries of cameras t, t + 512, ...
// kRows: the block's rows of S^ sit in shared memory (else streamed from device
// memory by every matvec); one instance per placement keeps registers in check
template <typename T, bool kRows>
__global__ void __launch_bounds__(kSpcgThreads, 1) k_spcg(SpcgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int W = spcg_words<T>();
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int n = a.n, ns = spcg_row_stride<T>(n), Cf = a.Cf;
  const int r0 = (int)(((long long)n * bid) / G), r1 = (int)(((long long)n * (bid + 1)) / G);
  const int nr = r1 - r0;
  unsigned char* sp = smem_raw;
  T* red = reinterpret_cast<T*>(sp);
  int rb = 0;  // which of the two reduction buffers the next block sum uses
  sp += kSpcgRedBytes;
  T* Srows = reinterpret_cast<T*>(sp);
  sp += kRows ? sizeof(T) * (size_t)nr * ns : 0;
  T* pv = reinterpret_cast<T*>(sp);
  // r, z, q, x and M^ follow p in shared memory, or sit in this block's slice of
  // the global scratch when they do not fit
  T* rv = a.vecs_in_smem ? pv + ns : a.scratch + (size_t)bid * a.scratch_stride;
  T* zv = rv + ns;
  T* qv = zv + ns;
  T* xv = qv + ns;
  // preconditioner blocks: this block's copy, or one copy shared by all blocks
  // (built before the launch) when the vectors live in device scratch
  T* Mv = a.Mshared ? nullptr : xv + ns;
  const T* Mr = a.Mshared ? a.Mshared : Mv;
  const T* Sg = a.Shat + (size_t)r0 * ns;
  const T* dinv = reinterpret_cast<const T*>(a.dscale + n);

  if constexpr (kRows) {
    // the block's rows of S^ (from HBM once per solve): asynchronous element
    // copies, all in flight together, overlapping the set-up below
    for (int r = warp; r < nr; r += nwarps) {
      const T* src = Sg + (size_t)r * ns;
      T* dst = Srows + (size_t)r * ns;
      for (int c = lane; c < ns; c += 32) cp_async_elem(dst + c, src + c);  // padding entries are zero
    }
    cp_async_commit();
  }
  for (int c = n + tid; c < ns; c += blockDim.x) pv[c] = zv[c] = xv[c] = T(0);
  if (Mv) spcg_build_precond<T>(Cf, a.Dinv, a.dscale, Mv, tid, blockDim.x);
  __syncthreads();
  // r = b^, z = M^ r, p = z, x = 0; (r, z) and (r, r)
  using D = Dot<T>;
  D d0[2];
  dot_zero(d0[0]);
  dot_zero(d0[1]);
  for (int f = tid; f < Cf; f += blockDim.x) {
    const int e = 9 * f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      rv[e + i] = a.b[e + i] * dinv[e + i];  // the correctly rounded product in T
      xv[e + i] = T(0);
    }
    spcg_precond(Mr + kMStride * f, rv + e, zv + e);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      pv[e + i] = zv[e + i];
      dot_fma(d0[0], rv[e + i], zv[e + i]);
      dot_fma(d0[1], rv[e + i], rv[e + i]);
    }
  }
  if constexpr (kRows) cp_async_wait_all();  // visible to the block after the barrier below
  block_allsum_dot<2>(d0, red + kSpcgRedStride * rb, 0);
  rb ^= 1;
  // the iteration's dots carried as D, the step lengths in the working precision
  D rz = d0[0];
  const double bnorm = sqrt(dot_value(d0[1]));
  D stop_rr;
  {
    const double st = (a.tol * bnorm) * (a.tol * bnorm);
    if constexpr (sizeof(T) == 4) stop_rr = f2_from_double(st);
    else stop_rr = st;
  }
  D rr_last = d0[1];
  int it = 0;
  T alpha = T(0);
  bool x_pending = false;  // x still lacks the last alpha p
  // FP32 with the rows in shared memory: x += a_prev p and p = z + b p are applied
  // by each warp to its own column slice inside the next matvec (no separate pass)
  constexpr bool kFused = sizeof(T) == 4 && kRows;
  T a_prev = T(0), b_next = T(0);  // a_prev = 0, b_next = 0 leave x = 0 and p = z
  unsigned long long* words = a.words;
  while (bnorm > 0.0 && it < a.max_iters) {
    const unsigned tag = a.tag_base + (unsigned)it;
    const size_t set_words = (size_t)n * W;
    unsigned long long* set = words + (size_t)(it & 1) * kSpcgReplicas * set_words;
    // q = S^_rows p for the owned rows, published as tagged words
    if constexpr (sizeof(T) == 4) {
      if constexpr (kRows) {
        // column split: warp w takes a slice of the float4 columns of every owned
        // row, so p is read from shared memory once per block; per chunk of 16
        // rows, a transposing butterfly leaves lane l with row (l >> 1)'s warp
        // partial, and warp r adds row r's 16 warp partials in a fixed order
        const float4* p4 = reinterpret_cast<const float4*>(pv);
        float* part = reinterpret_cast<float*>(smem_raw + kSpcgSumBytes);
        const int nc4 = ns / 4;
        const int c0 = (nc4 * warp) / nwarps, c1 = (nc4 * (warp + 1)) / nwarps;
        // (one pass even without rows: the x and p updates of the slice happen in it)
        for (int rc0 = 0; rc0 == 0 || rc0 < nr; rc0 += 16) {
          const int nrc = max(0, min(16, nr - rc0));
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
          for (int c = c0 + lane; c < c1; c += 32) {
            float4 pp = p4[c];
            if (rc0 == 0) {
              // this warp's columns of x and p (read by no other warp before the barrier below)
              const float4 zz = reinterpret_cast<const float4*>(zv)[c];
              float4 xx = reinterpret_cast<const float4*>(xv)[c];
              xx.x = fmaf(a_prev, pp.x, xx.x), xx.y = fmaf(a_prev, pp.y, xx.y);
              xx.z = fmaf(a_prev, pp.z, xx.z), xx.w = fmaf(a_prev, pp.w, xx.w);
              pp.x = fmaf(b_next, pp.x, zz.x), pp.y = fmaf(b_next, pp.y, zz.y);
              pp.z = fmaf(b_next, pp.z, zz.z), pp.w = fmaf(b_next, pp.w, zz.w);
              reinterpret_cast<float4*>(xv)[c] = xx;
              reinterpret_cast<float4*>(pv)[c] = pp;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              if (i < nrc) {
                const float4 s4 = reinterpret_cast<const float4*>(Srows + (size_t)(rc0 + i) * ns)[c];
                v[i] = fmaf(s4.x, pp.x, fmaf(s4.y, pp.y, fmaf(s4.z, pp.z, fmaf(s4.w, pp.w, v[i]))));
              }
            }
          }
          tstep<16, 16>(v, lane);
          tstep<8, 8>(v, lane);
          tstep<4, 4>(v, lane);
          tstep<2, 2>(v, lane);
          v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
          const int row = (lane >> 1) & 15;
          if (!(lane & 1) && row < nrc) part[16 * row + warp] = v[0];
          __syncthreads();
          if (warp < nrc) {
            float sr = lane < 16 ? part[16 * warp + lane] : 0.f;
#pragma unroll
            for (int m = 8; m > 0; m >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, m);
            if (lane < kSpcgReplicas)
              spcg_publish<T>(set + lane * set_words + (size_t)(r0 + rc0 + warp) * W, sr, tag);
          }
          if (rc0 + 16 < nr) __syncthreads();  // part is rewritten by the next chunk
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (!kRows) {
        // rows streamed from device memory: 16-byte loads, four in flight per lane
        const float4* p4 = reinterpret_cast<const float4*>(pv);
        const int rs = ns / 4;
        for (int r = warp; r < nr; r += nwarps) {
          const float4* row = reinterpret_cast<const float4*>(Sg + (size_t)r * ns);
          float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
          int c = lane;
          for (; c + 224 < rs; c += 256) {
            float4 sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = __ldcs(row + c + 32 * u);  // streamed once per iteration
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float4 q0 = p4[c + 32 * u];
              float& cu = (u & 3) == 0 ? c0 : (u & 3) == 1 ? c1 : (u & 3) == 2 ? c2 : c3;
              cu = fmaf(sv[u].x, q0.x, fmaf(sv[u].y, q0.y, fmaf(sv[u].z, q0.z, fmaf(sv[u].w, q0.w, cu))));
            }
          }
          for (; c < rs; c += 32) {
            const float4 s0 = __ldg(row + c), q0 = p4[c];
            c0 = fmaf(s0.x, q0.x, fmaf(s0.y, q0.y, fmaf(s0.z, q0.z, fmaf(s0.w, q0.w, c0))));
          }
          const float acc = warp_sum((c0 + c1) + (c2 + c3));
          if (lane < kSpcgReplicas) spcg_publish<T>(set + lane * set_words + (size_t)(r0 + r) * W, acc, tag);
        }
      }
    } else {
      const T* base = kRows ? Srows : Sg;
      for (int r = warp; r < nr; r += nwarps) {
        const T* row = base + (size_t)r * ns;
        T acc = T(0);
        for (int c = lane; c < n; c += 32) acc += row[c] * pv[c];
        acc = warp_sum(acc);
        if (lane < kSpcgReplicas) spcg_publish<T>(set + lane * set_words + (size_t)(r0 + r) * W, acc, tag);
      }
    }
    if constexpr (kFused) x_pending = false;  // the matvec pass applied a_prev p
    // gather q from this block's copy, coalesced (thread t: entries t, t + 512, ...,
    // up to four in flight), and (p, q)
    int late = 0;
    D d1[1];
    dot_zero(d1[0]);
    const unsigned long long* mine = set + (size_t)(bid % kSpcgReplicas) * set_words;
    const uint64_t t0 = globaltimer_ns();
    for (int eb = tid; eb < n && !late; eb += 4 * blockDim.x) {
      unsigned long long v[4][W];
      for (;;) {
        bool ready = true;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = eb + u * blockDim.x;
#pragma unroll
          for (int w = 0; w < W; ++w) {
            v[u][w] = e < n ? ld_relaxed_u64(mine + (size_t)e * W + w) : ((unsigned long long)tag << 32);
            ready &= (unsigned)(v[u][w] >> 32) == tag;
          }
        }
        if (ready) break;
        if ((long long)(globaltimer_ns() - t0) > a.timeout_ns) {
          late = 1;
          break;
        }
      }
      if (late) break;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = eb + u * blockDim.x;
        if (e < n) {
          const T q = spcg_unpack<T>(v[u]);
          qv[e] = q;
          dot_fma(d1[0], pv[e], q);
        }
      }
    }
    if (block_allsum_dot<1>(d1, red + kSpcgRedStride * rb, late)) {
      if (tid == 0) atomicOr(a.err, 1);
      break;
    }
    rb ^= 1;
    const D pq = d1[0];
    if (!dot_pos_finite(pq)) {
      if (bid == 0 && tid == 0) atomicOr(a.err, 2);
      break;
    }
    alpha = dot_div(rz, pq);
    // r -= alpha q, z = M^ r; (r, r) and (r, z) (x is updated with p below).  Two
    // threads per camera, adjacent lanes: rows 0-4 and rows 5-8; each takes the
    // other's rows of r by shuffle.  The loop's trip count is the same for every
    // thread, so whole warps meet at the shuffles.
    D d2[2];
    dot_zero(d2[0]);
    dot_zero(d2[1]);
    for (int base = 0; base < 2 * Cf; base += blockDim.x) {
      const int t = base + tid, f = t >> 1, h = t & 1;
      const bool on = t < 2 * Cf;
      const int e = 9 * f, i0 = h ? 5 : 0, nrow = h ? 4 : 5;
      T ro[5];  // this thread's rows of r after the update
#pragma unroll
      for (int ii = 0; ii < 5; ++ii) {
        ro[ii] = T(0);
        if (on && ii < nrow) {
          const int i = e + i0 + ii;
          ro[ii] = fma(-alpha, qv[i], rv[i]);
          rv[i] = ro[ii];
        }
      }
      T rc[9];
#pragma unroll
      for (int ii = 0; ii < 5; ++ii) {
        const T o = __shfl_xor_sync(0xffffffffu, ro[ii], 1);
        if (ii < 4) rc[5 + ii] = h ? ro[ii] : o;
        rc[ii] = h ? o : ro[ii];
      }
      if (on) {
        const T* M = Mr + kMStride * f + (h ? 48 : 0);
        T m[48];
        if constexpr (sizeof(T) == 4) {
          const float4* M4 = reinterpret_cast<const float4*>(M);
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < 9 || !h) v4 = M4[k];
            m[4 * k] = v4.x, m[4 * k + 1] = v4.y, m[4 * k + 2] = v4.z, m[4 * k + 3] = v4.w;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 45; ++k) m[k] = (k < 36 || !h) ? M[k] : T(0);
        }
#pragma unroll
        for (int ii = 0; ii < 5; ++ii) {
          if (ii < nrow) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < 9; ++j) acc += m[9 * ii + j] * rc[j];
            zv[e + i0 + ii] = acc;
            dot_fma(d2[0], ro[ii], ro[ii]);
            dot_fma(d2[1], ro[ii], acc);
          }
        }
      }
    }
    block_allsum_dot<2>(d2, red + kSpcgRedStride * rb, 0);
    rb ^= 1;
    ++it;
    x_pending = true;
    const D rr = d2[0], rz_new = d2[1];
    rr_last = rr;
    if (dot_le(rr, stop_rr)) break;
    const T beta = dot_nonzero(rz) ? (T)dot_div(rz_new, rz) : T(0);
    rz = rz_new;
    if constexpr (kFused) {
      a_prev = alpha;
      b_next = beta;
    } else {
      // x += alpha p, p = z + beta p, entry-parallel over the block
      for (int e = tid; e < n; e += blockDim.x) {
        const T pe = pv[e];
        xv[e] = fma(alpha, pe, xv[e]);
        pv[e] = fma(beta, pe, zv[e]);
      }
      x_pending = false;
      __syncthreads();
    }
  }
  if (x_pending)
    for (int e = tid; e < n; e += blockDim.x) xv[e] = fma(alpha, pv[e], xv[e]);
  __syncthreads();
  for (int e = r0 + tid; e < r1; e += blockDim.x) a.x[e] = xv[e] * dinv[e];
  if (bid == 0 && tid == 0) {
    a.sc->pcg_iters = it;
    a.sc->pcg_bnorm = bnorm;
    a.sc->pcg_rel_res = bnorm > 0.0 ? sqrt(dot_value(rr_last)) / bnorm : 0.0;
  }
}

template <typename T>
const void* spcg_kernel_ptr(bool rows_in_smem) {
  return rows_in_smem ? reinterpret_cast<const void*>(&k_spcg<T, true>)
                      : reinterpret_cast<const void*>(&k_spcg<T, false>);
}

template <typename T>
cudaError_t launch_spcg(const SpcgArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<SpcgArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel(spcg_kernel_ptr<T>(a.rows_in_smem != 0), dim3(grid),
                                     dim3(kSpcgThreads), args, smem, s);
}

// ---------------------------------------------------------------------------
// Partitioned PCG on the block-sparse system.  With few blocks per row, the
// redundant design above (every block updates every vector entry) spends its
// time on the full-length vector work; here block b owns the cameras of ranks
// [Cf b / G, Cf (b+1) / G) and keeps only their slices of x, r, z, p and q.  Per
// iteration: (1) the matvec of the owned block rows, reading the p entries of
// other blocks' cameras from their published words; (2) the block's partial
// (p, q), published, and the G partials summed by every block in one fixed order
// (the same alpha everywhere); (3) the slice updates, z = M r, the partials (r, r)
// and (r, z), exchanged the same way; (4) p = z + beta p, published.  Word sets
// alternate by iteration parity: a block writes iteration i + 2 only after it
// summed every block's last partials of i + 1, which each block published after
// its reads of iteration i.  Tags: tag_base for the set-up exchange, tag_base + 1
// + it for iteration it (a launch spans max_iters + 3 tags).
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T poll_word(const unsigned long long* w, unsigned tag, long long timeout_ns, int* late) {
  constexpr int W = spcg_words<T>();
  unsigned long long v[W];
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    bool ready = true;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      v[k] = ld_relaxed_u64(w + k);
      ready &= (unsigned)(v[k] >> 32) == tag;
    }
    if (ready) return spcg_unpack<T>(v);
    if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
      *late = 1;
      return T(0);
    }
  }
}

// partials of one exchange: K dots of this block, published as K values (their
// hi and lo words for FP32), then the G blocks' values summed in block order
template <int K, typename D>
__device__ __forceinline__ int exchange_partials(D (&v)[K], void* red, unsigned long long* set, int G, int bid,
                                                 unsigned tag, long long timeout_ns, int late_in) {
  using T = std::conditional_t<std::is_same<D, double>::value, double, float>;
  constexpr int W = spcg_words<T>();
  constexpr int NV = std::is_same<D, double>::value ? 1 : 2;  // values per dot
  int late = late_in;
  late = block_allsum_dot<K>(v, red, late);
  if (threadIdx.x < K * NV) {
    const int k = threadIdx.x / NV;
    T val;
    if constexpr (NV == 1) val = (T)reinterpret_cast<const double*>(&v[k])[0];
    else val = (threadIdx.x & 1) ? reinterpret_cast<const F2*>(&v[k])->l : reinterpret_cast<const F2*>(&v[k])->h;
    spcg_publish<T>(set + ((size_t)bid * 8 + threadIdx.x) * W, val, tag);
  }
  D acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) dot_zero(acc[k]);
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if constexpr (NV == 1) {
        acc[k] = dot_add(acc[k], poll_word<T>(set + ((size_t)g * 8 + k) * W, tag, timeout_ns, &late));
      } else {
        const float h = poll_word<float>(set + ((size_t)g * 8 + 2 * k) * W, tag, timeout_ns, &late);
        const float l = poll_word<float>(set + ((size_t)g * 8 + 2 * k + 1) * W, tag, timeout_ns, &late);
        acc[k] = dot_add(acc[k], F2{h, l});
      }
    }
  }
  late = block_allsum_dot<K>(acc, reinterpret_cast<char*>(red) + kSpcgRedStride * sizeof(double), late);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = acc[k];
  return late;
}

template <typename T>
__global__ void __launch_bounds__(kSpcgThreads, 1) k_bspcg(SpcgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using D = Dot<T>;
  constexpr int W = spcg_words<T>();
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int Cf = a.Cf, n = a.n;
  const int f0 = (int)(((long long)Cf * bid) / G), f1 = (int)(((long long)Cf * (bid + 1)) / G);
  const int nf = f1 - f0, m = 9 * nf;
  // shared memory: two block-sum buffers, the slices x r z p q, preconditioner blocks
  unsigned char* sp = smem_raw;
  void* red = sp;
  sp += 4 * kSpcgRedStride * sizeof(double);
  T* xs = reinterpret_cast<T*>(sp);
  T* rs = xs + m;
  T* zs = rs + m;
  T* ps = zs + m;
  T* qs = ps + m;
  T* Ms = qs + m;  // kMStride per owned camera
  const T* dinv = reinterpret_cast<const T*>(a.dscale + n);
  unsigned long long* pw = a.words;                                    // [2][n][W]
  unsigned long long* swd = a.words + (size_t)2 * n * W;               // [2][G][8][W]
  const size_t ps_words = (size_t)n * W, ss_words = (size_t)G * 8 * W;
  int late = 0;
  for (int f = tid; f < nf; f += blockDim.x) {
    // the owned cameras' preconditioner blocks (scaled, symmetrised)
    const T* Df = a.Dinv + 81 * (size_t)(f0 + f);
    T d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = (T)a.dscale[9 * (f0 + f) + i];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int j = 0; j < 9; ++j) Ms[kMStride * f + mrow(i) + j] = (T(0.5) * (Df[9 * i + j] + Df[9 * j + i])) * (d[i] * d[j]);
  }
  __syncthreads();
  // r = b^, z = M^ r, p = z, x = 0 on the owned slice; (r, z) and (r, r)
  D d0[2];
  dot_zero(d0[0]);
  dot_zero(d0[1]);
  for (int f = tid; f < nf; f += blockDim.x) {
    const int e = 9 * f, ge = 9 * (f0 + f);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      rs[e + i] = a.b[ge + i] * dinv[ge + i];
      xs[e + i] = T(0);
    }
    spcg_precond(Ms + kMStride * f, rs + e, zs + e);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      ps[e + i] = zs[e + i];
      dot_fma(d0[0], rs[e + i], zs[e + i]);
      dot_fma(d0[1], rs[e + i], rs[e + i]);
    }
  }
  const unsigned tag0 = a.tag_base;
  late = exchange_partials<2>(d0, red, swd + ss_words, G, bid, tag0, a.timeout_ns, late);
  D rz = d0[0];
  const double bnorm = sqrt(dot_value(d0[1]));
  D stop_rr;
  {
    const double st = (a.tol * bnorm) * (a.tol * bnorm);
    if constexpr (sizeof(T) == 4) stop_rr = f2_from_double(st);
    else stop_rr = st;
  }
  D rr_last = d0[1];
  int it = 0;
  const int grp = lane / 9, ra = lane - 9 * grp;
  while (bnorm > 0.0 && it < a.max_iters && !late) {
    const unsigned tag = a.tag_base + 1u + (unsigned)it;
    unsigned long long* pset = pw + (size_t)(it & 1) * ps_words;
    unsigned long long* sset = swd + (size_t)(it & 1) * ss_words;
    // publish this iteration's p slice
    for (int e = tid; e < m; e += blockDim.x) spcg_publish<T>(pset + (size_t)(9 * f0 + e) * W, ps[e], tag);
    __syncthreads();  // the slice is read from shared memory below by other warps
    // matvec of the owned block rows: one warp per camera, three groups of nine
    // lanes; the p entries of four rounds of three blocks are polled together
    // (one L2 round trip for twelve blocks instead of one per three)
    constexpr int kRounds = 4;
    for (int f = warp; f < nf; f += nwarps) {
      const int c = a.cam_map[f0 + f];
      const int e0 = a.brp[c], e1 = a.brp[c + 1];
      T acc = T(0);
      for (int eb = e0; eb < e1; eb += 3 * kRounds) {
        int2 ent[kRounds];
        int cf[kRounds];
        T pv[kRounds];
        unsigned long long wv[kRounds][W];
        bool remote[kRounds];
#pragma unroll
        for (int u = 0; u < kRounds; ++u) {
          const int e = eb + 3 * u + grp;
          ent[u] = make_int2(0, 0);
          cf[u] = -1;
          if (lane < 27 && e < e1) {
            ent[u] = a.bent[e];
            cf[u] = a.crank[ent[u].x];
          }
          remote[u] = cf[u] >= 0 && (cf[u] < f0 || cf[u] >= f1);
          pv[u] = (cf[u] >= 0 && !remote[u]) ? ps[9 * (cf[u] - f0) + ra] : T(0);
        }
        // lane ra of a group fetches entry ra of p for the column camera
        const uint64_t t0 = globaltimer_ns();
        for (;;) {
          bool ready = true;
#pragma unroll
          for (int u = 0; u < kRounds; ++u)
            if (remote[u]) {
#pragma unroll
              for (int k = 0; k < W; ++k) {
                wv[u][k] = ld_relaxed_u64(pset + (size_t)(9 * cf[u] + ra) * W + k);
                ready &= (unsigned)(wv[u][k] >> 32) == tag;
              }
            }
          if (ready) break;
          if ((long long)(globaltimer_ns() - t0) > a.timeout_ns) {
            late = 1;
            break;
          }
        }
#pragma unroll
        for (int u = 0; u < kRounds; ++u) {
          if (remote[u]) pv[u] = late ? T(0) : spcg_unpack<T>(wv[u]);
          const T* row = a.Bs + (size_t)kBlkStride * ent[u].y + 9 * ra;
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const T pt = __shfl_sync(0xffffffffu, pv[u], 9 * grp + t);
            if (cf[u] >= 0) acc = fma(__ldg(row + t), pt, acc);
          }
        }
      }
      const T v1 = __shfl_down_sync(0xffffffffu, acc, 9);
      const T v2 = __shfl_down_sync(0xffffffffu, acc, 18);
      if (lane < 9) qs[9 * f + lane] = (acc + v1) + v2;
    }
    __syncthreads();
    D d1[1];
    dot_zero(d1[0]);
    for (int e = tid; e < m; e += blockDim.x) dot_fma(d1[0], ps[e], qs[e]);
    late = exchange_partials<1>(d1, red, sset, G, bid, tag, a.timeout_ns, late);
    if (late) break;
    const D pq = d1[0];
    if (!dot_pos_finite(pq)) {
      if (bid == 0 && tid == 0) atomicOr(a.err, 2);
      break;
    }
    const T alpha = (T)dot_div(rz, pq);
    D d2[2];
    dot_zero(d2[0]);
    dot_zero(d2[1]);
    for (int e = tid; e < m; e += blockDim.x) {
      xs[e] = fma(alpha, ps[e], xs[e]);
      rs[e] = fma(-alpha, qs[e], rs[e]);
    }
    __syncthreads();
    for (int f = tid; f < nf; f += blockDim.x) {
      spcg_precond(Ms + kMStride * f, rs + 9 * f, zs + 9 * f);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        dot_fma(d2[0], rs[9 * f + i], rs[9 * f + i]);
        dot_fma(d2[1], rs[9 * f + i], zs[9 * f + i]);
      }
    }
    late = exchange_partials<2>(d2, red, sset + (size_t)2 * W, G, bid, tag, a.timeout_ns, late);
    ++it;
    const D rr = d2[0], rz_new = d2[1];
    rr_last = rr;
    if (late || dot_le(rr, stop_rr)) break;
    const T beta = dot_nonzero(rz) ? (T)dot_div(rz_new, rz) : T(0);
    rz = rz_new;
    for (int e = tid; e < m; e += blockDim.x) ps[e] = fma(beta, ps[e], zs[e]);
    __syncthreads();
  }
  if (late && tid == 0) atomicOr(a.err, 1);
  __syncthreads();
  for (int e = tid; e < m; e += blockDim.x) a.x[9 * f0 + e] = xs[e] * dinv[9 * f0 + e];
  if (bid == 0 && tid == 0) {
    a.sc->pcg_iters = it;
    a.sc->pcg_bnorm = bnorm;
    a.sc->pcg_rel_res = bnorm > 0.0 ? sqrt(dot_value(rr_last)) / bnorm : 0.0;
  }
}

template <typename T>
size_t bspcg_smem_bytes(int Cf, int grid) {
  const int nf = (Cf + grid - 1) / grid + 1;
  return 4 * kSpcgRedStride * sizeof(double) + sizeof(T) * ((size_t)5 * 9 * nf + (size_t)kMStride * nf) + 16;
}

template <typename T>
const void* bspcg_kernel_ptr() {
  return reinterpret_cast<const void*>(&k_bspcg<T>);
}

template <typename T>
cudaError_t launch_bspcg(const SpcgArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<SpcgArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel(bspcg_kernel_ptr<T>(), dim3(grid), dim3(kSpcgThreads), args, smem, s);
}

int spcg_threads() { return kSpcgThreads; }
int spcg_words_per_value(bool fp64) { return kSpcgReplicas * (fp64 ? spcg_words<double>() : spcg_words<float>()); }

// ---------------------------------------------------------------------------
// Point back-substitution dp = V*^-1 (-g_p - sum_k W_k^T dc_c(k)) and the point
// part of the predicted decrease, in two passes: one thread per observation forms
// W_k^T dc_c(k) (stored W rows when there are any (explicit system), else W
// recomputed; coalesced over point order), then one thread per point sums its
// observations' terms in point order.
// ---------------------------------------------------------------------------
// orec (FP32, nullable): W_k^T x = w Jp^T (Jc x) = R^T (G (N x_rot + T x_trans) +
// u (g . x_intr)) from the observation record (the factors of Jc and Jp = D R of
// the explicit system's formation), no W row
template <typename T>
__global__ void k_backsub_obs(Layout L, ModelParams mp, const T* __restrict__ camw, const T* __restrict__ ptsw,
                              const uint8_t* __restrict__ act_po, const int* __restrict__ crank,
                              const T* __restrict__ x, const T* __restrict__ Wst, T* __restrict__ wx,
                              const float* __restrict__ orec) {
  const T* po_uv = reinterpret_cast<const T*>(L.po_uvw);
  const T* po_tau = reinterpret_cast<const T*>(L.po_tauw);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += gridDim.x * blockDim.x) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int cr = act_po[k] ? crank[bidx(L.po_cam[k], L.C, 16)] : -1;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (cr >= 0 && orec) {
        const ObsRec r = load_rec(orec, k);
        const float* cam = reinterpret_cast<const float*>(camw) + kCamStride * (size_t)bidx(L.po_cam[k], L.C, 16);
        const bool centre = cam[15] != 0.f;
        const float a[3] = {r.a0, r.a1, r.a2}, g[3] = {r.gi0, r.gi1, r.gi2};
        const float* xv = reinterpret_cast<const float*>(x) + 9 * (size_t)cr;
        // y = N x_rot + T x_trans with N = -[a]x (x_rot x a), T = I or -R
        float y[3] = {xv[1] * a[2] - xv[2] * a[1], xv[2] * a[0] - xv[0] * a[2], xv[0] * a[1] - xv[1] * a[0]};
#pragma unroll
        for (int t = 0; t < 3; ++t)
          y[t] += centre ? -(cam[3 * t] * xv[3] + cam[3 * t + 1] * xv[4] + cam[3 * t + 2] * xv[5]) : xv[3 + t];
        const float gx = g[0] * xv[6] + g[1] * xv[7] + g[2] * xv[8];
        // W^T x = R^T (G y + u (g . x_intr))
        float z[3];
        rec_gvec(r, y, z);
        z[0] += r.u0 * gx, z[1] += r.u1 * gx, z[2] += r.u2 * gx;
        s0 = cam[0] * z[0] + cam[3] * z[1] + cam[6] * z[2];
        s1 = cam[1] * z[0] + cam[4] * z[1] + cam[7] * z[2];
        s2 = cam[2] * z[0] + cam[5] * z[1] + cam[8] * z[2];
        done = true;
      }
    }
    if (cr >= 0 && !done) {
      T W[27];
      if (Wst) {
        load_row27<T>(Wst + kWStride * (size_t)k, W);
      } else {
        T cw[kCamStride];
        load_cam_rec(camw, bidx(L.po_cam[k], L.C, 16), cw);
        obs_W(cw, ptsw + 4 * (size_t)bidx(L.po_pt[k], L.P, 17), po_uv[2 * (size_t)k], po_uv[2 * (size_t)k + 1], po_tau[k], mp, W);
      }
      const T* xv = x + 9 * (size_t)cr;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        s0 += W[3 * q] * xv[q];
        s1 += W[3 * q + 1] * xv[q];
        s2 += W[3 * q + 2] * xv[q];
      }
    }
    wx[3 * (size_t)k] = s0;
    wx[3 * (size_t)k + 1] = s1;
    wx[3 * (size_t)k + 2] = s2;
  }
}

template <typename T>
__global__ void k_backsub_pts(Layout L, const uint8_t* __restrict__ pt_act, const T* __restrict__ wx,
                              const T* __restrict__ Vinv, const T* __restrict__ V, const T* __restrict__ gp,
                              double lambda, T* __restrict__ dp, int Cf, const int* __restrict__ cam_map,
                              const T* __restrict__ x, const T* __restrict__ Ug, const T* __restrict__ dampc,
                              double* __restrict__ pred_parts, Scalars* sc) {
  __shared__ double red[32];
  double pred = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < L.P; p += gridDim.x * blockDim.x) {
    if (!pt_act[p]) {
      dp[3 * (size_t)p] = dp[3 * (size_t)p + 1] = dp[3 * (size_t)p + 2] = T(0);
      continue;
    }
    // the point's terms summed in the working precision (FP64 is the scarce pipe),
    // then combined with the gradient in FP64
    T w0 = T(0), w1 = T(0), w2 = T(0);
    for (int k = L.pt_off[p]; k < L.pt_off[p + 1]; ++k) {
      w0 += wx[3 * (size_t)k];
      w1 += wx[3 * (size_t)k + 1];
      w2 += wx[3 * (size_t)k + 2];
    }
    const double t0 = -(double)gp[3 * (size_t)p] - (double)w0, t1 = -(double)gp[3 * (size_t)p + 1] - (double)w1,
                 t2 = -(double)gp[3 * (size_t)p + 2] - (double)w2;
    const T* v = Vinv + 6 * (size_t)p;
    T d0 = (T)(v[0] * t0 + v[1] * t1 + v[2] * t2);
    T d1 = (T)(v[1] * t0 + v[3] * t1 + v[4] * t2);
    T d2 = (T)(v[2] * t0 + v[4] * t1 + v[5] * t2);
    dp[3 * (size_t)p] = d0;
    dp[3 * (size_t)p + 1] = d1;
    dp[3 * (size_t)p + 2] = d2;
    const T* vv = V + 6 * (size_t)p;
    double dd[3] = {(double)d0, (double)d1, (double)d2};
    double dg[3] = {fmin(fmax((double)vv[0], 1e-6), 1e32), fmin(fmax((double)vv[3], 1e-6), 1e32),
                    fmin(fmax((double)vv[5], 1e-6), 1e32)};
    for (int i = 0; i < 3; ++i) pred += dd[i] * (lambda * dg[i] * dd[i] - (double)gp[3 * (size_t)p + i]);
  }
  // the camera part dc^T (lambda D dc - g_c), spread over the same blocks
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 9 * Cf; e += gridDim.x * blockDim.x) {
    const int f = e / 9, i = e - 9 * f;
    const double d = (double)x[e];
    pred += d * (lambda * (double)dampc[e] * d - (double)Ug[54 * (size_t)cam_map[f] + 45 + i]);
  }
  double s = block_sum(pred, red);
  if (threadIdx.x == 0) pred_parts[blockIdx.x] = s;
  // the last block adds the partials in block order: sc->pred = 1/2 sum
  if (last_block_done(&sc->done_pred)) {
    double a = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) a += __ldcg(pred_parts + i);
    a = block_sum(a, red);
    if (threadIdx.x == 0) {
      sc->pred = 0.5 * a;
      sc->done_pred = 0u;
    }
  }
}

template <typename T>
cudaError_t launch_backsub_pts(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                               const uint8_t* act_po, const uint8_t* pt_act, const int* crank, const T* x,
                               const T* Vinv, const T* V, const T* gp, const T* Wst, double lambda, T* dp,
                               T* wx, int Cf, const int* cam_map, const T* Ug, const T* dampc, double* pred_parts,
                               Scalars* sc, int grid, cudaStream_t s, const float* orec) {
  if (L.N > 0) {
    const int g = (int)std::min<long long>(((long long)L.N + 255) / 256, 65535);
    k_backsub_obs<T><<<g, 256, 0, s>>>(L, mp, camw, ptsw, act_po, crank, x, Wst, wx,
                                       sizeof(T) == 4 ? orec : nullptr);
  }
  k_backsub_pts<T><<<grid, 256, 0, s>>>(L, pt_act, wx, Vinv, V, gp, lambda, dp, Cf, cam_map, x, Ug, dampc,
                                        pred_parts, sc);
  return cudaGetLastError();
}

#define BAB_SINST(T)                                                                                   \
  template cudaError_t launch_form_S<T>(const Layout&, int, const int4*, const int2*, const T*,        \
                                        const T*, const int*, const T*, const T*, double*, int, T*, T*, \
                                        bool, int, cudaEvent_t, cudaEvent_t, cudaEvent_t, cudaStream_t, \
                                        const int*, bool, const CamForm*, const FormRec*);              \
  template cudaError_t launch_dscale<T>(int, const int*, const T*, double, double*, cudaStream_t, int);  \
  template size_t spcg_smem_bytes<T>(int, int, int, int, int);                                         \
  template __host__ __device__ size_t spcg_vec_elems<T>(int, int);                                     \
  template const void* spcg_kernel_ptr<T>(bool);                                                         \
  template cudaError_t launch_spcg<T>(const SpcgArgs<T>&, int, size_t, cudaStream_t);                  \
  template cudaError_t launch_bspcg<T>(const SpcgArgs<T>&, int, size_t, cudaStream_t);                 \
  template size_t bspcg_smem_bytes<T>(int, int);                                                       \
  template const void* bspcg_kernel_ptr<T>();                                                          \
  template cudaError_t launch_spcg_precond<T>(int, const T*, const double*, T*, cudaStream_t);          \
  template cudaError_t launch_backsub_pts<T>(const Layout&, const ModelParams&, const T*, const T*,    \
                                             const uint8_t*, const uint8_t*, const int*, const T*,     \
                                             const T*, const T*, const T*, const T*, double, T*, T*,   \
                                             int, const int*, const T*, const T*, double*, Scalars*, int, \
                                             cudaStream_t, const float*);
BAB_SINST(float)
BAB_SINST(double)

BA_BOUNDS_QUERY(bounds_fault_schur)

}  // namespace bab
