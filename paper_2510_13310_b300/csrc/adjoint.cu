// adjoint.cu -- implicit differentiation of the converged bundle adjustment.
//
// At a stationary point of F the normal-equation gradient g(theta, y) = 0, with
// y the observations (pixels u, v and depth priors d).  With the active set and
// the IRLS weights rho' frozen and the Gauss-Newton matrix H = J^T W rho' J in
// place of the Hessian, the implicit function theorem gives
//   dL/dy = -(dg/dy)^T mu,   H mu = dL/dtheta.
// mu is found with the same Schur-complement solve as an LM step, undamped
// (lambda = 0) and with the gradient replaced by -dL/dtheta; then per
// observation, since dr_k/du_k = -e_0, dr_k/dv_k = -e_1 and
// dr_k/dd_k = sqrt(w) / d_k^2 e_2 (residual sqrt(w)(1/z - 1/d)):
//   dL/du_k = rho'_k (J_k mu)_0,  dL/dv_k = rho'_k (J_k mu)_1,
//   dL/dd_k = -rho'_k sqrt(w_k) tau_k^2 (J_k mu)_2   (tau_k = 1/d_k).
// The Jacobian blocks are recomputed, not stored.  dL/dtheta is the gradient
// in the stored camera parameters (axis-angle, t, f, k1, k2) and point
// coordinates.
#include "internal.h"
#include "model.cuh"

namespace bab {

// The solve runs in the coordinates of the LM update, w <- Log(Exp(dw) Exp(w)),
// in which d w / d dw = Jl(w)^-1 (inverse left Jacobian of SO(3)):
//   Jl^-1 = I - [w]x / 2 + c2 [w]x^2,  c2 = 1/th^2 - (1 + cos th) / (2 th sin th),
// with c2 = 1/12 + th^2/720 near th = 0.  So the rotation block of the adjoint
// right-hand side is Jl(w)^-T dL/dw; translation and intrinsics pass through.
__device__ __forceinline__ void so3_jl_inv_T_apply(const double* w, const double* g, double* out) {
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const double th = sqrt(th2);
  const double c2 = th < 1e-4 ? 1.0 / 12.0 + th2 / 720.0 : 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
  // out = (I - K/2 + c2 K^2)^T g = g + (K g)/2 + c2 K^2 g, with K = [w]x (K^T = -K, (K^2)^T = K^2)
  const double kg0 = w[1] * g[2] - w[2] * g[1];
  const double kg1 = w[2] * g[0] - w[0] * g[2];
  const double kg2 = w[0] * g[1] - w[1] * g[0];
  const double kkg0 = w[1] * kg2 - w[2] * kg1;
  const double kkg1 = w[2] * kg0 - w[0] * kg2;
  const double kkg2 = w[0] * kg1 - w[1] * kg0;
  out[0] = g[0] + 0.5 * kg0 + c2 * kkg0;
  out[1] = g[1] + 0.5 * kg1 + c2 * kkg1;
  out[2] = g[2] + 0.5 * kg2 + c2 * kkg2;
}

// g_c := -(Jl^-T dL/dw, dL/dt, dL/df, dL/dk) for free cameras (the gradient slot
// of the packed camera record), g_p := -dL/dpts for active points, zero elsewhere.
template <typename T>
__global__ void k_adjoint_rhs(int C, int P, const double* __restrict__ cams64, const int* __restrict__ crank,
                              const uint8_t* __restrict__ pt_act, const double* __restrict__ dL_dc,
                              const double* __restrict__ dL_dp, T* __restrict__ Ug, T* __restrict__ gp,
                              double* __restrict__ a_c, double* __restrict__ a_p, int kfix) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < C) {
    const int c = (int)i;
    T* g = Ug + 54 * (size_t)c + 45;
    double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (crank[c] >= 0) {
      const double* d = dL_dc + 9 * (size_t)c;
      so3_jl_inv_T_apply(cams64 + 9 * (size_t)c, d, a);
#pragma unroll
      for (int j = 3; j < 9; ++j) a[j] = d[j];
      if (kfix) a[7] = a[8] = 0.0;  // not parameters under the camera model of Sec. 3.2
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      g[j] = (T)(-a[j]);
      if (a_c) a_c[9 * (size_t)c + j] = a[j];
    }
  }
  if (i < 3LL * P) {
    const int p = (int)(i / 3);
    const double a = pt_act[p] ? dL_dp[i] : 0.0;
    gp[i] = (T)(-a);
    if (a_p) a_p[i] = a;
  }
}

template <typename T>
cudaError_t launch_adjoint_rhs(int C, int P, const double* cams64, const int* crank, const uint8_t* pt_act,
                               const double* dL_dc, const double* dL_dp, T* Ug, T* gp, cudaStream_t s,
                               double* a_c, double* a_p, int kfix) {
  const long long n = std::max((long long)C, 3LL * P);
  if (n > 0)
    k_adjoint_rhs<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, P, cams64, crank, pt_act, dL_dc, dL_dp, Ug, gp,
                                                                  a_c, a_p, kfix);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64-residual refinement of the FP32 adjoint solve.  The scale direction of
// these problems (fixed by the depth priors alone) is ~1e-6 as stiff as the rest,
// so an FP32 solve of H mu = a resolves it to a few percent.  The residual
// a - H mu is formed with FP64 Jacobian blocks at the FP64 state (H = J^T rho' J
// over the active observations, IRLS weights frozen), the correction solves
// H delta = a - H mu with the same FP32 Schur solver, and mu accumulates in FP64.
// ---------------------------------------------------------------------------

// per point: u_k = rho'_k (J_c mu_c + J_p mu_p) for its active observations (stored
// in point order) and (H mu)_p = sum_k J_p^T u_k
__global__ void k_adj_hmu_pts(Layout L, ModelParams mp, const double* __restrict__ camw64,
                              const double* __restrict__ pts64, const uint8_t* __restrict__ act_po,
                              const int* __restrict__ crank, const double* __restrict__ mu_c,
                              const double* __restrict__ mu_p, double* __restrict__ u_obs,
                              double* __restrict__ hmu_p) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.P) return;
  const double X0 = pts64[3 * (size_t)p], X1 = pts64[3 * (size_t)p + 1], X2 = pts64[3 * (size_t)p + 2];
  const double m0 = mu_p[3 * (size_t)p], m1 = mu_p[3 * (size_t)p + 1], m2 = mu_p[3 * (size_t)p + 2];
  double h0 = 0.0, h1 = 0.0, h2 = 0.0;
  for (int k = L.pt_off[p]; k < L.pt_off[p + 1]; ++k) {
    double* u = u_obs + 3 * (size_t)k;
    if (!act_po[k]) {
      u[0] = u[1] = u[2] = 0.0;
      continue;
    }
    const int c = bidx(L.po_cam[k], L.C, 20), cr = crank[c];
    const double tau = L.po_tau64[k];
    const double sw = tau > 0.0 ? mp.sw_valid : mp.sw_invalid;
    ObsLin<double> ol;
    linearize_obs<double>(camw64 + kCamStride * (size_t)c, X0, X1, X2, L.po_uv64[2 * (size_t)k],
                          L.po_uv64[2 * (size_t)k + 1], tau, sw, mp.cx, mp.cy, mp.huber, ol);
    double v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double acc = ol.Jp[r][0] * m0 + ol.Jp[r][1] * m1 + ol.Jp[r][2] * m2;
      if (cr >= 0)
#pragma unroll
        for (int i = 0; i < 9; ++i) acc += ol.Jc[r][i] * mu_c[9 * (size_t)cr + i];
      v[r] = ol.wrob * acc;
      u[r] = v[r];
    }
    h0 += ol.Jp[0][0] * v[0] + ol.Jp[1][0] * v[1] + ol.Jp[2][0] * v[2];
    h1 += ol.Jp[0][1] * v[0] + ol.Jp[1][1] * v[1] + ol.Jp[2][1] * v[2];
    h2 += ol.Jp[0][2] * v[0] + ol.Jp[1][2] * v[1] + ol.Jp[2][2] * v[2];
  }
  hmu_p[3 * (size_t)p] = h0;
  hmu_p[3 * (size_t)p + 1] = h1;
  hmu_p[3 * (size_t)p + 2] = h2;
}

// per camera-order chunk: sum over its active observations of J_c^T u_k (FP64),
// strided per thread, then a fixed-order block sum
constexpr int kAdjThreads = 128;
__global__ void __launch_bounds__(kAdjThreads) k_adj_hmu_cams(Layout L, ModelParams mp,
                                                              const double* __restrict__ camw64,
                                                              const double* __restrict__ pts64,
                                                              const uint8_t* __restrict__ act_co,
                                                              const int* __restrict__ crank,
                                                              const double* __restrict__ u_obs,
                                                              double* __restrict__ part) {
  __shared__ double red[kAdjThreads / 32][9];
  const int q = blockIdx.x, c = L.chunk_cam[q];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (crank[c] >= 0) {
    for (int kc = L.chunk_obs[q] + threadIdx.x; kc < L.chunk_obs[q + 1]; kc += blockDim.x) {
      if (!act_co[kc]) continue;
      const int k = bidx(L.co_po[kc], L.N, 21), p = bidx(L.co_pt[kc], L.P, 21);
      const double tau = L.po_tau64[k];
      const double sw = tau > 0.0 ? mp.sw_valid : mp.sw_invalid;
      ObsLin<double> ol;
      linearize_obs<double>(camw64 + kCamStride * (size_t)c, pts64[3 * (size_t)p], pts64[3 * (size_t)p + 1],
                            pts64[3 * (size_t)p + 2], L.po_uv64[2 * (size_t)k], L.po_uv64[2 * (size_t)k + 1], tau,
                            sw, mp.cx, mp.cy, mp.huber, ol);
      const double* u = u_obs + 3 * (size_t)k;
#pragma unroll
      for (int i = 0; i < 9; ++i) acc[i] += ol.Jc[0][i] * u[0] + ol.Jc[1][i] * u[1] + ol.Jc[2][i] * u[2];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double v = acc[i];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kAdjThreads / 32; ++w) v += red[w][threadIdx.x];
    part[9 * (size_t)q + threadIdx.x] = v;
  }
}

// r = a - H mu (cameras: the chunk partials summed in chunk order), written into
// the gradient slots as -r for the correction solve
template <typename T>
__global__ void k_adj_residual(int C, int P, const int* __restrict__ cam_chunk, const int* __restrict__ crank,
                               const uint8_t* __restrict__ pt_act, const double* __restrict__ part,
                               const double* __restrict__ hmu_p, const double* __restrict__ a_c,
                               const double* __restrict__ a_p, T* __restrict__ Ug, T* __restrict__ gp) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < C) {
    const int c = (int)i;
    T* g = Ug + 54 * (size_t)c + 45;
    if (crank[c] < 0) {
#pragma unroll
      for (int j = 0; j < 9; ++j) g[j] = T(0);
    } else {
      for (int j = 0; j < 9; ++j) {
        double h = 0.0;
        for (int q = cam_chunk[c]; q < cam_chunk[c + 1]; ++q) h += part[9 * (size_t)q + j];
        g[j] = (T)(-(a_c[9 * (size_t)c + j] - h));
      }
    }
  }
  if (i < 3LL * P) {
    const int p = (int)(i / 3);
    gp[i] = pt_act[p] ? (T)(-(a_p[i] - hmu_p[i])) : T(0);
  }
}

// mu (FP64) = x, dp of the latest solve (first) or mu + them
template <typename T>
__global__ void k_adj_mu_add(int Cf, int P, const T* __restrict__ x, const T* __restrict__ dp,
                             double* __restrict__ mu_c, double* __restrict__ mu_p, int first) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < 9LL * Cf) mu_c[i] = (first ? 0.0 : mu_c[i]) + (double)x[i];
  if (i < 3LL * P) mu_p[i] = (first ? 0.0 : mu_p[i]) + (double)dp[i];
}

// per-observation gradients from mu in FP64 (input order)
__global__ void k_adjoint_obs64(Layout L, ModelParams mp, const double* __restrict__ camw64,
                                const double* __restrict__ pts64, const uint8_t* __restrict__ act_po,
                                const int* __restrict__ crank, const double* __restrict__ mu_c,
                                const double* __restrict__ mu_p, double* __restrict__ duv,
                                double* __restrict__ ddepth) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.N) return;
  const int o = bidx(L.po_orig[k], L.N, 24);
  if (!act_po[k]) {
    duv[2 * (size_t)o] = 0.0;
    duv[2 * (size_t)o + 1] = 0.0;
    ddepth[o] = 0.0;
    return;
  }
  const int c = bidx(L.po_cam[k], L.C, 22), p = bidx(L.po_pt[k], L.P, 22), cr = crank[c];
  const double tau = L.po_tau64[k];
  const double sw = tau > 0.0 ? mp.sw_valid : mp.sw_invalid;
  ObsLin<double> ol;
  linearize_obs<double>(camw64 + kCamStride * (size_t)c, pts64[3 * (size_t)p], pts64[3 * (size_t)p + 1],
                        pts64[3 * (size_t)p + 2], L.po_uv64[2 * (size_t)k], L.po_uv64[2 * (size_t)k + 1], tau, sw,
                        mp.cx, mp.cy, mp.huber, ol);
  double Jm[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double acc = ol.Jp[r][0] * mu_p[3 * (size_t)p] + ol.Jp[r][1] * mu_p[3 * (size_t)p + 1] +
                 ol.Jp[r][2] * mu_p[3 * (size_t)p + 2];
    if (cr >= 0)
#pragma unroll
      for (int i = 0; i < 9; ++i) acc += ol.Jc[r][i] * mu_c[9 * (size_t)cr + i];
    Jm[r] = acc;
  }
  duv[2 * (size_t)o] = ol.wrob * Jm[0];
  duv[2 * (size_t)o + 1] = ol.wrob * Jm[1];
  ddepth[o] = tau > 0.0 ? -ol.wrob * sw * tau * tau * Jm[2] : 0.0;
}

cudaError_t launch_adj_hmu(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                           const uint8_t* act_po, const uint8_t* act_co, const int* crank, const double* mu_c,
                           const double* mu_p, double* u_obs, double* hmu_p, double* part, cudaStream_t s) {
  if (L.P > 0)
    k_adj_hmu_pts<<<(L.P + 127) / 128, 128, 0, s>>>(L, mp, camw64, pts64, act_po, crank, mu_c, mu_p, u_obs, hmu_p);
  if (L.n_chunks > 0)
    k_adj_hmu_cams<<<L.n_chunks, kAdjThreads, 0, s>>>(L, mp, camw64, pts64, act_co, crank, u_obs, part);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_residual(int C, int P, const int* cam_chunk, const int* crank, const uint8_t* pt_act,
                                const double* part, const double* hmu_p, const double* a_c, const double* a_p,
                                T* Ug, T* gp, cudaStream_t s) {
  const long long n = std::max((long long)C, 3LL * P);
  if (n > 0)
    k_adj_residual<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C, P, cam_chunk, crank, pt_act, part, hmu_p,
                                                                   a_c, a_p, Ug, gp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_mu_add(int Cf, int P, const T* x, const T* dp, double* mu_c, double* mu_p, bool first,
                              cudaStream_t s) {
  const long long n = std::max(9LL * Cf, 3LL * P);
  if (n > 0)
    k_adj_mu_add<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Cf, P, x, dp, mu_c, mu_p, first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_obs64(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                                 const uint8_t* act_po, const int* crank, const double* mu_c, const double* mu_p,
                                 double* duv, double* ddepth, cudaStream_t s) {
  if (L.N > 0)
    k_adjoint_obs64<<<(L.N + 127) / 128, 128, 0, s>>>(L, mp, camw64, pts64, act_po, crank, mu_c, mu_p, duv, ddepth);
  return cudaGetLastError();
}

// One thread per point-order observation; outputs in the input order.
template <typename T>
__global__ void k_adjoint_obs(Layout L, ModelParams mp, const T* __restrict__ camw, const T* __restrict__ ptsw,
                              const uint8_t* __restrict__ act_po, const int* __restrict__ crank,
                              const T* __restrict__ x, const T* __restrict__ dp, double* __restrict__ duv,
                              double* __restrict__ ddepth) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L.N) return;
  const int o = bidx(L.po_orig[k], L.N, 24);
  if (!act_po[k]) {
    duv[2 * (size_t)o] = 0.0;
    duv[2 * (size_t)o + 1] = 0.0;
    ddepth[o] = 0.0;
    return;
  }
  const T* po_uv = reinterpret_cast<const T*>(L.po_uvw);
  const T* po_tau = reinterpret_cast<const T*>(L.po_tauw);
  const int c = bidx(L.po_cam[k], L.C, 23), p = bidx(L.po_pt[k], L.P, 23);
  T cw[kCamStride];
#pragma unroll
  for (int q = 0; q < kCamStride; ++q) cw[q] = camw[kCamStride * (size_t)c + q];
  const T* X = ptsw + 4 * (size_t)p;
  const T tau = po_tau[k];
  const T sw = tau > T(0) ? (T)mp.sw_valid : (T)mp.sw_invalid;
  ObsLin<T> ol;
  linearize_obs<T>(cw, X[0], X[1], X[2], po_uv[2 * (size_t)k], po_uv[2 * (size_t)k + 1], tau, sw, (T)mp.cx,
                   (T)mp.cy, (T)mp.huber, ol);
  T mc[9];
  const int cr = crank[c];
#pragma unroll
  for (int i = 0; i < 9; ++i) mc[i] = cr >= 0 ? x[9 * (size_t)cr + i] : T(0);
  const T m0 = dp[3 * (size_t)p], m1 = dp[3 * (size_t)p + 1], m2 = dp[3 * (size_t)p + 2];
  T Jm[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    T acc = ol.Jp[r][0] * m0 + ol.Jp[r][1] * m1 + ol.Jp[r][2] * m2;
#pragma unroll
    for (int i = 0; i < 9; ++i) acc += ol.Jc[r][i] * mc[i];
    Jm[r] = acc;
  }
  duv[2 * (size_t)o] = (double)(ol.wrob * Jm[0]);
  duv[2 * (size_t)o + 1] = (double)(ol.wrob * Jm[1]);
  ddepth[o] = tau > T(0) ? (double)(-ol.wrob * sw * tau * tau * Jm[2]) : 0.0;
}

template <typename T>
cudaError_t launch_adjoint_obs(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                               const uint8_t* act_po, const int* crank, const T* x, const T* dp, double* duv,
                               double* ddepth, cudaStream_t s) {
  if (L.N > 0) k_adjoint_obs<T><<<(L.N + 255) / 256, 256, 0, s>>>(L, mp, camw, ptsw, act_po, crank, x, dp, duv, ddepth);
  return cudaGetLastError();
}

#define BAB_INST_ADJ(T)                                                                                   \
  template cudaError_t launch_adjoint_rhs<T>(int, int, const double*, const int*, const uint8_t*,      \
                                             const double*, const double*, T*, T*, cudaStream_t,         \
                                             double*, double*, int);                                     \
  template cudaError_t launch_adj_residual<T>(int, int, const int*, const int*, const uint8_t*,         \
                                              const double*, const double*, const double*, const double*, \
                                              T*, T*, cudaStream_t);                                     \
  template cudaError_t launch_adj_mu_add<T>(int, int, const T*, const T*, double*, double*, bool,       \
                                            cudaStream_t);                                               \
  template cudaError_t launch_adjoint_obs<T>(const Layout&, const ModelParams&, const T*, const T*,     \
                                             const uint8_t*, const int*, const T*, const T*, double*,    \
                                             double*, cudaStream_t);
BAB_INST_ADJ(float)
BAB_INST_ADJ(double)

BA_BOUNDS_QUERY(bounds_fault_adjoint)

}  // namespace bab
