// kernels.cu -- sm_103a kernels of one LM bundle-adjustment iteration.
//
// Observation streams are kept in two sorted layouts built once at creation:
// point order (tiles of whole points) for everything reduced per point and for
// the Schur matvec, camera order (chunks inside one camera) for everything
// reduced per camera.  No kernel uses global floating-point atomics: camera
// sums go through fixed-order chunk partials, point sums through per-tile
// shared memory.
#include "df.cuh"
#include "internal.h"
#include "model.cuh"

namespace bab {

// ---------------------------------------------------------------------------
// working copies of the state
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_prep_cams(const double* __restrict__ cams64, T* __restrict__ camw,
                            double* __restrict__ camw64, int C, int model) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double rec[kCamStride];
  cam_record(cams64 + 9 * (size_t)c, model, rec);
  for (int i = 0; i < kCamStride; ++i) camw[kCamStride * (size_t)c + i] = (T)rec[i];
  if (camw64)
    for (int i = 0; i < kCamStride; ++i) camw64[kCamStride * (size_t)c + i] = rec[i];
}

template <typename T>
cudaError_t launch_prep_cams(const double* cams64, T* camw, double* camw64, int C, cudaStream_t s, int model) {
  if (C > 0) k_prep_cams<T><<<(C + 127) / 128, 128, 0, s>>>(cams64, camw, camw64, C, model);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_prep_pts(const double* __restrict__ pts64, T* __restrict__ ptsw, int P) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  using V4 = typename Vec4<T>::type;
  V4 v;
  v.x = (T)pts64[3 * (size_t)p];
  v.y = (T)pts64[3 * (size_t)p + 1];
  v.z = (T)pts64[3 * (size_t)p + 2];
  v.w = T(0);
  reinterpret_cast<V4*>(ptsw)[p] = v;
}

template <typename T>
cudaError_t launch_prep_pts(const double* pts64, T* ptsw, int P, cudaStream_t s) {
  if (P > 0) k_prep_pts<T><<<(P + 255) / 256, 256, 0, s>>>(pts64, ptsw, P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// observation arrays of both layouts, gathered once at creation from the
// caller's arrays through the point-order and camera-order permutations
// ---------------------------------------------------------------------------

// inverse-depth prior tau = 1/d of one observation (Sec. 4.1), 0 where the
// depth is missing (not positive or not finite)
__device__ __forceinline__ double inv_depth_prior(double d) {
  return (d > 0.0 && isfinite(d)) ? 1.0 / d : 0.0;
}

template <typename T>
__global__ void k_obs_point_order(int N, const double* __restrict__ uv, const double* __restrict__ depth,
                                  const int* __restrict__ po, int* __restrict__ po_wrow,
                                  double* __restrict__ po_uv64, double* __restrict__ po_tau64,
                                  T* __restrict__ po_uvw, T* __restrict__ po_tauw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int k = po[i];
    po_wrow[i] = i;
    const double u = uv[2 * (size_t)k], v = uv[2 * (size_t)k + 1], tau = inv_depth_prior(depth[k]);
    po_uv64[2 * (size_t)i] = u;
    po_uv64[2 * (size_t)i + 1] = v;
    po_tau64[i] = tau;
    if (po_uvw) {
      po_uvw[2 * (size_t)i] = (T)u;
      po_uvw[2 * (size_t)i + 1] = (T)v;
      po_tauw[i] = (T)tau;
    }
  }
}

template <typename T>
__global__ void k_obs_camera_order(int N, const double* __restrict__ uv, const double* __restrict__ depth,
                                   const int* __restrict__ co, const int* __restrict__ co_po,
                                   const int* __restrict__ po_pt, int* __restrict__ co_pt, T* __restrict__ co_uvw,
                                   T* __restrict__ co_tauw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int k = co[i];
    co_pt[i] = po_pt[co_po[i]];
    co_uvw[2 * (size_t)i] = (T)uv[2 * (size_t)k];
    co_uvw[2 * (size_t)i + 1] = (T)uv[2 * (size_t)k + 1];
    co_tauw[i] = (T)inv_depth_prior(depth[k]);
  }
}

template <typename T>
cudaError_t launch_obs_layout(int N, const double* uv, const double* depth, const int* po, const int* co,
                              const int* co_po, const int* po_pt, int* po_wrow, double* po_uv64, double* po_tau64,
                              T* po_uvw, T* po_tauw, int* co_pt, T* co_uvw, T* co_tauw, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(((long long)N + 255) / 256, 65535);
  k_obs_point_order<T><<<grid, 256, 0, s>>>(N, uv, depth, po, po_wrow, po_uv64, po_tau64, po_uvw, po_tauw);
  k_obs_camera_order<T><<<grid, 256, 0, s>>>(N, uv, depth, co, co_po, po_pt, co_pt, co_uvw, co_tauw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 evaluation: cost over the active set and validity bits of a state
// (Eq. BA objective with depth; Sec. 4.2 step 1 validity)
// ---------------------------------------------------------------------------

// sc->cost[slot] = 1/2 sum, rmse_sum, n_act from the blocks' partials, in the
// last block of the evaluation kernel: each sum over the block partials in a
// fixed thread assignment and tree
__device__ __forceinline__ void eval_finish(const double* __restrict__ partials, Scalars* sc, int slot) {
  if (!last_block_done(&sc->done_eval)) return;
  __shared__ double red[32];
  double a = 0, b = 0, c = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(partials + 3 * i);
    b += __ldcg(partials + 3 * i + 1);
    c += __ldcg(partials + 3 * i + 2);
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  c = block_sum(c, red);
  if (threadIdx.x == 0) {
    sc->cost[slot] = 0.5 * a;
    sc->rmse_sum[slot] = b;
    sc->n_act[slot] = c;
    sc->done_eval = 0u;
  }
}

// bits: 1 = geometrically valid (z > min_depth, pixel inside the image),
//       2 = valid and |r_uv| above the residual-drop threshold.
// ref_bits (nullable): validity bits of another state; any difference in bit 1
// sets *flips (the active set extracted from ref_bits then still applies).
__global__ void k_eval64(Layout L, ModelParams mp, const double* __restrict__ camw64,
                         const double* __restrict__ pts64, const uint8_t* __restrict__ act,
                         uint8_t* __restrict__ bits, const uint8_t* __restrict__ ref_bits,
                         int* __restrict__ flips, double* __restrict__ partials, Scalars* sc, int slot) {
  int flip = 0;
  __shared__ double red[32];
  double acc_cost = 0.0, acc_e2 = 0.0;
  int acc_n = 0;
  // thresholds of the validity predicate as integer keys (FP64 comparisons are FP64-pipe work)
  const long long kz = dkey(mp.min_depth), kw = dkey((double)mp.img_w), kh = dkey((double)mp.img_h);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += gridDim.x * blockDim.x) {
    int c = bidx(L.po_cam[k], L.C, 0), p = bidx(L.po_pt[k], L.P, 1);
    const double* X = pts64 + 3 * (size_t)p;
    double tau = L.po_tau64[k];
    double sw = __double_as_longlong(tau) > 0 ? mp.sw_valid : mp.sw_invalid;  // tau > 0
    Eval64 e = eval_obs64(camw64 + kCamStride * (size_t)c, X[0], X[1], X[2], L.po_uv64[2 * (size_t)k],
                          L.po_uv64[2 * (size_t)k + 1], tau, sw, mp.cx, mp.cy);
    double e2 = fma(e.r0, e.r0, e.r1 * e.r1);
    if (bits) {
      const long long ku = dkey(e.uh), kv = dkey(e.vh);
      int ok = dkey(e.z) > kz && ku >= 0 && ku < kw && kv >= 0 && kv < kh;
      int b = ok ? 1 : 0;
      if (ok && mp.drop_px > 0.0 && sqrt(e2) > mp.drop_px) b |= 2;
      bits[k] = (uint8_t)b;
      if (ref_bits) flip |= (b ^ ref_bits[k]) & 1;
    }
    if (act && act[k]) {
      acc_cost += huber_loss(fma(e.r2, e.r2, e2), mp.huber);
      acc_e2 += e2;
      acc_n += 1;
    }
  }
  if (ref_bits) {
    if (__syncthreads_or(flip) && threadIdx.x == 0) atomicOr(flips, 1);
  }
  if (!partials) return;
  double s0 = block_sum(acc_cost, red);
  double s1 = block_sum(acc_e2, red);
  __shared__ int redi[32];
  int s2 = block_sum(acc_n, redi);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = s0;
    partials[3 * blockIdx.x + 1] = s1;
    partials[3 * blockIdx.x + 2] = (double)s2;
  }
  eval_finish(partials, sc, slot);
}

cudaError_t launch_eval64(const Layout& L, const ModelParams& mp, const double* camw64,
                          const double* pts64, const uint8_t* act, uint8_t* bits,
                          const uint8_t* ref_bits, int* flips, double* partials, Scalars* sc, int slot, int grid,
                          cudaStream_t s) {
  k_eval64<<<grid, kBlock, 0, s>>>(L, mp, camw64, pts64, act, bits, bits ? ref_bits : nullptr, flips,
                                    partials, sc, slot);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The same evaluation in double-float arithmetic (FP32 problems): FP64 is the
// scarce pipe on this part, and the projection needs ~1e-15 relative accuracy
// only because the residual uh - u cancels three to four digits.  Every
// validity decision whose double-float margin is within 2^-30 of the scale of
// its operands, and every observation with a non-finite intermediate, is
// re-evaluated in FP64 (eval_obs64), so the bits follow the FP64 definition.
// ---------------------------------------------------------------------------

// cameras [C][32] floats: R (9), t (3), f, k1, k2 as (hi, lo) pairs; points
// [P][2] float4: (X0, X1), (X2, 0)
__global__ void k_state_df(int C, int P, const double* __restrict__ camw64, const double* __restrict__ pts64,
                           F2* __restrict__ camdf, float4* __restrict__ ptdf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(C * 16, P); i += gridDim.x * blockDim.x) {
    if (i < C * 16) {
      const int c = i >> 4, q = i & 15;
      camdf[16 * (size_t)c + q] = q < 15 ? f2_from_double(camw64[kCamStride * (size_t)c + q]) : F2{0.f, 0.f};
    }
    if (i < P) {
      const F2 x0 = f2_from_double(pts64[3 * (size_t)i]), x1 = f2_from_double(pts64[3 * (size_t)i + 1]),
               x2 = f2_from_double(pts64[3 * (size_t)i + 2]);
      ptdf[2 * (size_t)i] = make_float4(x0.h, x0.l, x1.h, x1.l);
      ptdf[2 * (size_t)i + 1] = make_float4(x2.h, x2.l, 0.f, 0.f);
    }
  }
}

// observations in point order: (u, v) and tau as (hi, lo) pairs, once at creation
__global__ void k_obs_df(int N, const double* __restrict__ uv64, const double* __restrict__ tau64,
                         float4* __restrict__ uvdf, F2* __restrict__ taudf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const F2 u = f2_from_double(uv64[2 * (size_t)k]), v = f2_from_double(uv64[2 * (size_t)k + 1]);
    uvdf[k] = make_float4(u.h, u.l, v.h, v.l);
    taudf[k] = f2_from_double(tau64[k]);
  }
}

// |d| is not clearly away from 0 at the scale `scale` of the compared values
__device__ __forceinline__ bool near_zero(F2 d, float scale) { return fabsf(d.h) <= scale * 0x1p-30f; }

__global__ void __launch_bounds__(kBlock) k_eval_df(Layout L, ModelParams mp, EvalDFConst ec, const F2* __restrict__ camdf,
                                                    const float4* __restrict__ ptdf, const double* __restrict__ camw64,
                                                    const double* __restrict__ pts64, const uint8_t* __restrict__ act,
                                                    uint8_t* __restrict__ bits, const uint8_t* __restrict__ ref_bits,
                                                    int* __restrict__ flips, double* __restrict__ partials,
                                                    Scalars* sc, int slot, int cam_smem) {
  // the camera table in shared memory when it fits, 9 float4 per camera (the
  // odd stride spreads the lanes' random cameras over the bank groups)
  extern __shared__ __align__(16) float4 cam_s[];
  const bool cam_in_smem = cam_smem;
  if (cam_in_smem) {
    const float4* src = reinterpret_cast<const float4*>(camdf);
    for (int i = threadIdx.x; i < 8 * L.C; i += blockDim.x) cam_s[9 * (i >> 3) + (i & 7)] = src[i];
    __syncthreads();
  }
  int flip = 0;
  F2 acc_cost{0.f, 0.f}, acc_e2{0.f, 0.f};
  int acc_n = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += gridDim.x * blockDim.x) {
    const int c = bidx(L.po_cam[k], L.C, 2), p = bidx(L.po_pt[k], L.P, 3);
    F2 cw[16];
    {
      const float4* cr = cam_in_smem ? cam_s + 9 * c : reinterpret_cast<const float4*>(camdf) + 8 * (size_t)c;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = cr[q];
        cw[2 * q] = F2{v.x, v.y};
        cw[2 * q + 1] = F2{v.z, v.w};
      }
    }
    const float4 xa = ptdf[2 * (size_t)p], xb = ptdf[2 * (size_t)p + 1];
    const F2 X0{xa.x, xa.y}, X1{xa.z, xa.w}, X2{xb.x, xb.y};
    const float4 uv = L.po_uvdf[k];
    const F2 tau = L.po_taudf[k];
    const bool has_d = tau.h > 0.f;
    const F2 px = f2_add(f2_fma(cw[0], X0, f2_fma(cw[1], X1, f2_mul(cw[2], X2))), cw[9]);
    const F2 py = f2_add(f2_fma(cw[3], X0, f2_fma(cw[4], X1, f2_mul(cw[5], X2))), cw[10]);
    const F2 pz = f2_add(f2_fma(cw[6], X0, f2_fma(cw[7], X1, f2_mul(cw[8], X2))), cw[11]);
    const F2 iz = f2_recip(pz);
    const F2 xn = f2_mul(px, iz), yn = f2_mul(py, iz);
    const F2 rr = f2_fma(xn, xn, f2_mul(yn, yn));
    const F2 dist = f2_fma(rr, f2_fma(cw[14], rr, cw[13]), F2{1.f, 0.f});
    const F2 fd = f2_mul(cw[12], dist);
    const F2 uh = f2_fma(fd, xn, ec.cx), vh = f2_fma(fd, yn, ec.cy);
    const F2 r0 = f2_sub(uh, F2{uv.x, uv.y}), r1 = f2_sub(vh, F2{uv.z, uv.w});
    const F2 r2 = f2_mul(has_d ? ec.sw_valid : ec.sw_invalid, f2_sub(iz, tau));
    const F2 e2 = f2_fma(r0, r0, f2_mul(r1, r1));
    const F2 s = f2_fma(r2, r2, e2);
    bool slow = !(f2_finite(uh) && f2_finite(vh) && f2_finite(pz) && f2_finite(s));
    int b = 0;
    if (bits && !slow) {
      const F2 dz = f2_sub(pz, ec.min_depth);
      const F2 du = f2_sub(uh, ec.img_w), dv = f2_sub(vh, ec.img_h);
      const float su = fabsf(uh.h) + fabsf(ec.cx.h) + fabsf(ec.img_w.h);
      const float sv = fabsf(vh.h) + fabsf(ec.cy.h) + fabsf(ec.img_h.h);
      slow = near_zero(dz, fabsf(pz.h) + fabsf(ec.min_depth.h)) || near_zero(uh, su) || near_zero(du, su) ||
             near_zero(vh, sv) || near_zero(dv, sv);
      const bool ok = dz.h > 0.f && uh.h >= 0.f && du.h < 0.f && vh.h >= 0.f && dv.h < 0.f;
      b = ok ? 1 : 0;
      if (ok && ec.drop2.h > 0.f) {
        const F2 dd = f2_sub(e2, ec.drop2);
        slow = slow || near_zero(dd, e2.h + ec.drop2.h);
        if (dd.h > 0.f) b |= 2;
      }
    }
    F2 rho = s, e2v = e2;
    if (slow) {
      // FP64 evaluation of this observation (rare)
      const double* X = pts64 + 3 * (size_t)p;
      const double tau64 = L.po_tau64[k];
      const double sw = __double_as_longlong(tau64) > 0 ? mp.sw_valid : mp.sw_invalid;
      const Eval64 e = eval_obs64(camw64 + kCamStride * (size_t)c, X[0], X[1], X[2], L.po_uv64[2 * (size_t)k],
                                  L.po_uv64[2 * (size_t)k + 1], tau64, sw, mp.cx, mp.cy);
      const double e2d = fma(e.r0, e.r0, e.r1 * e.r1);
      if (bits) {
        const long long kz = dkey(mp.min_depth), kw = dkey((double)mp.img_w), kh = dkey((double)mp.img_h);
        const long long ku = dkey(e.uh), kv = dkey(e.vh);
        const int ok = dkey(e.z) > kz && ku >= 0 && ku < kw && kv >= 0 && kv < kh;
        b = ok ? 1 : 0;
        if (ok && mp.drop_px > 0.0 && sqrt(e2d) > mp.drop_px) b |= 2;
      }
      e2v = f2_from_double(e2d);
      rho = f2_from_double(huber_loss(fma(e.r2, e.r2, e2d), mp.huber));
    } else if (ec.huber.h > 0.f && f2_sub(s, ec.huber2).h > 0.f) {
      rho = f2_sub(f2_mul(ec.two_huber, f2_sqrt(s)), ec.huber2);  // 2 delta sqrt(s) - delta^2
    }
    if (bits) {
      bits[k] = (uint8_t)b;
      if (ref_bits) flip |= (b ^ ref_bits[k]) & 1;
    }
    if (act && act[k]) {
      acc_cost = f2_add(acc_cost, rho);
      acc_e2 = f2_add(acc_e2, e2v);
      acc_n += 1;
    }
  }
  if (ref_bits) {
    if (__syncthreads_or(flip) && threadIdx.x == 0) atomicOr(flips, 1);
  }
  if (!partials) return;
  // warp sums in double-float (fixed butterfly), then the warp sums in FP64 in warp order
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    acc_cost = f2_add(acc_cost, F2{__shfl_xor_sync(0xffffffffu, acc_cost.h, m), __shfl_xor_sync(0xffffffffu, acc_cost.l, m)});
    acc_e2 = f2_add(acc_e2, F2{__shfl_xor_sync(0xffffffffu, acc_e2.h, m), __shfl_xor_sync(0xffffffffu, acc_e2.l, m)});
    acc_n += __shfl_xor_sync(0xffffffffu, acc_n, m);
  }
  __shared__ double ws[3][kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    ws[0][warp] = f2_to_double(acc_cost);
    ws[1][warp] = f2_to_double(acc_e2);
    ws[2][warp] = (double)acc_n;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += ws[threadIdx.x][w];
    partials[3 * blockIdx.x + threadIdx.x] = t;
  }
  eval_finish(partials, sc, slot);
}

static F2 host_f2(double x) {
  const float h = (float)x;
  return F2{h, (float)(x - (double)h)};
}

cudaError_t launch_eval_df(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                           F2* camdf, float4* ptdf, bool convert, const uint8_t* act, uint8_t* bits,
                           const uint8_t* ref_bits, int* flips, double* partials, Scalars* sc, int slot, int grid,
                           cudaStream_t s) {
  const int nconv = std::max(L.C * 16, L.P);
  if (convert && nconv > 0)
    k_state_df<<<std::min((nconv + 255) / 256, 4096), 256, 0, s>>>(L.C, L.P, camw64, pts64, camdf, ptdf);
  EvalDFConst ec;
  ec.cx = host_f2(mp.cx);
  ec.cy = host_f2(mp.cy);
  ec.huber = host_f2(mp.huber > 0.0 ? mp.huber : 0.0);
  ec.huber2 = host_f2(mp.huber > 0.0 ? mp.huber * mp.huber : 0.0);
  ec.two_huber = host_f2(mp.huber > 0.0 ? 2.0 * mp.huber : 0.0);
  ec.sw_valid = host_f2(mp.sw_valid);
  ec.sw_invalid = host_f2(mp.sw_invalid);
  ec.min_depth = host_f2(mp.min_depth);
  ec.img_w = host_f2((double)mp.img_w);
  ec.img_h = host_f2((double)mp.img_h);
  ec.drop2 = host_f2(mp.drop_px > 0.0 ? mp.drop_px * mp.drop_px : 0.0);
  const size_t cam_bytes = (size_t)144 * L.C;
  const int cam_smem = cam_bytes <= 48 * 1024 ? 1 : 0;
  k_eval_df<<<grid, kBlock, cam_smem ? cam_bytes : 0, s>>>(L, mp, ec, camdf, ptdf, camw64, pts64, act, bits,
                                                          bits ? ref_bits : nullptr, flips, partials, sc, slot,
                                                          cam_smem);
  return cudaGetLastError();
}

cudaError_t launch_obs_df(int N, const double* uv64, const double* tau64, float4* uvdf, F2* taudf, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_obs_df<<<std::min((N + 255) / 256, 65535), 256, 0, s>>>(N, uv64, tau64, uvdf, taudf);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// dynamic parameter extraction (Sec. 4.2 steps 1-2)
// ---------------------------------------------------------------------------

__global__ void k_extract_begin(int N, uint8_t* __restrict__ alive, const uint8_t* __restrict__ bits,
                                uint8_t* __restrict__ valid, int drop) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    uint8_t b = bits[k];
    uint8_t a = alive[k];
    if (drop && (b & 3) == 3) a = 0;  // sticky residual drop of a valid observation
    alive[k] = a;
    valid[k] = (uint8_t)(a && (b & 1));
  }
}

cudaError_t launch_extract_begin(const Layout& L, uint8_t* alive, const uint8_t* bits,
                                 uint8_t* valid, int drop, cudaStream_t s) {
  if (L.N > 0) k_extract_begin<<<(L.N + 255) / 256, 256, 0, s>>>(L.N, alive, bits, valid, drop);
  return cudaGetLastError();
}

__global__ void k_fill_u8(uint8_t* p, uint8_t v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

cudaError_t launch_fill_u8(uint8_t* p, uint8_t v, int n, cudaStream_t s) {
  if (n > 0) k_fill_u8<<<(n + 255) / 256, 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

// One peeling round over points: a point stays active while it keeps >= min_pt
// valid observations in active cameras; the surviving observations are counted
// per camera for the camera round.
__global__ void k_peel_points(Layout L, const uint8_t* __restrict__ valid,
                              const uint8_t* __restrict__ cam_act, uint8_t* __restrict__ pt_act,
                              int* __restrict__ cam_cnt, int min_pt, Scalars* sc) {
  extern __shared__ int s_cnt[];
  bool use_smem = L.C <= 8192;
  if (use_smem) {
    for (int c = threadIdx.x; c < L.C; c += blockDim.x) s_cnt[c] = 0;
    __syncthreads();
  }
  int changed = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < L.P; p += gridDim.x * blockDim.x) {
    int k0 = L.pt_off[p], k1 = L.pt_off[p + 1];
    int cnt = 0;
    for (int k = k0; k < k1; ++k) cnt += (valid[k] && cam_act[L.po_cam[k]]) ? 1 : 0;
    uint8_t old = pt_act[p];
    uint8_t now = (uint8_t)(old && cnt >= min_pt);
    if (now != old) {
      pt_act[p] = now;
      changed = 1;
    }
    if (now)
      for (int k = k0; k < k1; ++k)
        if (valid[k] && cam_act[L.po_cam[k]]) {
          if (use_smem) atomicAdd(&s_cnt[L.po_cam[k]], 1);
          else atomicAdd(&cam_cnt[L.po_cam[k]], 1);
        }
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&sc->changed, 1);
  if (use_smem) {
    for (int c = threadIdx.x; c < L.C; c += blockDim.x)
      if (s_cnt[c]) atomicAdd(&cam_cnt[c], s_cnt[c]);
  }
}

cudaError_t launch_peel_points(const Layout& L, const uint8_t* valid, const uint8_t* cam_act,
                               uint8_t* pt_act, int* cam_cnt, int min_pt, Scalars* sc,
                               cudaStream_t s) {
  if (L.P == 0) return cudaSuccess;
  size_t smem = L.C <= 8192 ? sizeof(int) * (size_t)L.C : 0;
  int grid = (L.P + 255) / 256;
  if (grid > 2048) grid = 2048;
  k_peel_points<<<grid, 256, smem, s>>>(L, valid, cam_act, pt_act, cam_cnt, min_pt, sc);
  return cudaGetLastError();
}

__global__ void k_peel_cams(int C, const uint8_t* __restrict__ fixed, uint8_t* __restrict__ cam_act,
                            int* __restrict__ cam_cnt, int min_cam, Scalars* sc) {
  int changed = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    uint8_t old = cam_act[c];
    uint8_t now = (uint8_t)(fixed[c] || (old && cam_cnt[c] >= min_cam));
    if (now != old) {
      cam_act[c] = now;
      changed = 1;
    }
    cam_cnt[c] = 0;
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&sc->changed, 1);
}

cudaError_t launch_peel_cams(const Layout& L, uint8_t* cam_act, int* cam_cnt, int min_cam,
                             Scalars* sc, cudaStream_t s) {
  if (L.C > 0) k_peel_cams<<<(L.C + 255) / 256, 256, 0, s>>>(L.C, L.cam_fixed, cam_act, cam_cnt, min_cam, sc);
  return cudaGetLastError();
}

__global__ void k_finalize_obs(Layout L, const uint8_t* __restrict__ valid,
                               const uint8_t* __restrict__ cam_act, const uint8_t* __restrict__ pt_act,
                               uint8_t* __restrict__ obs_act, Scalars* sc) {
  int cnt = 0, changed = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += gridDim.x * blockDim.x) {
    uint8_t a = (uint8_t)(valid[k] && cam_act[L.po_cam[k]] && pt_act[L.po_pt[k]]);
    if (a != obs_act[k]) changed = 1;
    obs_act[k] = a;
    cnt += a;
  }
  __shared__ int red[32];
  int tot = block_sum(cnt, red);
  if (threadIdx.x == 0 && tot) atomicAdd(&sc->n_obs_act, tot);
  if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&sc->mask_changed, 1);
}

__global__ void k_gather_co(int N, const int* __restrict__ co_po, const uint8_t* __restrict__ obs_act,
                            uint8_t* __restrict__ obs_act_co) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
    obs_act_co[j] = obs_act[co_po[j]];
}

cudaError_t launch_finalize_obs(const Layout& L, const uint8_t* valid, const uint8_t* cam_act,
                                const uint8_t* pt_act, uint8_t* obs_act, uint8_t* obs_act_co,
                                Scalars* sc, cudaStream_t s) {
  if (L.N == 0) return cudaSuccess;
  int grid = (L.N + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_finalize_obs<<<grid, 256, 0, s>>>(L, valid, cam_act, pt_act, obs_act, sc);
  k_gather_co<<<grid, 256, 0, s>>>(L.N, L.co_po, obs_act, obs_act_co);
  return cudaGetLastError();
}

// free-camera flags (active and not gauge) and the number of active cameras
// (sc->n_cam_act, zeroed by the caller; integer atomics, order-free)
__global__ void k_cam_flags(int C, const uint8_t* __restrict__ fixed, const uint8_t* __restrict__ cam_act,
                            uint8_t* __restrict__ flags, Scalars* sc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int act = 0;
  if (c < C) {
    act = cam_act[c] ? 1 : 0;
    flags[c] = (uint8_t)(act && !fixed[c]);
  }
  act = warp_sum(act);
  if ((threadIdx.x & 31) == 0 && act) atomicAdd(&sc->n_cam_act, act);
}

cudaError_t launch_cam_flags(const Layout& L, const uint8_t* cam_act, uint8_t* flags, Scalars* sc, cudaStream_t s) {
  if (L.C > 0) k_cam_flags<<<(L.C + 255) / 256, 256, 0, s>>>(L.C, L.cam_fixed, cam_act, flags, sc);
  return cudaGetLastError();
}

// Exclusive scan of 0/1 flags into ascending ranks (Eq. rank): three passes,
// block counts -> scan of block counts -> local scan plus block offset.
constexpr int kScanItems = 8;
constexpr int kScanThreads = 256;
constexpr int kScanTile = kScanItems * kScanThreads;

int rank_blocks(int n) { return (n + kScanTile - 1) / kScanTile; }

__device__ int block_excl_scan(int v, int* sh /* >= 33 */, int* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int w = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  int base = wid > 0 ? sh[wid - 1] : 0;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void k_scan_count(const uint8_t* __restrict__ flags, int n, int* __restrict__ bsum) {
  __shared__ int red[32];
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int c = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) c += flags[base + i] ? 1 : 0;
  int t = block_sum(c, red);
  if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

__global__ void k_scan_blocks(int* __restrict__ bsum, int nb, int* __restrict__ count) {
  __shared__ int sh[33];
  int per = (nb + blockDim.x - 1) / blockDim.x;
  int beg = threadIdx.x * per;
  int s = 0;
  for (int i = 0; i < per; ++i)
    if (beg + i < nb) s += bsum[beg + i];
  int total;
  int off = block_excl_scan(s, sh, &total);
  for (int i = 0; i < per; ++i)
    if (beg + i < nb) {
      int v = bsum[beg + i];
      bsum[beg + i] = off;
      off += v;
    }
  if (threadIdx.x == 0) *count = total;
}

__global__ void k_scan_apply(const uint8_t* __restrict__ flags, int n, const int* __restrict__ boff,
                             int* __restrict__ rank, int* __restrict__ map) {
  __shared__ int sh[33];
  int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int c = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) c += flags[base + i] ? 1 : 0;
  int off = block_excl_scan(c, sh, nullptr) + boff[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    int j = base + i;
    if (j >= n) break;
    if (flags[j]) {
      rank[j] = off;
      if (map) map[off] = j;
      ++off;
    } else {
      rank[j] = -1;
    }
  }
}

cudaError_t launch_rank(const uint8_t* flags, int n, int* rank, int* map, int* count,
                        int* block_tmp, int n_block_tmp, cudaStream_t s) {
  int nb = rank_blocks(n);
  if (nb > n_block_tmp) return cudaErrorInvalidValue;
  if (n == 0) return cudaMemsetAsync(count, 0, sizeof(int), s);
  k_scan_count<<<nb, kScanThreads, 0, s>>>(flags, n, block_tmp);
  k_scan_blocks<<<1, 1024, 0, s>>>(block_tmp, nb, count);
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(flags, n, block_tmp, rank, map);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// steps (a)+(b), point side: W_k, V_p, g_p over tiles of whole points
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void load_cam(const T* __restrict__ camw, int c, T cw[kCamStride]) {
  using V4 = typename Vec4<T>::type;
  const V4* src = reinterpret_cast<const V4*>(camw + kCamStride * (size_t)c);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    V4 v = src[i];
    cw[4 * i] = v.x;
    cw[4 * i + 1] = v.y;
    cw[4 * i + 2] = v.z;
    cw[4 * i + 3] = v.w;
  }
}

template <typename T>
__device__ __forceinline__ void load_pt(const T* __restrict__ ptsw, int p, T& x, T& y, T& z) {
  using V4 = typename Vec4<T>::type;
  V4 v = reinterpret_cast<const V4*>(ptsw)[p];
  x = v.x;
  y = v.y;
  z = v.z;
}

// one 32-byte store (32-byte aligned address)
__device__ __forceinline__ void st_v8(float* p, float a, float b, float c, float d, float e, float f, float g,
                                      float h) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d), "f"(e), "f"(f), "f"(g), "f"(h)
               : "memory");
}

// W: stored W rows (nullptr when the matvec recomputes the Jacobian); wsgn: per
// observation IRLS weight rho', negated when the observation has no depth prior
// (0 for inactive observations), in the padded per-tile layout (nullptr if unused).
// orec (nullable, FP32): the observation's record [16] for the explicit system's
// formation and back-substitution: w D^T D (G00 G01 G02 G11 G12 G22), w D^T e
// (u0 u1 u2) with e = (xn, yn, 0), the intrinsic factor g = (dist, f rr, f rr^2)
// ((dist, 0, 0) for the centre model), the point the rotation increment acts on
// (a0 a1 a2), one zero; all zero when inactive (D = d r / d P, w the IRLS weight,
// rr = xn^2 + yn^2; model.cuh)
template <typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 4 : 2) k_pt_lin(Layout L, ModelParams mp, const T* __restrict__ camw,
                                                   const T* __restrict__ ptsw,
                                                   const uint8_t* __restrict__ obs_act, T* __restrict__ W,
                                                   T* __restrict__ wsgn, T* __restrict__ V,
                                                   T* __restrict__ gp, float* __restrict__ orec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);  // [kTileObs][kWStride]
  T* Vs = Ws + kTileObs * kWStride;        // [kTileObs][9]
  const TileDesc d = L.descs[blockIdx.x];
  int ob = d.obs_begin, n = d.n_obs;
  int pb = d.pt_begin, pe = d.pt_begin + d.n_pts;
  const T* uvw = reinterpret_cast<const T*>(L.po_uvw);
  const T* tauw = reinterpret_cast<const T*>(L.po_tauw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int k = ob + i;
    T* wrow = Ws + kWStride * i;
    T* vrow = Vs + 9 * i;
    if (!obs_act[k]) {
#pragma unroll
      for (int j = 0; j < kWStride; ++j) wrow[j] = T(0);
#pragma unroll
      for (int j = 0; j < 9; ++j) vrow[j] = T(0);
      if (wsgn) wsgn[(size_t)d.g_row + i] = T(0);
      if (sizeof(T) == 4 && orec) {
        st_v8(orec + 16 * (size_t)k, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        st_v8(orec + 16 * (size_t)k + 8, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    T cw[kCamStride];
    load_cam(camw, bidx(L.po_cam[k], L.C, 4), cw);
    T X0, X1, X2;
    load_pt(ptsw, bidx(L.po_pt[k], L.P, 5), X0, X1, X2);
    T tau = tauw[k];
    T sw = tau > T(0) ? (T)mp.sw_valid : (T)mp.sw_invalid;
    ObsLin<T> o;
    linearize_obs<T>(cw, X0, X1, X2, uvw[2 * (size_t)k], uvw[2 * (size_t)k + 1], tau, sw, (T)mp.cx,
                     (T)mp.cy, (T)mp.huber, o);
    T w = o.wrob;
    if (wsgn) wsgn[(size_t)d.g_row + i] = tau > T(0) ? w : -w;
    if (W) {
      // the row in registers, then stored as 16-byte words (the 28-word row
      // stride puts the 8 lanes of a quarter-warp on distinct bank groups)
      using V4 = typename Vec4<T>::type;
      T wr[kWStride];
#pragma unroll
      for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          wr[3 * a + b] = w * (o.Jc[0][a] * o.Jp[0][b] + o.Jc[1][a] * o.Jp[1][b] + o.Jc[2][a] * o.Jp[2][b]);
      wr[27] = T(0);
      V4* w4 = reinterpret_cast<V4*>(wrow);
#pragma unroll
      for (int q = 0; q < kWStride / 4; ++q) {
        V4 v;
        v.x = wr[4 * q], v.y = wr[4 * q + 1], v.z = wr[4 * q + 2], v.w = wr[4 * q + 3];
        w4[q] = v;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = a; b < 3; ++b)
        vrow[sym3(a, b)] = w * (o.Jp[0][a] * o.Jp[0][b] + o.Jp[1][a] * o.Jp[1][b] + o.Jp[2][a] * o.Jp[2][b]);
      vrow[6 + a] = w * (o.Jp[0][a] * o.r[0] + o.Jp[1][a] * o.r[1] + o.Jp[2][a] * o.r[2]);
    }
    if (sizeof(T) == 4 && orec) {  // FP32 problems only
      // columns of D: (D00, D01, 0), (D01, D11, 0), (D02, D12, D22)
      const float d00 = (float)o.D00, d01 = (float)o.D01, d02 = (float)o.D02, d11 = (float)o.D11,
                  d12 = (float)o.D12, d22 = (float)o.D22, xn = (float)o.xn, yn = (float)o.yn, wf = (float)w;
      const float rr = xn * xn + yn * yn, f = (float)cw[12];
      const float dist = 1.f + rr * ((float)cw[13] + (float)cw[14] * rr);
      const bool centre = cw[15] != T(0);
      float* rk = orec + 16 * (size_t)k;
      st_v8(rk, wf * (d00 * d00 + d01 * d01), wf * (d00 * d01 + d01 * d11), wf * (d00 * d02 + d01 * d12),
            wf * (d01 * d01 + d11 * d11), wf * (d01 * d02 + d11 * d12), wf * (d02 * d02 + d12 * d12 + d22 * d22),
            wf * (d00 * xn + d01 * yn), wf * (d01 * xn + d11 * yn));
      st_v8(rk + 8, wf * (d02 * xn + d12 * yn), dist, centre ? 0.f : f * rr, centre ? 0.f : f * rr * rr,
            (float)o.a0, (float)o.a1, (float)o.a2, 0.f);
    }
  }
  __syncthreads();
  if (W) {
    // 16-byte coalesced copy of the tile's rows (rows are 16-byte aligned)
    using V4 = typename Vec4<T>::type;
    V4* Wdst = reinterpret_cast<V4*>(W + kWStride * (size_t)d.w_row);
    const V4* Wsrc = reinterpret_cast<const V4*>(Ws);
    for (int j = threadIdx.x; j < (kWStride / 4) * n; j += blockDim.x) Wdst[j] = Wsrc[j];
  }
  // nine threads per point, one per entry of (V, g_p), each summing the point's
  // observations in order
  for (int t = threadIdx.x; t < 9 * (pe - pb); t += blockDim.x) {
    const int p = pb + t / 9, j = t - 9 * (t / 9);
    T acc = T(0);
    for (int k = L.pt_off[p]; k < L.pt_off[p + 1]; ++k) acc += Vs[9 * (k - ob) + j];
    if (j < 6) V[6 * (size_t)p + j] = acc;
    else gp[3 * (size_t)p + j - 6] = acc;
  }
}

template <typename T>
cudaError_t launch_pt_lin(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                          const uint8_t* obs_act, T* W, T* wsgn, T* V, T* gp, cudaStream_t s, float* orec) {
  if (L.n_tiles == 0) return cudaSuccess;
  size_t smem = sizeof(T) * kTileObs * (kWStride + 9);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_pt_lin<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_pt_lin<T><<<L.n_tiles, kBlock, smem, s>>>(L, mp, camw, ptsw, obs_act, W, wsgn, V, gp, orec);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// steps (a)+(b), camera side: per-chunk sums over one camera's observations.
// mode 0: U_i (45 packed) and g_c (9).
// mode 1: Schur terms sum_k W_k V*^-1 W_k^T (45) and sum_k W_k V*^-1 g_p (9), using
//         W_k V^-1 W_k^T = w^2 Jc^T (Jp V^-1 Jp^T) Jc.
// ---------------------------------------------------------------------------

constexpr int kCamThreads = 128;

template <typename T, int MODE>
__global__ void __launch_bounds__(kCamThreads) k_cam_accum(
    Layout L, ModelParams mp, const T* __restrict__ camw, const T* __restrict__ ptsw,
    const uint8_t* __restrict__ act_co, const uint8_t* __restrict__ cam_act,
    const int* __restrict__ crank, const T* __restrict__ Vinv, const T* __restrict__ z0,
    T* __restrict__ partials) {
  __shared__ T red[kCamThreads / 32][54];
  __shared__ T s_cw[kCamStride];
  int q = blockIdx.x;
  int c = L.chunk_cam[q];
  int kb = L.chunk_obs[q], ke = L.chunk_obs[q + 1];
  bool live = MODE == 0 ? (cam_act[c] != 0) : (crank[c] >= 0);
  T* out = partials + 54 * (size_t)q;
  if (!live) {
    for (int j = threadIdx.x; j < 54; j += blockDim.x) out[j] = T(0);
    return;
  }
  if (threadIdx.x < kCamStride) s_cw[threadIdx.x] = camw[kCamStride * (size_t)c + threadIdx.x];
  __syncthreads();
  T cw[kCamStride];
#pragma unroll
  for (int i = 0; i < kCamStride; ++i) cw[i] = s_cw[i];
  const T* uvw = reinterpret_cast<const T*>(L.co_uvw);
  const T* tauw = reinterpret_cast<const T*>(L.co_tauw);
  T acc[54];
#pragma unroll
  for (int j = 0; j < 54; ++j) acc[j] = T(0);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    if (!act_co[k]) continue;
    int p = bidx(L.co_pt[k], L.P, 6);
    T X0, X1, X2;
    load_pt(ptsw, p, X0, X1, X2);
    T tau = tauw[k];
    T sw = tau > T(0) ? (T)mp.sw_valid : (T)mp.sw_invalid;
    ObsLin<T> o;
    linearize_obs<T>(cw, X0, X1, X2, uvw[2 * (size_t)k], uvw[2 * (size_t)k + 1], tau, sw, (T)mp.cx,
                     (T)mp.cy, (T)mp.huber, o);
    T w = o.wrob;
    if (MODE == 0) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
#pragma unroll
        for (int b = a; b < 9; ++b)
          acc[sym9(a, b)] += w * (o.Jc[0][a] * o.Jc[0][b] + o.Jc[1][a] * o.Jc[1][b] + o.Jc[2][a] * o.Jc[2][b]);
        acc[45 + a] += w * (o.Jc[0][a] * o.r[0] + o.Jc[1][a] * o.r[1] + o.Jc[2][a] * o.r[2]);
      }
    } else {
      const T* vi = Vinv + 6 * (size_t)p;
      T Vi[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Vi[a][b] = vi[sym3(a, b)];
      // A = Jp V^-1 (3x3), Q = A Jp^T (3x3 symmetric)
      T A[3][3], Q[3][3];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          A[m][b] = o.Jp[m][0] * Vi[0][b] + o.Jp[m][1] * Vi[1][b] + o.Jp[m][2] * Vi[2][b];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          Q[m][l] = w * w * (A[m][0] * o.Jp[l][0] + A[m][1] * o.Jp[l][1] + A[m][2] * o.Jp[l][2]);
      // M = Q Jc (3x9); acc += Jc^T M
      T M[3][9];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int b = 0; b < 9; ++b) M[m][b] = Q[m][0] * o.Jc[0][b] + Q[m][1] * o.Jc[1][b] + Q[m][2] * o.Jc[2][b];
#pragma unroll
      for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = a; b < 9; ++b)
          acc[sym9(a, b)] += o.Jc[0][a] * M[0][b] + o.Jc[1][a] * M[1][b] + o.Jc[2][a] * M[2][b];
      // W z0 = w Jc^T (Jp z0)
      const T* zp = z0 + 3 * (size_t)p;
      T jz[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) jz[m] = w * (o.Jp[m][0] * zp[0] + o.Jp[m][1] * zp[1] + o.Jp[m][2] * zp[2]);
#pragma unroll
      for (int a = 0; a < 9; ++a) acc[45 + a] += o.Jc[0][a] * jz[0] + o.Jc[1][a] * jz[1] + o.Jc[2][a] * jz[2];
    }
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // warp reduce-scatter of the 54 sums (padded to 64): each round a lane keeps
  // half of its entries and adds its partner's copy of them (62 shuffles instead
  // of 54 x 5); lane L ends with entries 32 b0 + 16 b1 + 8 b2 + 4 b3 + 2 b4 + (0, 1)
  {
    T v[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) v[j] = j < 54 ? acc[j] : T(0);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int H = 32 >> r;
      const bool hi = (lane >> r) & 1;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (i < H) {
          const T send = hi ? v[i] : v[H + i];
          const T keep = hi ? v[H + i] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << r);
        }
      }
    }
    const int base = 32 * (lane & 1) + 16 * ((lane >> 1) & 1) + 8 * ((lane >> 2) & 1) + 4 * ((lane >> 3) & 1) +
                     2 * ((lane >> 4) & 1);
#pragma unroll
    for (int t = 0; t < 2; ++t)
      if (base + t < 54) red[wid][base + t] = v[t];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < 54; j += blockDim.x) {
    T s = T(0);
    for (int w = 0; w < kCamThreads / 32; ++w) s += red[w][j];
    out[j] = s;
  }
}

template <typename T>
cudaError_t launch_cam_accum(const Layout& L, const ModelParams& mp, int mode, const T* camw,
                             const T* ptsw, const uint8_t* act_co, const uint8_t* cam_act,
                             const int* crank, const T* Vinv, const T* z0, T* partials,
                             cudaStream_t s) {
  if (L.n_chunks == 0) return cudaSuccess;
  if (mode == 0)
    k_cam_accum<T, 0><<<L.n_chunks, kCamThreads, 0, s>>>(L, mp, camw, ptsw, act_co, cam_act, crank,
                                                         Vinv, z0, partials);
  else
    k_cam_accum<T, 1><<<L.n_chunks, kCamThreads, 0, s>>>(L, mp, camw, ptsw, act_co, cam_act, crank,
                                                         Vinv, z0, partials);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_cam_reduce(int C, const int* __restrict__ cam_chunk, const T* __restrict__ partials,
                             T* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * 54) return;
  int c = i / 54, j = i - 54 * c;
  double s = 0.0;
  for (int q = cam_chunk[c]; q < cam_chunk[c + 1]; ++q) s += (double)partials[54 * (size_t)q + j];
  out[i] = (T)s;
}

template <typename T>
cudaError_t launch_cam_reduce(const Layout& L, const T* partials, T* out, cudaStream_t s) {
  int n = L.C * 54;
  if (n > 0) k_cam_reduce<T><<<(n + 255) / 256, 256, 0, s>>>(L.C, L.cam_chunk, partials, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// damping (Eq. LM, Marquardt scaling with the clamped diagonal)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double clamp_diag(double a) { return fmin(fmax(a, 1e-6), 1e32); }

template <typename T>
__global__ void k_damp_pts(int P, const T* __restrict__ V, const T* __restrict__ gp,
                           const uint8_t* __restrict__ pt_act, double lambda, T* __restrict__ Vinv,
                           T* __restrict__ z0, int* err) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  T* vo = Vinv + 6 * (size_t)p;
  T* zo = z0 + 3 * (size_t)p;
  if (!pt_act[p]) {
    for (int j = 0; j < 6; ++j) vo[j] = T(0);
    for (int j = 0; j < 3; ++j) zo[j] = T(0);
    return;
  }
  const T* v = V + 6 * (size_t)p;
  double a = v[0], b = v[1], c = v[2], d = v[3], e = v[4], f = v[5];  // [[a b c][b d e][c e f]]
  a += lambda * clamp_diag(a);
  d += lambda * clamp_diag(d);
  f += lambda * clamp_diag(f);
  // adjugate of the symmetric matrix
  double A = d * f - e * e, B = c * e - b * f, Cc = b * e - c * d;
  double det = a * A + b * B + c * Cc;
  if (!(det > 0.0) || !isfinite(det)) {
    atomicOr(err, 4);
    for (int j = 0; j < 6; ++j) vo[j] = T(0);
    for (int j = 0; j < 3; ++j) zo[j] = T(0);
    return;
  }
  double id = recip_nr(det);
  double i00 = A * id, i01 = B * id, i02 = Cc * id;
  double i11 = (a * f - c * c) * id, i12 = (b * c - a * e) * id, i22 = (a * d - b * b) * id;
  vo[0] = (T)i00; vo[1] = (T)i01; vo[2] = (T)i02; vo[3] = (T)i11; vo[4] = (T)i12; vo[5] = (T)i22;
  double g0 = gp[3 * (size_t)p], g1 = gp[3 * (size_t)p + 1], g2 = gp[3 * (size_t)p + 2];
  zo[0] = (T)(i00 * g0 + i01 * g1 + i02 * g2);
  zo[1] = (T)(i01 * g0 + i11 * g1 + i12 * g2);
  zo[2] = (T)(i02 * g0 + i12 * g1 + i22 * g2);
}

// FP32 problems: the same damped inverse in double-float arithmetic (about 48
// significant bits, on the FP32 pipe instead of the narrow FP64 one); the results
// are rounded to FP32 as before.  The clamp and the determinant's sign test are
// taken on the leading FP32 word, which carries the sign and magnitude.
__device__ __forceinline__ F2 f2_of(float x) { return F2{x, 0.f}; }
__device__ __forceinline__ float f2_round(F2 a) { return __fadd_rn(a.h, a.l); }

// prec (nullable): the point record [8] of the explicit system's formation from
// observation records: V*^-1 (6, as in Vinv), two zeros
__global__ void k_damp_pts_df(int P, const float* __restrict__ V, const float* __restrict__ gp,
                              const uint8_t* __restrict__ pt_act, F2 lambda, float* __restrict__ Vinv,
                              float* __restrict__ z0, int* err, float* __restrict__ prec) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float* vo = Vinv + 6 * (size_t)p;
  float* zo = z0 + 3 * (size_t)p;
  auto point_record = [&]() {
    if (!prec) return;
    float4* r4 = reinterpret_cast<float4*>(prec) + 2 * (size_t)p;
    r4[0] = make_float4(vo[0], vo[1], vo[2], vo[3]);
    r4[1] = make_float4(vo[4], vo[5], 0.f, 0.f);
  };
  if (!pt_act[p]) {
    for (int j = 0; j < 6; ++j) vo[j] = 0.f;
    for (int j = 0; j < 3; ++j) zo[j] = 0.f;
    point_record();
    return;
  }
  const float* v = V + 6 * (size_t)p;
  const float v0 = v[0], v3 = v[3], v5 = v[5];
  const F2 b = f2_of(v[1]), c = f2_of(v[2]), e = f2_of(v[4]);
  auto damp = [&](float x) { return f2_add(f2_of(x), f2_mul(lambda, f2_of(fminf(fmaxf(x, 1e-6f), 1e32f)))); };
  const F2 a = damp(v0), d = damp(v3), f = damp(v5);
  // adjugate of the symmetric matrix
  const F2 A = f2_sub(f2_mul(d, f), f2_mul(e, e)), B = f2_sub(f2_mul(c, e), f2_mul(b, f)),
           Cc = f2_sub(f2_mul(b, e), f2_mul(c, d));
  const F2 det = f2_add(f2_add(f2_mul(a, A), f2_mul(b, B)), f2_mul(c, Cc));
  if (!(det.h > 0.f) || !f2_finite(det)) {
    atomicOr(err, 4);
    for (int j = 0; j < 6; ++j) vo[j] = 0.f;
    for (int j = 0; j < 3; ++j) zo[j] = 0.f;
    point_record();
    return;
  }
  const F2 id = f2_recip(det);
  const F2 i00 = f2_mul(A, id), i01 = f2_mul(B, id), i02 = f2_mul(Cc, id);
  const F2 i11 = f2_mul(f2_sub(f2_mul(a, f), f2_mul(c, c)), id);
  const F2 i12 = f2_mul(f2_sub(f2_mul(b, c), f2_mul(a, e)), id);
  const F2 i22 = f2_mul(f2_sub(f2_mul(a, d), f2_mul(b, b)), id);
  vo[0] = f2_round(i00); vo[1] = f2_round(i01); vo[2] = f2_round(i02);
  vo[3] = f2_round(i11); vo[4] = f2_round(i12); vo[5] = f2_round(i22);
  const F2 g0 = f2_of(gp[3 * (size_t)p]), g1 = f2_of(gp[3 * (size_t)p + 1]), g2 = f2_of(gp[3 * (size_t)p + 2]);
  zo[0] = f2_round(f2_add(f2_add(f2_mul(i00, g0), f2_mul(i01, g1)), f2_mul(i02, g2)));
  zo[1] = f2_round(f2_add(f2_add(f2_mul(i01, g0), f2_mul(i11, g1)), f2_mul(i12, g2)));
  zo[2] = f2_round(f2_add(f2_add(f2_mul(i02, g0), f2_mul(i12, g1)), f2_mul(i22, g2)));
  point_record();
}

template <typename T>
cudaError_t launch_damp_pts(int P, const T* V, const T* gp, const uint8_t* pt_act, double lambda,
                            T* Vinv, T* z0, int* err, cudaStream_t s, float* prec) {
  if (P <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    const float lh = (float)lambda;
    const F2 lam{lh, (float)(lambda - (double)lh)};
    k_damp_pts_df<<<(P + 255) / 256, 256, 0, s>>>(P, V, gp, pt_act, lam, Vinv, z0, err, prec);
  } else
    k_damp_pts<T><<<(P + 255) / 256, 256, 0, s>>>(P, V, gp, pt_act, lambda, Vinv, z0, err);
  return cudaGetLastError();
}

// Per free camera f (one warp each): damped U block, block-Jacobi inverse of the
// Schur diagonal D_f = U*_f - sum W V*^-1 W^T (FP64 Cholesky in shared memory
// across the warp, the 9 inverse columns solved by 9 lanes with the reciprocal
// pivots), Schur RHS b_f = -g_c + sum W V*^-1 g_p.
constexpr int kDiagWarps = 4;

template <typename T>
__global__ void k_schur_diag(int Cf, const int* __restrict__ cam_map, const T* __restrict__ Ug,
                             const T* __restrict__ Sg, double lambda, T* __restrict__ Ud,
                             T* __restrict__ Dinv, T* __restrict__ b, T* __restrict__ dampc,
                             T* __restrict__ Dblk, double* __restrict__ dscale, int* err, int kfix) {
  // kfix (camera model of Sec. 3.2): slots 7 and 8 are not parameters; U holds
  // them with a unit diagonal (zero Jacobian columns and gradient entries), which
  // decouples them and keeps the undamped adjoint system nonsingular.
  // D = U* - W V*^-1 W^T, its Cholesky factor and its inverse in FP64 (the two
  // terms can nearly cancel; an FP32 factorisation measurably weakens the
  // preconditioner of the undamped adjoint system)
  using A = double;
  __shared__ A Ds[kDiagWarps][81];
  __shared__ A Rs[kDiagWarps][9];  // reciprocal pivots 1 / L_jj
  __shared__ int okS[kDiagWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kDiagWarps + w;
  if (f >= Cf) return;
  const int c = cam_map[f];
  const T* u = Ug + 54 * (size_t)c;
  const T* sch = Sg + 54 * (size_t)c;
  A* D = Ds[w];
  for (int q = lane; q < 81; q += 32) {
    int i = q / 9, j = q - 9 * i;
    double uij = (kfix && (i >= 7 || j >= 7)) ? (i == j ? 1.0 : 0.0) : (double)u[sym9(i, j)];
    if (i == j) {
      double dc = clamp_diag(uij);
      dampc[9 * (size_t)f + i] = (T)dc;
      uij += lambda * dc;
    }
    double v = uij - (double)sch[sym9(i, j)];
    D[q] = (A)v;
    if (j >= i) {
      Ud[45 * (size_t)f + sym9(i, j)] = (T)uij;
      if (Dblk) Dblk[45 * (size_t)f + sym9(i, j)] = (T)v;
    }
    if (dscale && i == j) {
      // Jacobi scaling of the explicit system: D = sqrt(diag U*), then 1/D in T
      const double d = (double)(T)uij;
      const double sd = sqrt(d > 0.0 ? d : 1e-30);
      dscale[9 * (size_t)f + i] = sd;
      reinterpret_cast<T*>(dscale + 9 * (size_t)Cf)[9 * (size_t)f + i] = (T)(1.0 / sd);
    }
  }
  if (lane < 9) b[9 * (size_t)f + lane] = (T)(-(double)u[45 + lane] + (double)sch[45 + lane]);
  __syncwarp();
  // Cholesky D = L L^T in place (lower), right-looking across the warp: lane 0
  // takes pivot j (reciprocal square root), the lanes below scale column j, and
  // the lanes update the trailing lower triangle (one entry each)
  A* Rp = Rs[w];
  for (int j = 0; j < 9; ++j) {
    if (lane == 0) {
      const A sj = D[9 * j + j];
      const int good = sj > A(0);  // false for NaN
      const A r = good ? rsqrt(sj) : A(0);
      D[9 * j + j] = sj * r;
      Rp[j] = r;
      okS[w] = good;
    }
    __syncwarp();
    if (!okS[w]) break;
    if (lane > j && lane < 9) D[9 * lane + j] *= Rp[j];
    __syncwarp();
    const int m = 8 - j;  // trailing block rows j+1 .. 8
    for (int q = lane; q < m * (m + 1) / 2; q += 32) {
      int i0 = 0, k0 = q;
      while (k0 > i0) k0 -= ++i0;  // q -> (i0, k0), k0 <= i0, row-major lower triangle
      const int i = j + 1 + i0, k = j + 1 + k0;
      D[9 * i + k] -= D[9 * i + j] * D[9 * k + j];
    }
    __syncwarp();
  }
  __syncwarp();
  T* out = Dinv + 81 * (size_t)f;
  if (!okS[w]) {
    // fall back to the Jacobi diagonal of the damped U block
    if (lane == 0) atomicOr(err, 8);
    for (int q = lane; q < 81; q += 32) {
      int i = q / 9, j = q - 9 * i;
      out[q] = i == j ? (T)(1.0 / (double)Ud[45 * (size_t)f + sym9(i, i)]) : T(0);
    }
    return;
  }
  if (lane < 9) {
    // column `lane` of the inverse: solve L L^T x = e_lane
    const int j = lane;
    A x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      A s = i == j ? A(1) : A(0);
#pragma unroll
      for (int l = 0; l < i; ++l) s -= D[9 * i + l] * x[l];
      x[i] = s * Rp[i];
    }
#pragma unroll
    for (int i = 8; i >= 0; --i) {
      A s = x[i];
#pragma unroll
      for (int l = i + 1; l < 9; ++l) s -= D[9 * l + i] * x[l];
      x[i] = s * Rp[i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) out[9 * i + j] = (T)x[i];
  }
}

template <typename T>
cudaError_t launch_schur_diag(int Cf, const int* cam_map, const T* Ug, const T* Sg, double lambda,
                              T* Ud, T* Dinv, T* b, T* dampc, T* Dblk, double* dscale, int* err, cudaStream_t s,
                              int kfix) {
  if (Cf > 0)
    k_schur_diag<T><<<(Cf + kDiagWarps - 1) / kDiagWarps, 32 * kDiagWarps, 0, s>>>(Cf, cam_map, Ug, Sg, lambda, Ud,
                                                                                    Dinv, b, dampc, Dblk, dscale,
                                                                                    err, kfix);
  return cudaGetLastError();
}

// predicted decrease, camera part: 1/2 dx^T (lambda D dx - g) over the free cameras
template <typename T>
__global__ void k_pred_cams(int Cf, const int* __restrict__ cam_map, const T* __restrict__ x,
                            const T* __restrict__ Ug, const T* __restrict__ dampc, double lambda,
                            double* __restrict__ pred_parts) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 9 * Cf; e += gridDim.x * blockDim.x) {
    int f = e / 9, i = e - 9 * f;
    int c = cam_map[f];
    double d = (double)x[e];
    acc += d * (lambda * (double)dampc[e] * d - (double)Ug[54 * (size_t)c + 45 + i]);
  }
  double s = block_sum(acc, red);
  if (threadIdx.x == 0) pred_parts[blockIdx.x] = s;
}

template <typename T>
cudaError_t launch_pred_cams(int Cf, const int* cam_map, const T* x, const T* Ug, const T* dampc,
                             double lambda, double* pred_parts, int offset, cudaStream_t s) {
  k_pred_cams<T><<<1, 256, 0, s>>>(Cf, cam_map, x, Ug, dampc, lambda, pred_parts + offset);
  return cudaGetLastError();
}

__global__ void k_reduce_pred(const double* __restrict__ parts, int n, Scalars* sc) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += parts[i];
  a = block_sum(a, red);
  if (threadIdx.x == 0) sc->pred = 0.5 * a;
}

cudaError_t launch_reduce_pred(const double* parts, int n, Scalars* sc, cudaStream_t s) {
  k_reduce_pred<<<1, 256, 0, s>>>(parts, n, sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// step (e) candidate x (+) dx and scatter of the compact camera step (Sec. 4.2 step 3)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_candidate_cams(int C, const int* __restrict__ crank, const T* __restrict__ x,
                                 const double* __restrict__ src, double* __restrict__ dst,
                                 double* __restrict__ camw64, T* __restrict__ camw, F2* __restrict__ camdf,
                                 int model) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double* s = src + 9 * (size_t)c;
  double o[9];
  int r = crank[c];
  if (r >= 0) {
    const T* d = x + 9 * (size_t)r;
    double dw[3] = {(double)d[0], (double)d[1], (double)d[2]};
    double w[3] = {s[0], s[1], s[2]};
    rotvec_left_compose(dw, w, o);
    for (int i = 3; i < 9; ++i) o[i] = s[i] + (double)d[i];
  } else {
    for (int i = 0; i < 9; ++i) o[i] = s[i];
  }
  for (int i = 0; i < 9; ++i) dst[9 * (size_t)c + i] = o[i];
  double rec[kCamStride];
  cam_record(o, model, rec);
  for (int i = 0; i < kCamStride; ++i) camw64[kCamStride * (size_t)c + i] = rec[i];
  if (camw)
    for (int i = 0; i < kCamStride; ++i) camw[kCamStride * (size_t)c + i] = (T)rec[i];
  if (camdf)  // the double-float copy the FP32 problems' evaluation reads
    for (int i = 0; i < 16; ++i) camdf[16 * (size_t)c + i] = i < 15 ? f2_from_double(rec[i]) : F2{0.f, 0.f};
}

template <typename T>
__global__ void k_candidate_pts(int P, const T* __restrict__ dp, const double* __restrict__ src,
                                double* __restrict__ dst, T* __restrict__ ptsw, float4* __restrict__ ptdf) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double v[3];
  for (int i = 0; i < 3; ++i) {
    v[i] = src[3 * (size_t)p + i] + (double)dp[3 * (size_t)p + i];
    dst[3 * (size_t)p + i] = v[i];
  }
  using V4 = typename Vec4<T>::type;
  V4 q;
  q.x = (T)v[0];
  q.y = (T)v[1];
  q.z = (T)v[2];
  q.w = T(0);
  reinterpret_cast<V4*>(ptsw)[p] = q;
  if (ptdf) {
    const F2 x0 = f2_from_double(v[0]), x1 = f2_from_double(v[1]), x2 = f2_from_double(v[2]);
    ptdf[2 * (size_t)p] = make_float4(x0.h, x0.l, x1.h, x1.l);
    ptdf[2 * (size_t)p + 1] = make_float4(x2.h, x2.l, 0.f, 0.f);
  }
}

template <typename T>
cudaError_t launch_candidate(int C, int P, const int* crank, const T* x, const T* dp,
                             const double* cams_src, const double* pts_src, double* cams_dst,
                             double* pts_dst, double* camw64_dst, T* camw_dst, T* ptsw_dst,
                             F2* camdf_dst, float4* ptdf_dst, cudaStream_t s, int model) {
  // 32-thread blocks: the FP64 rotation work (sincos, atan2) of 32 cameras per SM
  if (C > 0)
    k_candidate_cams<T><<<(C + 31) / 32, 32, 0, s>>>(C, crank, x, cams_src, cams_dst, camw64_dst, camw_dst, camdf_dst,
                                                     model);
  if (P > 0) k_candidate_pts<T><<<(P + 255) / 256, 256, 0, s>>>(P, dp, pts_src, pts_dst, ptsw_dst, ptdf_dst);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_scatter_cams(int C, const int* __restrict__ crank, const T* __restrict__ x,
                               double* __restrict__ dc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * C) return;
  int c = i / 9, j = i - 9 * c;
  int r = crank[c];
  dc[i] = r >= 0 ? (double)x[9 * (size_t)r + j] : 0.0;
}

template <typename T>
cudaError_t launch_scatter_cams(int C, const int* crank, const T* x, double* dc, cudaStream_t s) {
  if (C > 0) k_scatter_cams<T><<<(9 * C + 255) / 256, 256, 0, s>>>(C, crank, x, dc);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t s) {
  if (n > 0) {
    long long g = (n + 255) / 256;
    k_to_double<T><<<(int)(g > 65535 ? 65535 : g), 256, 0, s>>>(src, dst, n);
  }
  return cudaGetLastError();
}

__global__ void k_permute_u8(const int* __restrict__ orig, const uint8_t* __restrict__ src,
                             uint8_t* __restrict__ dst, int N) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) dst[orig[k]] = src[k];
}

cudaError_t launch_permute_u8(const int* orig, const uint8_t* src, uint8_t* dst, int N, cudaStream_t s) {
  if (N > 0) k_permute_u8<<<(N + 255) / 256, 256, 0, s>>>(orig, src, dst, N);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_permute_rows(const int* __restrict__ orig, const int* __restrict__ row,
                               const T* __restrict__ src, int src_stride, double* __restrict__ dst,
                               int N, int width) {
  long long tot = (long long)N * width;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    int k = (int)(i / width), j = (int)(i - (long long)k * width);
    size_t r = row ? (size_t)row[k] : (size_t)k;
    dst[(size_t)orig[k] * width + j] = (double)src[r * src_stride + j];
  }
}

template <typename T>
cudaError_t launch_permute_rows(const int* orig, const int* row, const T* src, int src_stride,
                                double* dst, int N, int width, cudaStream_t s) {
  long long tot = (long long)N * width;
  if (tot > 0) {
    long long g = (tot + 255) / 256;
    k_permute_rows<T><<<(int)(g > 65535 ? 65535 : g), 256, 0, s>>>(orig, row, src, src_stride, dst, N, width);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define BAB_INST(T)                                                                                \
  template cudaError_t launch_prep_cams<T>(const double*, T*, double*, int, cudaStream_t, int);     \
  template cudaError_t launch_prep_pts<T>(const double*, T*, int, cudaStream_t);                    \
  template cudaError_t launch_obs_layout<T>(int, const double*, const double*, const int*, const int*,  \
                                            const int*, const int*, int*, double*, double*, T*, T*,    \
                                            int*, T*, T*, cudaStream_t);                               \
  template cudaError_t launch_pt_lin<T>(const Layout&, const ModelParams&, const T*, const T*,      \
                                        const uint8_t*, T*, T*, T*, T*, cudaStream_t, float*);      \
  template cudaError_t launch_cam_accum<T>(const Layout&, const ModelParams&, int, const T*,        \
                                           const T*, const uint8_t*, const uint8_t*, const int*,    \
                                           const T*, const T*, T*, cudaStream_t);                   \
  template cudaError_t launch_cam_reduce<T>(const Layout&, const T*, T*, cudaStream_t);             \
  template cudaError_t launch_damp_pts<T>(int, const T*, const T*, const uint8_t*, double, T*, T*,  \
                                          int*, cudaStream_t, float*);                              \
  template cudaError_t launch_schur_diag<T>(int, const int*, const T*, const T*, double, T*, T*,    \
                                            T*, T*, T*, double*, int*, cudaStream_t, int);          \
  template cudaError_t launch_pred_cams<T>(int, const int*, const T*, const T*, const T*, double,   \
                                           double*, int, cudaStream_t);                             \
  template cudaError_t launch_candidate<T>(int, int, const int*, const T*, const T*, const double*, \
                                           const double*, double*, double*, double*, T*, T*,        \
                                           F2*, float4*, cudaStream_t, int);                        \
  template cudaError_t launch_scatter_cams<T>(int, const int*, const T*, double*, cudaStream_t);    \
  template cudaError_t launch_to_double<T>(const T*, double*, long long, cudaStream_t);              \
  template cudaError_t launch_permute_rows<T>(const int*, const int*, const T*, int, double*, int,    \
                                              int, cudaStream_t);

BAB_INST(float)
BAB_INST(double)

BA_BOUNDS_QUERY(bounds_fault_kernels)

}  // namespace bab
