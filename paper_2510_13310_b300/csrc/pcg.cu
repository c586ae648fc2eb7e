// pcg.cu -- step (d): persistent block-Jacobi PCG on the reduced camera system
// with the point back-substitution (Sec. 4.2 step 3: "preconditioned conjugate
// gradient", then scatter of the compact update).
//
// One cooperative launch runs the whole solve.  The Schur matvec
//   S p = U* p - sum_pts W_p V*_p^-1 (sum_k W_k^T p_c(k))
// walks the observations in point order, one tile of whole points at a time.
// Tiles arrive in shared memory through bulk asynchronous copies (TMA,
// cp.async.bulk) into a ring of stages, so later tiles load while the current
// one is computed.  W_k = rho'_k Jc_k^T Jp_k is applied in one of two ways:
//   stored     W rows (9x3, padded to 28 entries) are streamed;
//   recompute  only the signed IRLS weight of each observation is streamed and
//              the Jacobian pieces are recomputed from the point and camera
//              (Jp = D R, Jc = [D(-[R X]x) | D | J_intr], D = dr/dP), using
//                W^T p = rho' R^T D^T (D (p_w x R X + p_t) + J_intr p_intr)
//                W z   = rho' [ R X x g ; g ; J_intr^T e ],  e = D R z, g = D^T e.
// Inside a tile every warp owns a range of whole points (at most 32
// observations, or one longer point) and works warp-synchronously:
//   1. per observation  a_k = W_k^T p_c(k)
//   2. per point        z_p = V*_p^-1 sum_k a_k       (segmented warp scan)
//   3. per observation  v_k = W_k z_p(k)
// then, after one block barrier,
//   4. per camera run   y_c += sum_k v_k    (the tile's observations pre-sorted
//                                             by camera: fixed-order sums).
// Each block owns a contiguous slice of the free cameras: it keeps that slice
// of x, r, z, U* and the preconditioner in shared memory and reduces the
// blocks' partial y in a fixed order after a grid barrier.  Every block keeps
// its own full copy of the search direction p (p <- z + beta p) so only z and
// the partial y cross blocks.  Dot products are FP64 and summed in one fixed
// order by every block, so all blocks take the same convergence decision; no
// floating-point atomics are used, and runs are bit-reproducible.  Grid
// barriers and mbarrier waits give up after a time limit and raise a flag.
#include <cuda/atomic>

#include "internal.h"
#include "tile_meta.cuh"
#include "tma.cuh"

namespace bab {

constexpr int kVtRows = kTileObs + 2;


// Byte layout of one pipeline stage.
struct StageLayout {
  size_t w, m, x, v, bytes;
};
__host__ __device__ __forceinline__ StageLayout stage_layout(size_t tsize, int recompute) {
  StageLayout L;
  L.w = 0;
  size_t wb = recompute ? tsize * kTileObs : tsize * kTileObs * kWStride;
  L.m = wb;
  L.x = L.m + kMetaBytes;
  size_t xb = recompute ? tsize * kVtRows * 4 : 0;
  L.v = L.x + xb;
  L.bytes = L.v + tsize * kVtRows * 6;
  L.bytes = (L.bytes + 127) & ~size_t(127);
  return L;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err,
                                             long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(*bar);
    __threadfence();
    cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    uint64_t t0 = globaltimer_ns();
    while (cnt.load(cuda::memory_order_acquire) < target) {
      if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
        atomicOr(err, 1);
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
  }
  __syncthreads();
  cuda::atomic_ref<int, cuda::thread_scope_device> e(*err);
  return (e.load(cuda::memory_order_relaxed) & 1) == 0;  // bit 0: a wait timed out
}

constexpr int kMaxStages = 4;

template <typename T>
struct PcgSmem {
  unsigned char* stage[kMaxStages];
  StageLayout lay;
  uint64_t* mbar;
  TileDesc* dtab;   // this block's tile descriptors
  double* dred;
  T* vb;
  T* osum;
  T* xs;    // full search direction p (every block keeps its own copy)
  T* ys;    // block partial of sum W z, then the owned q
  T* xo;    // owned x, r
  T* ro;
  T* Udo;   // owned damped U blocks (45 packed) and preconditioner blocks (81)
  T* Dio;
  T* camtab;
  int* crank;
};

template <typename T>
size_t pcg_smem_bytes(int n, int C, int stages, int own_max, int recompute, int cam_in_smem,
                      int max_tiles_per_block) {
  StageLayout L = stage_layout(sizeof(T), recompute);
  size_t b = (size_t)stages * L.bytes;
  b += kMaxStages * sizeof(uint64_t);
  b += sizeof(TileDesc) * (size_t)max_tiles_per_block;
  b += sizeof(double) * (2 * kPcgThreads + 8);
  b += sizeof(T) * kTileObs * 9;                          // vb
  b += sizeof(T) * kPcgThreads;                           // osum
  b += sizeof(T) * (size_t)n * 2;                         // xs, ys
  b += sizeof(T) * (size_t)own_max * (9 * 2 + 45 + 81);   // owned slice
  b += cam_in_smem ? sizeof(T) * (size_t)C * kCamStride : 0;
  b += sizeof(int) * (size_t)C;                           // crank
  return (b + 15) & ~size_t(15);
}

template <typename T>
__device__ PcgSmem<T> carve(unsigned char* base, const PcgArgs<T>& a) {
  PcgSmem<T> s;
  s.lay = stage_layout(sizeof(T), a.recompute);
  unsigned char* p = base;
  for (int i = 0; i < kMaxStages; ++i) s.stage[i] = p + (size_t)(i < a.stages ? i : 0) * s.lay.bytes;
  p += (size_t)a.stages * s.lay.bytes;
  s.mbar = reinterpret_cast<uint64_t*>(p);
  p += kMaxStages * sizeof(uint64_t);
  s.dtab = reinterpret_cast<TileDesc*>(p);
  p += sizeof(TileDesc) * (size_t)a.max_tiles_per_block;
  s.dred = reinterpret_cast<double*>(p);
  p += sizeof(double) * (2 * kPcgThreads + 8);
  s.vb = reinterpret_cast<T*>(p);
  p += sizeof(T) * kTileObs * 9;
  s.osum = reinterpret_cast<T*>(p);
  p += sizeof(T) * kPcgThreads;
  s.xs = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)a.n;
  s.ys = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)a.n;
  s.xo = reinterpret_cast<T*>(p);
  s.ro = s.xo + 9 * a.own_max;
  s.Udo = s.ro + 9 * a.own_max;
  s.Dio = s.Udo + 45 * a.own_max;
  p += sizeof(T) * (size_t)a.own_max * (9 * 2 + 45 + 81);
  s.camtab = reinterpret_cast<T*>(p);
  p += a.cam_in_smem ? sizeof(T) * (size_t)a.C * kCamStride : 0;
  s.crank = reinterpret_cast<int*>(p);
  return s;
}

// thread 0: start the bulk copies of this block's j-th tile into stage s
template <typename T, bool REC>
__device__ void issue_tile(const PcgArgs<T>& a, PcgSmem<T>& sm, int j, int s) {
  const TileDesc d = sm.dtab[j];
  unsigned char* st = sm.stage[s];
  unsigned mbytes = (unsigned)tile_meta_bytes(d.n_obs, d.n_pts, d.n_runs);
  int pb2 = d.pt_begin & ~1, pe2 = (d.pt_begin + d.n_pts + 1) & ~1;
  unsigned vbytes = (unsigned)((pe2 - pb2) * 6 * sizeof(T));
  unsigned wbytes, xbytes = 0;
  if (REC) {
    wbytes = (unsigned)(pad4(d.n_obs) * sizeof(T));
    xbytes = (unsigned)((pe2 - pb2) * 4 * sizeof(T));
  } else {
    wbytes = (unsigned)(d.n_obs * kWStride * sizeof(T));
  }
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sm.mbar[s], wbytes + mbytes + xbytes + vbytes);
  if (wbytes) {
    if (REC) bulk_g2s(st + sm.lay.w, a.wsgn + (size_t)d.g_row, wbytes, &sm.mbar[s]);
    else bulk_g2s(st + sm.lay.w, a.W + kWStride * (size_t)d.w_row, wbytes, &sm.mbar[s]);
  }
  bulk_g2s(st + sm.lay.m, a.meta + d.meta_off, mbytes, &sm.mbar[s]);
  if (xbytes) bulk_g2s(st + sm.lay.x, a.ptsw + 4 * (size_t)pb2, xbytes, &sm.mbar[s]);
  bulk_g2s(st + sm.lay.v, a.Vinv + 6 * (size_t)pb2, vbytes, &sm.mbar[s]);
}

template <typename T>
__device__ __forceinline__ void load_wrow(const T* __restrict__ src, T w[27]) {
  if constexpr (sizeof(T) == 4) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      float4 v = q[i];
      if (4 * i < 27) w[4 * i] = v.x;
      if (4 * i + 1 < 27) w[4 * i + 1] = v.y;
      if (4 * i + 2 < 27) w[4 * i + 2] = v.z;
      if (4 * i + 3 < 27) w[4 * i + 3] = v.w;
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int i = 0; i < 14; ++i) {
      double2 v = q[i];
      if (2 * i < 27) w[2 * i] = v.x;
      if (2 * i + 1 < 27) w[2 * i + 1] = v.y;
    }
  }
}

// The operator W_k of one observation: either a stored row or recomputed pieces.
template <typename T>
struct WOp {
  T w[27];                                 // stored
  T R[9], a0, a1, a2;                      // recompute: rotation, R X
  T D00, D01, D02, D10, D11, D12, D22;     // dr/dP
  T ju0, ju1, ju2, jv0, jv1, jv2;          // intrinsic partials of u, v
  T rw;                                    // rho'
  bool ctr;                                // centre model: a = R (X - c), slots 3-5 the centre

  __device__ __forceinline__ void wt_x(const T* __restrict__ x, bool rec, T& o0, T& o1, T& o2) const {
    if (!rec) {
      o0 = o1 = o2 = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        T xq = x[q];
        o0 += w[3 * q] * xq;
        o1 += w[3 * q + 1] * xq;
        o2 += w[3 * q + 2] * xq;
      }
      return;
    }
    // t = Jc x = D (x_w x a + x_t) + J_intr x_intr (radial: a = RX); centre
    // model: D (x_w x a - R x_c) with a = R (X - c)
    T m0 = x[1] * a2 - x[2] * a1, m1 = x[2] * a0 - x[0] * a2, m2 = x[0] * a1 - x[1] * a0;
    if (ctr) {
      m0 -= R[0] * x[3] + R[1] * x[4] + R[2] * x[5];
      m1 -= R[3] * x[3] + R[4] * x[4] + R[5] * x[5];
      m2 -= R[6] * x[3] + R[7] * x[4] + R[8] * x[5];
    } else {
      m0 += x[3];
      m1 += x[4];
      m2 += x[5];
    }
    T tu = D00 * m0 + D01 * m1 + D02 * m2 + ju0 * x[6] + ju1 * x[7] + ju2 * x[8];
    T tv = D10 * m0 + D11 * m1 + D12 * m2 + jv0 * x[6] + jv1 * x[7] + jv2 * x[8];
    T td = D22 * m2;
    // W^T x = rho' R^T D^T t
    T g0 = D00 * tu + D10 * tv, g1 = D01 * tu + D11 * tv, g2 = D02 * tu + D12 * tv + D22 * td;
    o0 = rw * (R[0] * g0 + R[3] * g1 + R[6] * g2);
    o1 = rw * (R[1] * g0 + R[4] * g1 + R[7] * g2);
    o2 = rw * (R[2] * g0 + R[5] * g1 + R[8] * g2);
  }

  __device__ __forceinline__ void w_z(T z0, T z1, T z2, bool rec, T* __restrict__ o) const {
    if (!rec) {
#pragma unroll
      for (int q = 0; q < 9; ++q) o[q] = w[3 * q] * z0 + w[3 * q + 1] * z1 + w[3 * q + 2] * z2;
      return;
    }
    // e = D R z, g = D^T e; W z = rho' [RX x g ; g ; J_intr^T e]
    T q0 = R[0] * z0 + R[1] * z1 + R[2] * z2;
    T q1 = R[3] * z0 + R[4] * z1 + R[5] * z2;
    T q2 = R[6] * z0 + R[7] * z1 + R[8] * z2;
    T eu = D00 * q0 + D01 * q1 + D02 * q2;
    T ev = D10 * q0 + D11 * q1 + D12 * q2;
    T ed = D22 * q2;
    T g0 = D00 * eu + D10 * ev, g1 = D01 * eu + D11 * ev, g2 = D02 * eu + D12 * ev + D22 * ed;
    o[0] = rw * (a1 * g2 - a2 * g1);
    o[1] = rw * (a2 * g0 - a0 * g2);
    o[2] = rw * (a0 * g1 - a1 * g0);
    if (ctr) {  // centre columns -D R: -(R^T g)
      o[3] = -rw * (R[0] * g0 + R[3] * g1 + R[6] * g2);
      o[4] = -rw * (R[1] * g0 + R[4] * g1 + R[7] * g2);
      o[5] = -rw * (R[2] * g0 + R[5] * g1 + R[8] * g2);
    } else {
      o[3] = rw * g0;
      o[4] = rw * g1;
      o[5] = rw * g2;
    }
    o[6] = rw * (ju0 * eu + jv0 * ev);
    o[7] = rw * (ju1 * eu + jv1 * ev);
    o[8] = rw * (ju2 * eu + jv2 * ev);
  }
};

// Build the operator of observation i of the current tile.
template <typename T, bool REC>
__device__ __forceinline__ void make_op(const PcgArgs<T>& a, const PcgSmem<T>& sm,
                                        const unsigned char* st, int i, int cam, int seg, int pt_off2,
                                        WOp<T>& op) {
  if (!REC) {
    load_wrow(reinterpret_cast<const T*>(st + sm.lay.w) + kWStride * i, op.w);
    return;
  }
  T ws = reinterpret_cast<const T*>(st + sm.lay.w)[i];
  const T* X = reinterpret_cast<const T*>(st + sm.lay.x) + 4 * (pt_off2 + seg);
  T cw[kCamStride];
  if (a.cam_in_smem) {
    const T* c = sm.camtab + kCamStride * cam;
#pragma unroll
    for (int q = 0; q < kCamStride; ++q) cw[q] = c[q];
  } else {
    using V4 = typename Vec4<T>::type;
    const V4* c = reinterpret_cast<const V4*>(a.camw + kCamStride * (size_t)cam);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      V4 v;
      if constexpr (sizeof(T) == 4) v = __ldg(c + q);
      else v = c[q];
      cw[4 * q] = v.x;
      cw[4 * q + 1] = v.y;
      cw[4 * q + 2] = v.z;
      cw[4 * q + 3] = v.w;
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) op.R[q] = cw[q];
  T X0 = X[0], X1 = X[1], X2 = X[2];
  op.a0 = cw[0] * X0 + cw[1] * X1 + cw[2] * X2;
  op.a1 = cw[3] * X0 + cw[4] * X1 + cw[5] * X2;
  op.a2 = cw[6] * X0 + cw[7] * X1 + cw[8] * X2;
  T px = op.a0 + cw[9], py = op.a1 + cw[10], pz = op.a2 + cw[11];
  T f = cw[12], k1 = cw[13], k2 = cw[14];
  T iz = T(1) / pz;
  T xn = px * iz, yn = py * iz;
  T rr = xn * xn + yn * yn;
  T dist = T(1) + rr * (k1 + k2 * rr);
  T fd = f * dist;
  T g = T(2) * f * (k1 + T(2) * k2 * rr);
  op.D00 = fd * iz + g * xn * xn * iz;
  op.D01 = g * xn * yn * iz;
  op.D02 = -fd * xn * iz - g * xn * rr * iz;
  op.D10 = op.D01;
  op.D11 = fd * iz + g * yn * yn * iz;
  op.D12 = -fd * yn * iz - g * yn * rr * iz;
  T sw = ws > T(0) ? (T)a.sw_valid : (T)a.sw_invalid;
  op.D22 = -sw * iz * iz;
  op.ju0 = dist * xn;
  op.ju1 = f * xn * rr;
  op.ju2 = f * xn * rr * rr;
  op.jv0 = dist * yn;
  op.jv1 = f * yn * rr;
  op.jv2 = f * yn * rr * rr;
  op.rw = ws < T(0) ? -ws : ws;
  op.ctr = cw[15] != T(0);
  if (op.ctr) {
    // centre model: the rotation increment acts on P = R (X - c); no distortion columns
    op.a0 = px, op.a1 = py, op.a2 = pz;
    op.ju1 = op.ju2 = op.jv1 = op.jv2 = T(0);
  }
}

template <typename T>
__device__ __forceinline__ void backsub_point(const PcgArgs<T>& a, const T* v, size_t p, T s0, T s1,
                                              T s2, double& pred) {
  double t0 = -(double)a.gp[3 * p] - (double)s0, t1 = -(double)a.gp[3 * p + 1] - (double)s1,
         t2 = -(double)a.gp[3 * p + 2] - (double)s2;
  T d0 = (T)(v[0] * t0 + v[1] * t1 + v[2] * t2);
  T d1 = (T)(v[1] * t0 + v[3] * t1 + v[4] * t2);
  T d2 = (T)(v[2] * t0 + v[4] * t1 + v[5] * t2);
  a.dp[3 * p] = d0;
  a.dp[3 * p + 1] = d1;
  a.dp[3 * p + 2] = d2;
  const T* vv = a.V + 6 * p;
  double dd3[3] = {(double)d0, (double)d1, (double)d2};
  double dg[3] = {fmin(fmax((double)vv[0], 1e-6), 1e32), fmin(fmax((double)vv[3], 1e-6), 1e32),
                  fmin(fmax((double)vv[5], 1e-6), 1e32)};
  for (int k = 0; k < 3; ++k) pred += dd3[k] * (a.lambda * dg[k] * dd3[k] - (double)a.gp[3 * p + k]);
}

// Per-tile work.  MODE 0: Schur matvec contribution into ys.  MODE 1: point
// back-substitution dp = V*^-1 (-g_p - sum_k W_k^T x) and the point part of the
// predicted decrease 1/2 dx^T (lambda D dx - g), accumulated into pred.
template <typename T, int MODE, bool REC>
__device__ void tile_compute(const PcgArgs<T>& a, PcgSmem<T>& sm, int j, int s, double& pred) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileDesc d = sm.dtab[j];
  const unsigned char* st = sm.stage[s];
  const int nobs = d.n_obs, npts = d.n_pts, nruns = d.n_runs;
  const int* camS = reinterpret_cast<const int*>(st + sm.lay.m);
  const int* poffS = camS + pad4(nobs);
  const unsigned* runsS = reinterpret_cast<const unsigned*>(poffS + pad4(npts + 1));
  const int* wrS = reinterpret_cast<const int*>(runsS + pad4(nruns));
  const uint8_t* cpermS = reinterpret_cast<const uint8_t*>(wrS + 16);
  const uint8_t* lidS = cpermS + pad16(nobs);
  const int off2 = d.pt_begin - (d.pt_begin & ~1);
  const T* Vt = reinterpret_cast<const T*>(st + sm.lay.v) + 6 * off2;
  constexpr bool rec = REC;
  T* vb = sm.vb;
  const unsigned FULL = 0xffffffffu;

  // ---- steps 1-3, one warp per range of whole points
  {
    const int wb = wrS[warp], we = wrS[warp + 1];
    const int nw = we - wb;
    if (nw > 0 && nw <= 32) {
      int i = wb + lane;
      bool on = lane < nw;
      WOp<T> op;
      int cr = -1, seg = 1024 + lane;
      T a0 = T(0), a1 = T(0), a2 = T(0);
      if (on) {
        int cam = camS[i];
        cr = sm.crank[cam];
        seg = lidS[i];
        if (cr >= 0) {
          make_op<T, REC>(a, sm, st, i, cam, seg, off2, op);
          op.wt_x(sm.xs + 9 * cr, rec, a0, a1, a2);
        }
      }
      // segmented inclusive scan over lanes of the same point
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        T t0 = __shfl_up_sync(FULL, a0, dd), t1 = __shfl_up_sync(FULL, a1, dd),
          t2 = __shfl_up_sync(FULL, a2, dd);
        int ts = __shfl_up_sync(FULL, seg, dd);
        if (lane >= dd && ts == seg) {
          a0 += t0;
          a1 += t1;
          a2 += t2;
        }
      }
      int last = on ? poffS[seg + 1] - 1 - wb : lane;  // the point's last lane holds the total
      T s0 = __shfl_sync(FULL, a0, last), s1 = __shfl_sync(FULL, a1, last),
        s2 = __shfl_sync(FULL, a2, last);
      if (on) {
        if (MODE == 0) {
          T* o = vb + 9 * i;
          if (cr >= 0) {
            const T* v = Vt + 6 * seg;
            T z0 = v[0] * s0 + v[1] * s1 + v[2] * s2;
            T z1 = v[1] * s0 + v[3] * s1 + v[4] * s2;
            T z2 = v[2] * s0 + v[4] * s1 + v[5] * s2;
            op.w_z(z0, z1, z2, rec, o);
          } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) o[q] = T(0);
          }
        } else if (lane == last) {
          backsub_point(a, Vt + 6 * seg, (size_t)d.pt_begin + seg, s0, s1, s2, pred);
        }
      }
    } else if (nw > 32) {
      // one point with more than 32 observations: chunked warp reduction
      int seg = lidS[wb];
      T a0 = T(0), a1 = T(0), a2 = T(0);
      for (int i = wb + lane; i < we; i += 32) {
        int cam = camS[i];
        int cr = sm.crank[cam];
        if (cr < 0) continue;
        WOp<T> op;
        T b0, b1, b2;
        make_op<T, REC>(a, sm, st, i, cam, seg, off2, op);
        op.wt_x(sm.xs + 9 * cr, rec, b0, b1, b2);
        a0 += b0;
        a1 += b1;
        a2 += b2;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(FULL, a0, o);
        a1 += __shfl_xor_sync(FULL, a1, o);
        a2 += __shfl_xor_sync(FULL, a2, o);
      }
      const T* v = Vt + 6 * seg;
      if (MODE == 0) {
        T z0 = v[0] * a0 + v[1] * a1 + v[2] * a2;
        T z1 = v[1] * a0 + v[3] * a1 + v[4] * a2;
        T z2 = v[2] * a0 + v[4] * a1 + v[5] * a2;
        for (int i = wb + lane; i < we; i += 32) {
          T* o = vb + 9 * i;
          int cam = camS[i];
          if (sm.crank[cam] < 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) o[q] = T(0);
            continue;
          }
          WOp<T> op;
          make_op<T, REC>(a, sm, st, i, cam, seg, off2, op);
          op.w_z(z0, z1, z2, rec, o);
        }
      } else if (lane == 0) {
        backsub_point(a, v, (size_t)d.pt_begin + seg, a0, a1, a2, pred);
      }
    }
  }
  if (MODE == 1) {
    // points without any observation: dp = -V*^-1 g_p (zero when inactive)
    for (int jp = tid; jp < npts; jp += blockDim.x) {
      if (poffS[jp + 1] > poffS[jp]) continue;
      size_t p = (size_t)d.pt_begin + jp;
      const T* v = Vt + 6 * jp;
      double t0 = -(double)a.gp[3 * p], t1 = -(double)a.gp[3 * p + 1], t2 = -(double)a.gp[3 * p + 2];
      a.dp[3 * p] = (T)(v[0] * t0 + v[1] * t1 + v[2] * t2);
      a.dp[3 * p + 1] = (T)(v[1] * t0 + v[3] * t1 + v[4] * t2);
      a.dp[3 * p + 2] = (T)(v[2] * t0 + v[4] * t1 + v[5] * t2);
    }
    return;
  }
  __syncthreads();
  // ---- step 4: per camera run (distinct cameras in a tile): y_c += sum v_k
  for (int r = tid; r < nruns; r += blockDim.x) {
    unsigned u = runsS[r];
    int cr = sm.crank[u >> 8];
    if (cr < 0) continue;
    int jb = (int)(u & 255u);
    int je = r + 1 < nruns ? (int)(runsS[r + 1] & 255u) : nobs;
    T acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = T(0);
    for (int jj = jb; jj < je; ++jj) {
      const T* o = vb + 9 * cpermS[jj];
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q] += o[q];
    }
    T* yv = sm.ys + 9 * cr;
#pragma unroll
    for (int q = 0; q < 9; ++q) yv[q] += acc[q];
  }
}

// Tile pipeline: `issued` / `consumed` count tiles over the whole launch; the
// q-th tile uses stage q % S and the mbarrier phase (q / S) & 1.
struct Pipe {
  int issued, consumed;
};

__device__ __forceinline__ int block_tiles(int n_tiles) {
  return (int)blockIdx.x < n_tiles ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
}

// Issue the first S-1 tiles of the next walk (may run before vectors are staged).
template <typename T, bool REC>
__device__ void walk_prologue(const PcgArgs<T>& a, PcgSmem<T>& sm, Pipe& pp) {
  const int S = a.stages, ntl = block_tiles(a.n_tiles);
  const int want = min(S > 1 ? S - 1 : 0, ntl);
  while (pp.issued - pp.consumed < want) {
    if (threadIdx.x == 0) issue_tile<T, REC>(a, sm, pp.issued - pp.consumed, pp.issued % S);
    ++pp.issued;
  }
}

template <typename T, int MODE, bool REC>
__device__ bool walk_tiles(const PcgArgs<T>& a, PcgSmem<T>& sm, Pipe& pp, double& pred) {
  const int S = a.stages, ntl = block_tiles(a.n_tiles);
  walk_prologue<T, REC>(a, sm, pp);
  const int base = pp.consumed;
  for (int j = 0; j < ntl; ++j) {
    int jn = S > 1 ? j + S - 1 : j;
    if (jn < ntl && pp.issued - base == jn) {
      if (threadIdx.x == 0) issue_tile<T, REC>(a, sm, jn, pp.issued % S);
      ++pp.issued;
    }
    const int q = base + j;
    const int s = q % S;
    const unsigned parity = (unsigned)((q / S) & 1);
    if (!mbar_wait(&sm.mbar[s], parity, a.timeout_ns)) {
      atomicOr(a.err, 1);
      mbar_wait(&sm.mbar[s], parity, a.timeout_ns);  // let a late copy land before leaving
      return false;
    }
    tile_compute<T, MODE, REC>(a, sm, j, s, pred);
    __syncthreads();
  }
  pp.consumed = base + ntl;
  return true;
}

__device__ __forceinline__ double sum_dots(const double* region, int slot, int G, double* red) {
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) s += region[4 * g + slot];
  return block_sum(s, red);
}

template <typename T, bool REC>
__global__ void __launch_bounds__(kPcgThreads, REC ? 2 : 1) k_pcg(PcgArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PcgSmem<T> sm = carve<T>(smem_raw, a);
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int n = a.n;
  const int f0 = (int)(((long long)a.Cf * bid) / G), f1 = (int)(((long long)a.Cf * (bid + 1)) / G);
  const int e0 = 9 * f0, ne = 9 * (f1 - f0);
  const int cnt = min(ne, (int)blockDim.x);
  double* dout = sm.dred + 2 * kPcgThreads;
  unsigned epoch = 0;
  Pipe pp{0, 0};
  double unused = 0.0;

  if (tid == 0) {
    for (int i = 0; i < kMaxStages; ++i) mbar_init(&sm.mbar[i], 1);
    fence_mbar_init();
  }
  for (int j = tid; j < block_tiles(a.n_tiles); j += blockDim.x) sm.dtab[j] = a.descs[bid + j * G];
  for (int c = tid; c < a.C; c += blockDim.x) sm.crank[c] = a.crank[c];
  if (a.cam_in_smem)
    for (int q = tid; q < a.C * kCamStride; q += blockDim.x) sm.camtab[q] = a.camw[q];
  // owned slice: damped U blocks, preconditioner, b
  for (int q = tid; q < 45 * (f1 - f0); q += blockDim.x) sm.Udo[q] = a.Ud[45 * (size_t)f0 + q];
  for (int q = tid; q < 81 * (f1 - f0); q += blockDim.x) sm.Dio[q] = a.Dinv[81 * (size_t)f0 + q];
  for (int q = tid; q < ne; q += blockDim.x) {
    sm.xo[q] = T(0);
    sm.ro[q] = a.b[e0 + q];
  }
  __syncthreads();

  // ---- x = 0, r = b, z = M^-1 r (published), first p = z; dots r.z and b.b
  double loc_rz = 0.0, loc_bb = 0.0;
  for (int q = tid; q < ne; q += blockDim.x) {
    int f = q / 9, i = q - 9 * f;
    const T* Mi = sm.Dio + 81 * f + 9 * i;
    T zz = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) zz += Mi[k] * sm.ro[9 * f + k];
    a.z[e0 + q] = zz;
    double rv = (double)sm.ro[q];
    loc_rz += rv * (double)zz;
    loc_bb += rv * rv;
  }
  // Dot products of consecutive phases alternate between two regions of G x 4
  // doubles: a region is rewritten only after every block passed the barrier
  // that follows its last read.
  int dph = 0;
  auto dregion = [&](int ph) { return a.dots + (size_t)(ph & 1) * 4 * G; };
  {
    double s0, s1;
    warp0_sum2(loc_rz, loc_bb, cnt, sm.dred, dout, s0, s1);
    if (tid == 0) {
      dregion(dph)[4 * bid + 0] = s0;
      dregion(dph)[4 * bid + 1] = s1;
    }
  }
  if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
  double rz, bb;
  warp0_sum_slots(dregion(dph), G, 0, 1, dout + 4, rz, bb);
  ++dph;
  double bnorm = sqrt(bb);
  int it = 0;
  double rr_last = bb;
  double beta = 0.0;
  bool first = true;
  while (bnorm > 0.0 && it < a.max_iters) {
    walk_prologue<T, REC>(a, sm, pp);
    // ---- p = z (first) or z + beta p, in every block's own copy; clear the partial.
    // Every load of z is issued before any use.
    for (int base = 0; base < n; base += 4 * (int)blockDim.x) {
      T zv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = base + u * blockDim.x + tid;
        zv[u] = e < n ? a.z[e] : T(0);
      }
      const T bt = (T)beta;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = base + u * blockDim.x + tid;
        if (e < n) {
          sm.xs[e] = first ? zv[u] : zv[u] + bt * sm.xs[e];
          sm.ys[e] = T(0);
        }
      }
    }
    first = false;
    __syncthreads();
    if (!walk_tiles<T, 0, REC>(a, sm, pp, unused)) return;
    T* mypart = a.partials + (size_t)bid * n;
    for (int e = tid; e < n; e += blockDim.x) mypart[e] = sm.ys[e];
    if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;

    // ---- owners: q = U* p - sum_g partial_g (fixed order); p.q
    double loc_pq = 0.0;
    for (int base = 0; base < ne; base += blockDim.x) {
      int cnt = min(ne - base, (int)blockDim.x);
      int grp = (int)blockDim.x / cnt;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      if (tid < cnt * grp) {
        int el = tid % cnt, g = tid / cnt;
        const T* col = a.partials + e0 + base + el;
        for (; g + 3 * grp < G; g += 4 * grp) {
          s0 += col[(size_t)g * n];
          s1 += col[(size_t)(g + grp) * n];
          s2 += col[(size_t)(g + 2 * grp) * n];
          s3 += col[(size_t)(g + 3 * grp) * n];
        }
        for (; g < G; g += grp) s0 += col[(size_t)g * n];
      }
      sm.osum[tid] = (s0 + s1) + (s2 + s3);
      __syncthreads();
      if (tid < cnt) {
        T tot = T(0);
        for (int g0 = 0; g0 < grp; ++g0) tot += sm.osum[g0 * cnt + tid];
        int q = base + tid;
        int f = q / 9, i = q - 9 * f;
        const T* ud = sm.Udo + 45 * f;
        const T* pv = sm.xs + e0 + 9 * f;
        T up = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) up += ud[sym9(i, k)] * pv[k];
        T qv = up - tot;
        sm.ys[e0 + q] = qv;  // owned q kept in shared memory
        loc_pq += (double)pv[i] * (double)qv;
      }
      __syncthreads();
    }
    {
      double s0, s1;
      warp0_sum2(loc_pq, 0.0, cnt, sm.dred, dout, s0, s1);
      if (tid == 0) dregion(dph)[4 * bid + 2] = s0;
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double pq, unused_pq;
    warp0_sum_slots(dregion(dph), G, 2, 2, dout + 4, pq, unused_pq);
    ++dph;
    if (!(pq > 0.0) || !isfinite(pq)) {
      if (bid == 0 && tid == 0) atomicOr(a.err, 2);
      break;
    }
    double alpha = rz / pq;
    // ---- owners: x += alpha p, r -= alpha q, z = M^-1 r (published); r.r and r.z
    for (int q = tid; q < ne; q += blockDim.x) {
      sm.xo[q] = (T)((double)sm.xo[q] + alpha * (double)sm.xs[e0 + q]);
      sm.ro[q] = (T)((double)sm.ro[q] - alpha * (double)sm.ys[e0 + q]);
    }
    __syncthreads();
    double loc_rr = 0.0, loc_rz2 = 0.0;
    for (int q = tid; q < ne; q += blockDim.x) {
      int f = q / 9, i = q - 9 * f;
      const T* Mi = sm.Dio + 81 * f + 9 * i;
      T zz = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) zz += Mi[k] * sm.ro[9 * f + k];
      a.z[e0 + q] = zz;
      double rv = (double)sm.ro[q];
      loc_rr += rv * rv;
      loc_rz2 += rv * (double)zz;
    }
    {
      double s0, s1;
      warp0_sum2(loc_rr, loc_rz2, cnt, sm.dred, dout, s0, s1);
      if (tid == 0) {
        dregion(dph)[4 * bid + 0] = s0;
        dregion(dph)[4 * bid + 1] = s1;
      }
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double rr, rz2;
    warp0_sum_slots(dregion(dph), G, 0, 1, dout + 4, rr, rz2);
    ++dph;
    ++it;
    rr_last = rr;
    if (sqrt(rr) <= a.tol * bnorm) break;
    beta = rz2 / rz;
    rz = rz2;
  }
  if (bid == 0 && tid == 0) {
    a.sc->pcg_iters = it;
    a.sc->pcg_bnorm = bnorm;
    a.sc->pcg_rel_res = bnorm > 0.0 ? sqrt(rr_last) / bnorm : 0.0;
  }

  // ---- publish x; back-substitution with the final x (every block needs all of x)
  for (int q = tid; q < ne; q += blockDim.x) a.x[e0 + q] = sm.xo[q];
  if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
  walk_prologue<T, REC>(a, sm, pp);
  for (int e = tid; e < n; e += blockDim.x) sm.xs[e] = a.x[e];
  __syncthreads();
  double pred = 0.0;
  if (!walk_tiles<T, 1, REC>(a, sm, pp, pred)) return;
  double ps, unused_ps;
  warp0_sum2(pred, 0.0, blockDim.x, sm.dred, dout, ps, unused_ps);
  if (tid == 0) a.pred_parts[bid] = ps;
}

// FP32 recomputes the W blocks, FP64 streams stored ones.
template <typename T>
const void* pcg_kernel_ptr() {
  return reinterpret_cast<const void*>(&k_pcg<T, sizeof(T) == 4>);
}

template <typename T>
cudaError_t launch_pcg(const PcgArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  if (a.stages < 1 || a.stages > kMaxStages || a.recompute != (sizeof(T) == 4 ? 1 : 0))
    return cudaErrorInvalidValue;
  void* args[] = {const_cast<PcgArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel(pcg_kernel_ptr<T>(), dim3(grid), dim3(kPcgThreads), args, smem, s);
}

int pcg_threads() { return kPcgThreads; }
int pcg_max_stages() { return kMaxStages; }


template size_t pcg_smem_bytes<float>(int, int, int, int, int, int, int);
template size_t pcg_smem_bytes<double>(int, int, int, int, int, int, int);
template const void* pcg_kernel_ptr<float>();
template const void* pcg_kernel_ptr<double>();
template cudaError_t launch_pcg<float>(const PcgArgs<float>&, int, size_t, cudaStream_t);
template cudaError_t launch_pcg<double>(const PcgArgs<double>&, int, size_t, cudaStream_t);

}  // namespace bab
