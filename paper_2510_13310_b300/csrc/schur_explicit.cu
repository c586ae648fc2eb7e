// schur_explicit.cu -- step (b)/(d) on an explicit reduced camera system.
//
// When the free cameras are few enough for the Schur complement
//   S = U* - sum_p sum_{k,k' in p} W_k V*_p^-1 W_k'^T          (Eq. LM, Schur form)
// to be held densely, it is formed once per damping value and the PCG runs on
// it directly: each block keeps its rows of S in shared memory, so a matvec is
// a dense row-block product with no cross-block partial sums.
//
// S is formed Jacobi-scaled, S^ = D^-1 S D^-1 with D = sqrt(diag U*), so every
// entry is of order one.  Off-diagonal blocks are accumulated by their row
// camera: a block owns one free camera i (and a range of columns) and, for each
// of its observations k of point p and each observation k' of p in a camera
// ranked after i, adds W_k V*_p^-1 W_k'^T into a shared-memory row block held
// as 64-bit fixed point (2^-48 units).  Integer addition is associative, so the
// result does not depend on the order in which threads add: S^ is
// bit-reproducible.  The diagonal blocks come from the block-Jacobi pass
// (U* - sum W V*^-1 W^T) and the lower triangle is mirrored from the upper.
#include <cuda/atomic>

#include "internal.h"
#include "model.cuh"

namespace bab {

// Fixed-point accumulators.  Every partial sum of W_k V*^-1 W_k'^T scaled by
// D^-1 (.) D^-1 is bounded by 1 in magnitude (it is a block of a PSD matrix no
// larger than D^-1 U* D^-1, whose diagonal is 1), so FP32 accumulates in 32-bit
// integers of 2^-30 units (range +-2, finer than FP32 rounding of the terms),
// FP64 in 64-bit integers of 2^-48 units.
template <typename T> struct FixAcc;
template <> struct FixAcc<float> {
  using type = int;
  static constexpr double scale = 1073741824.0;  // 2^30
  __device__ static __forceinline__ int conv(float v) { return __float2int_rn(v); }
  __device__ static __forceinline__ void add(int* p, int v) { atomicAdd(p, v); }
  __device__ static __forceinline__ void gadd(int* p, int v) { atomicAdd(p, v); }
};
template <> struct FixAcc<double> {
  using type = long long;
  static constexpr double scale = 281474976710656.0;  // 2^48
  __device__ static __forceinline__ long long conv(double v) { return __double2ll_rn(v); }
  __device__ static __forceinline__ void add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
  }
  __device__ static __forceinline__ void gadd(long long* p, long long v) { add(p, v); }
};
constexpr int kFormThreads = 256;

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

// grid (Cf, n_col_chunks, n_obs_parts): row camera a = blockIdx.x, columns
// [9 (a+1) + blockIdx.y * chunk, ... + chunk) of the strictly upper part, and
// part blockIdx.z of camera a's observations.  W rows (point order, stride
// kWStride) are read, not recomputed.  The block's shared-memory row block is
// flushed into the global integer accumulator Sacc with integer atomics.
template <typename T>
__global__ void __launch_bounds__(kFormThreads) k_form_S(Layout L, const T* __restrict__ W,
                                                         const uint8_t* __restrict__ act_co,
                                                         const uint8_t* __restrict__ act_po,
                                                         const int* __restrict__ crank,
                                                         const int* __restrict__ cam_map,
                                                         const T* __restrict__ Vinv,
                                                         const double* __restrict__ dscale, int Cf,
                                                         int chunk,
                                                         typename FixAcc<T>::type* __restrict__ Sacc) {
  using Acc = typename FixAcc<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* acc = reinterpret_cast<Acc*>(smem_raw);  // [9][chunk]
  const int a = blockIdx.x;
  const int n = 9 * Cf;
  const int start = 9 * (a + 1) + blockIdx.y * chunk;
  if (start >= n) return;
  const int width = min(chunk, n - start);
  const int ci = cam_map[a];
  const int kb0 = L.chunk_obs[L.cam_chunk[ci]], ke0 = L.chunk_obs[L.cam_chunk[ci + 1]];
  const int per = (ke0 - kb0 + gridDim.z - 1) / gridDim.z;
  const int kb = kb0 + blockIdx.z * per, ke = min(ke0, kb + per);
  if (kb >= ke) return;
  for (int q = threadIdx.x; q < 9 * chunk; q += blockDim.x) acc[q] = 0;
  __syncthreads();
  // row scale with the fixed-point unit folded in; each term is rounded once,
  // deterministically, before the integer (order-free) sums
  T dsa[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) dsa[r] = (T)(FixAcc<T>::scale / dscale[9 * a + r]);
  const T* dinv = reinterpret_cast<const T*>(dscale + n);
  for (int k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    if (!act_co[k]) continue;
    const int p = L.co_pt[k];
    const T* Wk = W + kWStride * (size_t)L.co_po[k];
    const T* vi = Vinv + 6 * (size_t)p;
    T v00 = vi[0], v01 = vi[1], v02 = vi[2], v11 = vi[3], v12 = vi[4], v22 = vi[5];
    T Y[27];  // diag(dsa) W V*^-1
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      T w0 = Wk[3 * r], w1 = Wk[3 * r + 1], w2 = Wk[3 * r + 2];
      Y[3 * r] = dsa[r] * (w0 * v00 + w1 * v01 + w2 * v02);
      Y[3 * r + 1] = dsa[r] * (w0 * v01 + w1 * v11 + w2 * v12);
      Y[3 * r + 2] = dsa[r] * (w0 * v02 + w1 * v12 + w2 * v22);
    }
    for (int k2 = L.pt_off[p]; k2 < L.pt_off[p + 1]; ++k2) {
      const int b = crank[L.po_cam[k2]];
      if (b <= a || !act_po[k2]) continue;
      const int col0 = 9 * b - start;
      if (col0 < 0 || col0 >= width) continue;
      const T* W2 = W + kWStride * (size_t)k2;
      T Z[27];  // W2 scaled by its column scales
#pragma unroll
      for (int s2 = 0; s2 < 9; ++s2) {
        T ds = dinv[9 * b + s2];
        Z[3 * s2] = ds * W2[3 * s2];
        Z[3 * s2 + 1] = ds * W2[3 * s2 + 1];
        Z[3 * s2 + 2] = ds * W2[3 * s2 + 2];
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        Acc* row = acc + r * chunk + col0;
#pragma unroll
        for (int s2 = 0; s2 < 9; ++s2) {
          T cv = Y[3 * r] * Z[3 * s2] + Y[3 * r + 1] * Z[3 * s2 + 1] + Y[3 * r + 2] * Z[3 * s2 + 2];
          FixAcc<T>::add(row + s2, FixAcc<T>::conv(cv));
        }
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 9 * width; q += blockDim.x) {
    int r = q / width, c = q - r * width;
    Acc v = acc[r * chunk + c];
    if (v != 0) FixAcc<T>::gadd(Sacc + (size_t)(9 * a + r) * n + start + c, v);
  }
}

// Upper off-diagonal entries of S^ from the integer accumulator (S^ = -sum / scale).
template <typename T>
__global__ void k_S_convert(int Cf, const typename FixAcc<T>::type* __restrict__ Sacc, T* __restrict__ Shat) {
  const int n = 9 * Cf;
  const T unit = (T)(-1.0 / FixAcc<T>::scale);
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const size_t row = (size_t)r * n;
    for (int c = 9 * (r / 9 + 1) + threadIdx.x; c < n; c += blockDim.x)
      Shat[row + c] = (T)Sacc[row + c] * unit;
  }
}

// Diagonal blocks from the block-Jacobi blocks D_a = U*_a - sum W V*^-1 W^T (packed),
// scaled; and the lower triangle mirrored from the upper one.
template <typename T>
__global__ void k_S_finalize(int Cf, const T* __restrict__ Dblk, const double* __restrict__ dscale,
                             T* __restrict__ Shat) {
  __shared__ T tile[32][33];
  const int n = 9 * Cf;
  const int bx = blockIdx.x, by = blockIdx.y;  // tile column, tile row
  if (bx > by) return;                          // only tiles on or below the diagonal
  // read the transposed tile (upper triangle source)
  int r0 = bx * 32, c0 = by * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < n && c < n) ? Shat[(size_t)r * n + c] : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int r = by * 32 + i, c = bx * 32 + threadIdx.x;
    if (r >= n || c >= n) continue;
    int fr = r / 9, fc = c / 9;
    if (fr == fc) {
      int ir = r - 9 * fr, ic = c - 9 * fc;
      const T* di = reinterpret_cast<const T*>(dscale + n);
      Shat[(size_t)r * n + c] = Dblk[45 * (size_t)fr + sym9(ir, ic)] * di[r] * di[c];
    } else if (c < r) {
      Shat[(size_t)r * n + c] = tile[threadIdx.x][i];
    }
  }
}

// Diagonal blocks of the upper triangle too (the mirror above writes only c <= r).
template <typename T>
__global__ void k_S_diag_upper(int Cf, const T* __restrict__ Dblk, const double* __restrict__ dscale,
                               T* __restrict__ Shat) {
  int f = blockIdx.x;
  if (f >= Cf) return;
  int n = 9 * Cf;
  for (int q = threadIdx.x; q < 81; q += blockDim.x) {
    int ir = q / 9, ic = q - 9 * ir;
    if (ic <= ir) continue;
    int r = 9 * f + ir, c = 9 * f + ic;
    const T* di = reinterpret_cast<const T*>(dscale + n);
    Shat[(size_t)r * n + c] = Dblk[45 * (size_t)f + sym9(ir, ic)] * di[r] * di[c];
  }
}

// D = sqrt(diag U*) in FP64, and 1/D in the working precision (dscale + n) so that
// per-entry work needs no FP64 division.
template <typename T>
__global__ void k_dscale(int Cf, const T* __restrict__ Ud, double* __restrict__ dscale) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int n = 9 * Cf;
  if (e >= n) return;
  int f = e / 9, i = e - 9 * f;
  double d = (double)Ud[45 * (size_t)f + sym9(i, i)];
  double sd = sqrt(d > 0.0 ? d : 1e-30);
  dscale[e] = sd;
  reinterpret_cast<T*>(dscale + n)[e] = (T)(1.0 / sd);
}

template <typename T>
cudaError_t launch_form_S(const Layout& L, const T* W, const uint8_t* act_co, const uint8_t* act_po,
                          const int* crank, const int* cam_map, const T* Vinv, const T* Ud, const T* Dblk,
                          double* dscale, int Cf, void* Sacc, T* Shat, int num_sms, cudaStream_t s) {
  if (Cf <= 0) return cudaSuccess;
  using Acc = typename FixAcc<T>::type;
  const int n = 9 * Cf;
  k_dscale<T><<<(n + 255) / 256, 256, 0, s>>>(Cf, Ud, dscale);
  cudaError_t e = cudaMemsetAsync(Sacc, 0, sizeof(Acc) * (size_t)n * n, s);
  if (e != cudaSuccess) return e;
  // column chunk: as many 9-column camera blocks as fit in ~96 KB of accumulator rows
  const int asz = (int)sizeof(Acc);
  int chunk = (96 * 1024) / (9 * asz);
  chunk = (chunk / 9) * 9;
  if (n - 9 < chunk) chunk = n - 9 > 9 ? n - 9 : 9;
  int nch = (n - 9 + chunk - 1) / chunk;
  if (nch < 1) nch = 1;
  // split every camera's observations so that about 4 blocks per SM run
  int nz = (4 * num_sms + Cf * nch - 1) / (Cf * nch);
  nz = nz < 1 ? 1 : (nz > 16 ? 16 : nz);
  size_t smem = (size_t)9 * chunk * asz;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_form_S<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  if (n > 9)
    k_form_S<T><<<dim3(Cf, nch, nz), kFormThreads, smem, s>>>(L, W, act_co, act_po, crank, cam_map, Vinv,
                                                               dscale, Cf, chunk, reinterpret_cast<Acc*>(Sacc));
  k_S_convert<T><<<n < 8 * num_sms ? n : 8 * num_sms, 256, 0, s>>>(Cf, reinterpret_cast<const Acc*>(Sacc), Shat);
  int nt = (n + 31) / 32;
  k_S_finalize<T><<<dim3(nt, nt), dim3(32, 8), 0, s>>>(Cf, Dblk, dscale, Shat);
  k_S_diag_upper<T><<<Cf, 128, 0, s>>>(Cf, Dblk, dscale, Shat);
  return cudaGetLastError();
}

int form_acc_bytes(int fp64) { return fp64 ? 8 : 4; }

// ---------------------------------------------------------------------------
// PCG on the scaled explicit system S^ x^ = b^ (b^ = D^-1 b, x = D^-1 x^) with the
// block-Jacobi preconditioner of S^.  Each block owns a contiguous slice of free
// cameras (rows) and keeps those rows of S^ in shared memory when they fit.
// ---------------------------------------------------------------------------

constexpr int kSpcgThreads = 512;

__device__ __forceinline__ bool grid_barrier2(unsigned* bar, unsigned target, int* err,
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
  return (e.load(cuda::memory_order_relaxed) & 1) == 0;
}

__device__ __forceinline__ double sum_dots2(const double* region, int slot, int G, double* red) {
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) s += region[4 * g + slot];
  return block_sum(s, red);
}

template <typename T>
size_t spcg_smem_bytes(int n, int own_max, int rows_in_smem) {
  size_t b = sizeof(double) * (2 * kSpcgThreads + 8);            // FP64 reduction scratch
  b += rows_in_smem ? sizeof(T) * (size_t)9 * own_max * n : 0;  // own rows of S^
  b += sizeof(T) * (size_t)n;                                    // p^ (full)
  b += sizeof(T) * (size_t)9 * own_max * 4;                      // x^, r^, q, b^ (owned)
  b += sizeof(T) * (size_t)81 * own_max;                         // preconditioner blocks
  return (b + 15) & ~size_t(15);
}

template <typename T>
__global__ void __launch_bounds__(kSpcgThreads, 1) k_spcg(SpcgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int n = a.n;
  const int f0 = (int)(((long long)a.Cf * bid) / G), f1 = (int)(((long long)a.Cf * (bid + 1)) / G);
  const int e0 = 9 * f0, ne = 9 * (f1 - f0);
  unsigned char* p = smem_raw;
  double* dbuf = reinterpret_cast<double*>(p);  // [2 * threads]
  double* dout = dbuf + 2 * kSpcgThreads;       // [8]
  p += sizeof(double) * (2 * kSpcgThreads + 8);
  const int cnt = min(ne, (int)blockDim.x);
  T* Srows = reinterpret_cast<T*>(p);
  p += a.rows_in_smem ? sizeof(T) * (size_t)9 * a.own_max * n : 0;
  T* ps = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)n;
  T* xo = reinterpret_cast<T*>(p);
  T* ro = xo + 9 * a.own_max;
  T* qo = ro + 9 * a.own_max;
  T* bo = qo + 9 * a.own_max;
  T* Mo = bo + 9 * a.own_max;
  const T* Sg = a.Shat + (size_t)e0 * n;
  const T* Srow_base = a.rows_in_smem ? Srows : Sg;
  unsigned epoch = 0;

  if (a.rows_in_smem)
    for (size_t q = tid; q < (size_t)ne * n; q += blockDim.x) Srows[q] = Sg[q];
  // owned preconditioner blocks of S^: D_f^-1 scaled, M^_f = diag(d) M_f diag(d)
  for (int q = tid; q < 81 * (f1 - f0); q += blockDim.x) {
    int f = q / 81, ij = q - 81 * f, i = ij / 9, j = ij - 9 * i;
    int ei = e0 + 9 * f + i, ej = e0 + 9 * f + j;
    Mo[q] = (T)((double)a.Dinv[81 * (size_t)(f0 + f) + ij] * a.dscale[ei] * a.dscale[ej]);
  }
  for (int q = tid; q < ne; q += blockDim.x) {
    xo[q] = T(0);
    T bv = (T)((double)a.b[e0 + q] / a.dscale[e0 + q]);
    ro[q] = bv;
    bo[q] = bv;
  }
  __syncthreads();
  double loc_rz = 0.0, loc_bb = 0.0;
  for (int q = tid; q < ne; q += blockDim.x) {
    int f = q / 9, i = q - 9 * f;
    T zz = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) zz += Mo[81 * f + 9 * i + k] * ro[9 * f + k];
    a.z[e0 + q] = zz;
    double rv = (double)ro[q];
    loc_rz += rv * (double)zz;
    loc_bb += rv * rv;
  }
  int dph = 0;
  auto dregion = [&](int ph) { return a.dots + (size_t)(ph & 1) * 4 * G; };
  {
    double s0, s1;
    warp0_sum2(loc_rz, loc_bb, cnt, dbuf, dout, s0, s1);
    if (tid == 0) {
      dregion(dph)[4 * bid] = s0;
      dregion(dph)[4 * bid + 1] = s1;
    }
  }
  if (!grid_barrier2(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
  double rz, bb;
  warp0_sum_slots(dregion(dph), G, 0, 1, dout + 4, rz, bb);
  ++dph;
  const double bnorm = sqrt(bb);
  int it = 0;
  double rr_last = bb, beta = 0.0;
  bool first = true;
  while (bnorm > 0.0 && it < a.max_iters) {
    // p = z (first) or z + beta p: every load of z issued before any use
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
        if (e < n) ps[e] = first ? zv[u] : zv[u] + bt * ps[e];
      }
    }
    first = false;
    __syncthreads();
    // q = S^_rows p^: one warp per row
    for (int r = warp; r < ne; r += nwarps) {
      const T* row = Srow_base + (size_t)r * n;
      T acc = T(0);
      for (int c = lane; c < n; c += 32) acc += row[c] * ps[c];
      acc = warp_sum(acc);
      if (lane == 0) qo[r] = acc;
    }
    __syncthreads();
    double loc_pq = 0.0;
    for (int q = tid; q < ne; q += blockDim.x) loc_pq += (double)ps[e0 + q] * (double)qo[q];
    {
      double s0, s1;
      warp0_sum2(loc_pq, 0.0, cnt, dbuf, dout, s0, s1);
      if (tid == 0) dregion(dph)[4 * bid + 2] = s0;
    }
    if (!grid_barrier2(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double pq, unused;
    warp0_sum_slots(dregion(dph), G, 2, 2, dout + 4, pq, unused);
    ++dph;
    if (!(pq > 0.0) || !isfinite(pq)) {
      if (bid == 0 && tid == 0) atomicOr(a.err, 2);
      break;
    }
    double alpha = rz / pq;
    for (int q = tid; q < ne; q += blockDim.x) {
      xo[q] = (T)((double)xo[q] + alpha * (double)ps[e0 + q]);
      ro[q] = (T)((double)ro[q] - alpha * (double)qo[q]);
    }
    __syncthreads();
    double loc_rr = 0.0, loc_rz2 = 0.0;
    for (int q = tid; q < ne; q += blockDim.x) {
      int f = q / 9, i = q - 9 * f;
      T zz = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) zz += Mo[81 * f + 9 * i + k] * ro[9 * f + k];
      a.z[e0 + q] = zz;
      double rv = (double)ro[q];
      loc_rr += rv * rv;
      loc_rz2 += rv * (double)zz;
    }
    {
      double s0, s1;
      warp0_sum2(loc_rr, loc_rz2, cnt, dbuf, dout, s0, s1);
      if (tid == 0) {
        dregion(dph)[4 * bid] = s0;
        dregion(dph)[4 * bid + 1] = s1;
      }
    }
    if (!grid_barrier2(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double rr, rz2;
    warp0_sum_slots(dregion(dph), G, 0, 1, dout + 4, rr, rz2);
    ++dph;
    ++it;
    rr_last = rr;
    if (sqrt(rr) <= a.tol * bnorm) break;
    beta = rz2 / rz;
    rz = rz2;
  }
  for (int q = tid; q < ne; q += blockDim.x) a.x[e0 + q] = (T)((double)xo[q] / a.dscale[e0 + q]);
  if (bid == 0 && tid == 0) {
    a.sc->pcg_iters = it;
    a.sc->pcg_bnorm = bnorm;
    a.sc->pcg_rel_res = bnorm > 0.0 ? sqrt(rr_last) / bnorm : 0.0;
  }
}

template <typename T>
const void* spcg_kernel_ptr() {
  return reinterpret_cast<const void*>(&k_spcg<T>);
}

template <typename T>
cudaError_t launch_spcg(const SpcgArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<SpcgArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel(spcg_kernel_ptr<T>(), dim3(grid), dim3(kSpcgThreads), args, smem, s);
}

int spcg_threads() { return kSpcgThreads; }

// ---------------------------------------------------------------------------
// Point back-substitution dp = V*^-1 (-g_p - sum_k W_k^T dc_c(k)), W recomputed,
// and the point part of the predicted decrease.  One thread per point.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_backsub_pts(Layout L, ModelParams mp, const T* __restrict__ camw, const T* __restrict__ ptsw,
                              const uint8_t* __restrict__ act_po, const uint8_t* __restrict__ pt_act,
                              const int* __restrict__ crank, const T* __restrict__ x,
                              const T* __restrict__ Vinv, const T* __restrict__ V, const T* __restrict__ gp,
                              double lambda, T* __restrict__ dp, double* __restrict__ pred_parts) {
  __shared__ double red[32];
  double pred = 0.0;
  const T* po_uv = reinterpret_cast<const T*>(L.po_uvw);
  const T* po_tau = reinterpret_cast<const T*>(L.po_tauw);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < L.P; p += gridDim.x * blockDim.x) {
    if (!pt_act[p]) {
      dp[3 * (size_t)p] = dp[3 * (size_t)p + 1] = dp[3 * (size_t)p + 2] = T(0);
      continue;
    }
    const T* X = ptsw + 4 * (size_t)p;
    double t0 = -(double)gp[3 * (size_t)p], t1 = -(double)gp[3 * (size_t)p + 1], t2 = -(double)gp[3 * (size_t)p + 2];
    for (int k = L.pt_off[p]; k < L.pt_off[p + 1]; ++k) {
      if (!act_po[k]) continue;
      int c = L.po_cam[k];
      int cr = crank[c];
      if (cr < 0) continue;
      T cw[kCamStride];
      load_cam_rec(camw, c, cw);
      T W[27];
      obs_W(cw, X, po_uv[2 * (size_t)k], po_uv[2 * (size_t)k + 1], po_tau[k], mp, W);
      const T* xv = x + 9 * (size_t)cr;
      T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        s0 += W[3 * q] * xv[q];
        s1 += W[3 * q + 1] * xv[q];
        s2 += W[3 * q + 2] * xv[q];
      }
      t0 -= (double)s0;
      t1 -= (double)s1;
      t2 -= (double)s2;
    }
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
  double s = block_sum(pred, red);
  if (threadIdx.x == 0) pred_parts[blockIdx.x] = s;
}

template <typename T>
cudaError_t launch_backsub_pts(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                               const uint8_t* act_po, const uint8_t* pt_act, const int* crank, const T* x,
                               const T* Vinv, const T* V, const T* gp, double lambda, T* dp,
                               double* pred_parts, int grid, cudaStream_t s) {
  k_backsub_pts<T><<<grid, 256, 0, s>>>(L, mp, camw, ptsw, act_po, pt_act, crank, x, Vinv, V, gp, lambda, dp,
                                         pred_parts);
  return cudaGetLastError();
}

#define BAB_SINST(T)                                                                                   \
  template cudaError_t launch_form_S<T>(const Layout&, const T*, const uint8_t*, const uint8_t*,      \
                                        const int*, const int*, const T*, const T*, const T*, double*, \
                                        int, void*, T*, int, cudaStream_t);                            \
  template size_t spcg_smem_bytes<T>(int, int, int);                                                   \
  template const void* spcg_kernel_ptr<T>();                                                           \
  template cudaError_t launch_spcg<T>(const SpcgArgs<T>&, int, size_t, cudaStream_t);                  \
  template cudaError_t launch_backsub_pts<T>(const Layout&, const ModelParams&, const T*, const T*,    \
                                             const uint8_t*, const uint8_t*, const int*, const T*,     \
                                             const T*, const T*, const T*, double, T*, double*, int,   \
                                             cudaStream_t);
BAB_SINST(float)
BAB_SINST(double)

}  // namespace bab
