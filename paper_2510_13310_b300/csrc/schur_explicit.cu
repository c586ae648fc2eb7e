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
// (the co-visibility runs), so each block is summed by one warp in registers in
// a fixed order: no atomics, bit-reproducible.  The diagonal blocks come from the
// block-Jacobi pass (U* - sum W V*^-1 W^T) and the lower triangle is mirrored.
#include <cuda/atomic>

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
__global__ void __launch_bounds__(kYRows) k_form_Y(int N, const int* __restrict__ po_cam,
                                                  const int* __restrict__ po_pt, const T* __restrict__ W,
                                                  const T* __restrict__ Vinv, const int* __restrict__ crank,
                                                  const double* __restrict__ dscale, int Cf,
                                                  T* __restrict__ Y) {
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
    const int a = crank[po_cam[k]];
    if (a < 0) {
#pragma unroll
      for (int q = 0; q < 27; ++q) y[q] = T(0);
    } else {
      const T* dinv = reinterpret_cast<const T*>(dscale + 9 * Cf) + 9 * a;
      const T* vi = Vinv + 6 * (size_t)po_pt[k];
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
  uint4* dst = reinterpret_cast<uint4*>(Y + kWStride * (size_t)k0);
  for (int i = threadIdx.x; i < rows * kVec; i += kYRows) dst[i] = sb[i];
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
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1)
    k_form_S_runs(int n_runs, const int4* __restrict__ runs, const int2* __restrict__ pairs,
                  const T* __restrict__ Y, const int* __restrict__ crank, int Cf, T* __restrict__ Shat) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = 9 * Cf;
  for (int ri = gw; ri < n_runs; ri += nw) {
    const int4 rn = runs[ri];  // (camera i, camera j, first pair, pair count)
    const int a = crank[rn.x], b = crank[rn.y];
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
      load_row27<T>(Y + kWStride * (size_t)pr.x, y1);
      load_row27<T>(Y + kWStride * (size_t)pr.y, y2);
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
        Shat[(size_t)(9 * a + r) * n + 9 * b + s2] = -v[j];
      }
    }
  }
}

// The same blocks with one lane per run, for scenes with very many short runs
// (every camera pair sharing a few dozen points): each lane accumulates its run
// in registers and writes the 81 entries itself, so no cross-lane reduction is
// needed; lanes of a warp take consecutive runs of similar length.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1)
    k_form_S_lanes(int n_runs, const int4* __restrict__ runs, const int2* __restrict__ pairs,
                   const T* __restrict__ Y, const int* __restrict__ crank, int Cf, T* __restrict__ Shat) {
  const int n = 9 * Cf;
  for (int ri = blockIdx.x * blockDim.x + threadIdx.x; ri < n_runs; ri += gridDim.x * blockDim.x) {
    const int4 rn = runs[ri];
    const int a = crank[rn.x], b = crank[rn.y];
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
      load_row27<T>(Y + kWStride * (size_t)pr.y, y2);
      const T* y1 = Y + kWStride * (size_t)pr.x;
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
      for (int s2 = 0; s2 < 9; ++s2) Shat[(size_t)(9 * a + r) * n + 9 * b + s2] = -acc[9 * r + s2];
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
cudaError_t launch_form_S(const Layout& L, int n_runs, const int4* runs, const int2* pairs, const T* W,
                          const T* Vinv, const int* crank, const T* Ud, const T* Dblk, double* dscale,
                          int Cf, T* Y, T* Shat, bool lanes, int num_sms, cudaStream_t s) {
  if (Cf <= 0) return cudaSuccess;
  const int n = 9 * Cf;
  k_dscale<T><<<(n + 255) / 256, 256, 0, s>>>(Cf, Ud, dscale);
  if (L.N > 0) k_form_Y<T><<<(L.N + kYRows - 1) / kYRows, kYRows, 0, s>>>(L.N, L.po_cam, L.po_pt, W, Vinv, crank, dscale, Cf, Y);
  cudaError_t e = cudaMemsetAsync(Shat, 0, sizeof(T) * (size_t)n * n, s);
  if (e != cudaSuccess) return e;
  if (n_runs > 0) {
    const int wpb = 4;  // warps per 128-thread block
    if (lanes) {
      // many short runs: one lane per run
      int grid = (n_runs + 127) / 128;
      if (grid > 16 * num_sms) grid = 16 * num_sms;
      k_form_S_lanes<T><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat);
    } else {
      int grid = (n_runs + wpb - 1) / wpb;
      if (grid > 32 * num_sms) grid = 32 * num_sms;
      k_form_S_runs<T><<<grid, 128, 0, s>>>(n_runs, runs, pairs, Y, crank, Cf, Shat);
    }
  }
  int nt = (n + 31) / 32;
  k_S_finalize<T><<<dim3(nt, nt), dim3(32, 8), 0, s>>>(Cf, Dblk, dscale, Shat);
  k_S_diag_upper<T><<<Cf, 128, 0, s>>>(Cf, Dblk, dscale, Shat);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// PCG on the scaled explicit system S^ x^ = b^ (b^ = D^-1 b, x = D^-1 x^) with the
// block-Jacobi preconditioner of S^.  Each block owns a contiguous slice of free
// cameras (rows) and keeps those rows of S^ in shared memory when they fit.
// ---------------------------------------------------------------------------

constexpr int kSpcgThreads = 512;

// Cross-block reductions without a separate barrier.  Each block publishes its
// FP64 partials as 64-bit words whose 4 low mantissa bits are replaced by the
// reduction's epoch tag (a relative change below 2^-48), with a release store
// after its other global writes; warp 0 of every block then polls the G slots
// until every tag matches, and sums them in a fixed order.
// Seeing all tags is the barrier: writes a block made before publishing are
// visible after it.  Slots alternate between two sets by epoch parity, so a
// block that is one reduction ahead never overwrites a slot still being read.
__device__ __forceinline__ unsigned long long tag_value(double v, unsigned tag) {
  return ((unsigned long long)__double_as_longlong(v) & ~0xFull) | (unsigned long long)(tag & 0xFu);
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Called by warp 0 only (all lanes), after a __syncthreads that ordered the
// block's global writes.  mine: this block's K partials (lane 0's values are
// published).  out: the K sums over the G blocks (every lane).  Each lane polls
// its slots g = lane + 32 m in batches of 8 (all loads of a batch in flight at
// once) until every tag matches; an acquire fence then orders the block's later
// reads after the other blocks' published writes.  false on timeout.
template <int K>
__device__ bool warp0_tagged_allreduce(unsigned long long* slots, int G, int bid, unsigned epoch,
                                       const double (&mine)[K], double (&out)[K], long long timeout_ns) {
  const int lane = threadIdx.x & 31;
  unsigned long long* set = slots + (size_t)(epoch & 1u) * 4 * G;
  const unsigned tag = epoch & 0xFu;
  if (lane == 0) {
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) st_release_u64(&set[4 * bid + k], tag_value(mine[k], tag));
  }
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  bool ok = true;
  const uint64_t t0 = globaltimer_ns();
  for (int base = 0; base < G; base += 256) {
    unsigned long long v[K][8];
    for (;;) {
      bool ready = true;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int g = base + lane + 32 * m;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          v[k][m] = g < G ? ld_relaxed_u64(&set[4 * g + k]) : (unsigned long long)tag;
          ready &= (unsigned)(v[k][m] & 0xFull) == tag;
        }
      }
      if (__all_sync(0xffffffffu, ready)) break;
      if ((long long)(globaltimer_ns() - t0) > timeout_ns) {
        ok = false;
        break;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (base + lane + 32 * m < G) acc[k] += __longlong_as_double((long long)(v[k][m] & ~0xFull));
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = warp_sum(acc[k]);
  return __all_sync(0xffffffffu, ok);
}

// alpha = (r, z) / (p, q) and beta = (r', z') / (r, z) from the FP64 dot products:
// the FP32 path needs them to FP32 accuracy only (x, r, p are FP32 vectors), and an
// FP64 division is a long dependent chain on B300; the FP64 path divides in FP64.
template <typename T>
__device__ __forceinline__ double spcg_ratio(double num, double den) {
  if constexpr (sizeof(T) == 4) return (double)__fdiv_rn((float)num, (float)den);
  else return num / den;
}

template <typename T>
__host__ __device__ inline int spcg_row_stride(int n) {
  return sizeof(T) == 4 ? (n + 3) & ~3 : n;  // FP32 rows padded for 16-byte vector loads
}

template <typename T>
size_t spcg_smem_bytes(int n, int own_max, int rows_in_smem) {
  const int ns = spcg_row_stride<T>(n);
  size_t b = sizeof(double) * 16;                                   // broadcast scalars
  b += rows_in_smem ? sizeof(T) * (size_t)9 * own_max * ns : 0;    // own rows of S^
  b += sizeof(T) * (size_t)ns;                                      // p^ (full)
  b += sizeof(T) * (size_t)9 * own_max * 5;                         // x^, r^, q, b^, z (owned)
  b += sizeof(T) * (size_t)81 * own_max;                            // preconditioner blocks
  return (b + 15) & ~size_t(15);
}

// Dot products of the owned slice by warp 0 (FP64 accumulation, fixed order).
template <typename T>
__device__ __forceinline__ double warp0_dot(const T* a, const T* b, int ne) {
  double s = 0.0;
  for (int q = threadIdx.x; q < ne; q += 32) s += (double)a[q] * (double)b[q];
  return warp_sum(s);
}

// Persistent PCG on the scaled system: standard preconditioned CG (x0 = 0,
// block-Jacobi M^), two cross-block reductions per iteration (p^T q, then
// r^T r and r^T z) and no other grid synchronisation.  alpha, beta and the
// stopping test are formed by one thread (FP64 division is scarce) and
// broadcast through shared memory.
template <typename T>
__global__ void __launch_bounds__(kSpcgThreads, 1) k_spcg(SpcgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int n = a.n, ns = spcg_row_stride<T>(n);
  const int f0 = (int)(((long long)a.Cf * bid) / G), f1 = (int)(((long long)a.Cf * (bid + 1)) / G);
  const int e0 = 9 * f0, ne = 9 * (f1 - f0);
  unsigned char* p = smem_raw;
  double* sb = reinterpret_cast<double*>(p);  // [16]
  p += sizeof(double) * 16;
  T* Srows = reinterpret_cast<T*>(p);
  p += a.rows_in_smem ? sizeof(T) * (size_t)9 * a.own_max * ns : 0;
  T* ps = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)ns;
  T* xo = reinterpret_cast<T*>(p);
  T* ro = xo + 9 * a.own_max;
  T* qo = ro + 9 * a.own_max;
  T* bo = qo + 9 * a.own_max;
  T* zo = bo + 9 * a.own_max;
  T* Mo = zo + 9 * a.own_max;
  const T* Sg = a.Shat + (size_t)e0 * n;
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(a.dots);
  unsigned epoch = 0;
  const T* dinv = reinterpret_cast<const T*>(a.dscale + n);

  if (a.rows_in_smem) {
    // eight loads per lane in flight: the block's rows come from HBM once per solve
    for (int r = warp; r < ne; r += nwarps) {
      const T* src = Sg + (size_t)r * n;
      T* dst = Srows + (size_t)r * ns;
      for (int c0 = 0; c0 < ns; c0 += 256) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + 32 * u + lane;
          v[u] = c < n ? src[c] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + 32 * u + lane;
          if (c < ns) dst[c] = v[u];
        }
      }
    }
  }
  for (int c = n + tid; c < ns; c += blockDim.x) ps[c] = T(0);
  // owned preconditioner blocks of S^: D_f^-1 scaled, M^_f = diag(d) M_f diag(d)
  for (int q = tid; q < 81 * (f1 - f0); q += blockDim.x) {
    int f = q / 81, ij = q - 81 * f, i = ij / 9, j = ij - 9 * i;
    int ei = e0 + 9 * f + i, ej = e0 + 9 * f + j;
    Mo[q] = (T)((double)a.Dinv[81 * (size_t)(f0 + f) + ij] * a.dscale[ei] * a.dscale[ej]);
  }
  for (int q = tid; q < ne; q += blockDim.x) {
    xo[q] = T(0);
    T bv = (T)((double)a.b[e0 + q] * (double)dinv[e0 + q]);
    ro[q] = bv;
    bo[q] = bv;
  }
  __syncthreads();
  for (int q = tid; q < ne; q += blockDim.x) {
    int f = q / 9, i = q - 9 * f;
    T zz = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) zz += Mo[81 * f + 9 * i + k] * ro[9 * f + k];
    a.z[e0 + q] = zz;
    zo[q] = zz;
  }
  __syncthreads();
  if (warp == 0) {
    const double mine[2] = {warp0_dot(ro, zo, ne), warp0_dot(ro, ro, ne)};
    double tot[2];
    const bool ok = warp0_tagged_allreduce<2>(slots, G, bid, ++epoch, mine, tot, a.timeout_ns);
    if (lane == 0) {
      sb[0] = tot[0];
      sb[1] = tot[1];
      sb[2] = sqrt(tot[1]);
      sb[7] = ok ? 1.0 : 0.0;
      if (!ok) atomicOr(a.err, 1);
    }
  } else {
    ++epoch;
  }
  __syncthreads();
  if (sb[7] == 0.0) return;
  double rz = sb[0];
  const double bnorm = sb[2];
  const double stop_rr = (a.tol * bnorm) * (a.tol * bnorm);
  int it = 0;
  double rr_last = sb[1];
  T beta = T(0);
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
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = base + u * blockDim.x + tid;
        if (e < n) ps[e] = first ? zv[u] : zv[u] + beta * ps[e];
      }
    }
    first = false;
    __syncthreads();
    // q = S^_rows p^: one warp per row
    if constexpr (sizeof(T) == 4) {
      if (a.rows_in_smem) {
        const float4* p4 = reinterpret_cast<const float4*>(ps);
        for (int r = warp; r < ne; r += nwarps) {
          const float4* row = reinterpret_cast<const float4*>(Srows + (size_t)r * ns);
          float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
          for (int c = lane; c < ns / 4; c += 32) {
            const float4 sv = row[c], pv = p4[c];
            c0 += sv.x * pv.x;
            c1 += sv.y * pv.y;
            c2 += sv.z * pv.z;
            c3 += sv.w * pv.w;
          }
          const float acc = warp_sum((c0 + c1) + (c2 + c3));
          if (lane == 0) qo[r] = acc;
        }
      }
    }
    if (sizeof(T) != 4 || !a.rows_in_smem) {
      const T* base = a.rows_in_smem ? Srows : Sg;
      const int ld = a.rows_in_smem ? ns : n;
      for (int r = warp; r < ne; r += nwarps) {
        const T* row = base + (size_t)r * ld;
        T acc = T(0);
        for (int c = lane; c < n; c += 32) acc += row[c] * ps[c];
        acc = warp_sum(acc);
        if (lane == 0) qo[r] = acc;
      }
    }
    __syncthreads();
    if (warp == 0) {
      const double mine[1] = {warp0_dot(ps + e0, qo, ne)};
      double tot[1];
      const bool ok = warp0_tagged_allreduce<1>(slots, G, bid, ++epoch, mine, tot, a.timeout_ns);
      if (lane == 0) {
        const double pq = tot[0];
        const bool fine = ok && pq > 0.0 && isfinite(pq);
        sb[3] = fine ? spcg_ratio<T>(rz, pq) : 0.0;
        sb[7] = fine ? 1.0 : 0.0;
        if (!ok) atomicOr(a.err, 1);
        else if (!fine && bid == 0) atomicOr(a.err, 2);
      }
    } else {
      ++epoch;
    }
    __syncthreads();
    if (sb[7] == 0.0) break;
    const double alpha = sb[3];
    for (int q = tid; q < ne; q += blockDim.x) {
      if constexpr (sizeof(T) == 4) {
        xo[q] = fmaf((float)alpha, ps[e0 + q], xo[q]);
        ro[q] = fmaf(-(float)alpha, qo[q], ro[q]);
      } else {
        xo[q] = (T)((double)xo[q] + alpha * (double)ps[e0 + q]);
        ro[q] = (T)((double)ro[q] - alpha * (double)qo[q]);
      }
    }
    __syncthreads();
    for (int q = tid; q < ne; q += blockDim.x) {
      int f = q / 9, i = q - 9 * f;
      T zz = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) zz += Mo[81 * f + 9 * i + k] * ro[9 * f + k];
      a.z[e0 + q] = zz;
      zo[q] = zz;
    }
    __syncthreads();
    if (warp == 0) {
      const double mine[2] = {warp0_dot(ro, ro, ne), warp0_dot(ro, zo, ne)};
      double tot[2];
      const bool ok = warp0_tagged_allreduce<2>(slots, G, bid, ++epoch, mine, tot, a.timeout_ns);
      if (lane == 0) {
        sb[4] = tot[0];
        sb[5] = tot[0] <= stop_rr ? 1.0 : 0.0;
        sb[6] = rz != 0.0 ? spcg_ratio<T>(tot[1], rz) : 0.0;
        sb[0] = tot[1];
        sb[7] = ok ? 1.0 : 0.0;
        if (!ok) atomicOr(a.err, 1);
      }
    } else {
      ++epoch;
    }
    __syncthreads();
    if (sb[7] == 0.0) break;
    ++it;
    rr_last = sb[4];
    if (sb[5] != 0.0) break;
    beta = (T)sb[6];
    rz = sb[0];
  }
  for (int q = tid; q < ne; q += blockDim.x) a.x[e0 + q] = (T)((double)xo[q] * (double)dinv[e0 + q]);
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
// Point back-substitution dp = V*^-1 (-g_p - sum_k W_k^T dc_c(k)), with the
// stored W rows when there are any (explicit system), else W recomputed; and the
// point part of the predicted decrease.  One thread per point.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_backsub_pts(Layout L, ModelParams mp, const T* __restrict__ camw, const T* __restrict__ ptsw,
                              const uint8_t* __restrict__ act_po, const uint8_t* __restrict__ pt_act,
                              const int* __restrict__ crank, const T* __restrict__ x,
                              const T* __restrict__ Vinv, const T* __restrict__ V, const T* __restrict__ gp,
                              const T* __restrict__ Wst, double lambda, T* __restrict__ dp,
                              double* __restrict__ pred_parts) {
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
      T W[27];
      if (Wst) {
        load_row27<T>(Wst + kWStride * (size_t)k, W);
      } else {
        T cw[kCamStride];
        load_cam_rec(camw, c, cw);
        obs_W(cw, X, po_uv[2 * (size_t)k], po_uv[2 * (size_t)k + 1], po_tau[k], mp, W);
      }
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
                               const T* Vinv, const T* V, const T* gp, const T* Wst, double lambda, T* dp,
                               double* pred_parts, int grid, cudaStream_t s) {
  k_backsub_pts<T><<<grid, 256, 0, s>>>(L, mp, camw, ptsw, act_po, pt_act, crank, x, Vinv, V, gp, Wst, lambda,
                                         dp, pred_parts);
  return cudaGetLastError();
}

#define BAB_SINST(T)                                                                                   \
  template cudaError_t launch_form_S<T>(const Layout&, int, const int4*, const int2*, const T*,        \
                                        const T*, const int*, const T*, const T*, double*, int, T*, T*, \
                                        bool, int, cudaStream_t);                                      \
  template size_t spcg_smem_bytes<T>(int, int, int);                                                   \
  template const void* spcg_kernel_ptr<T>();                                                           \
  template cudaError_t launch_spcg<T>(const SpcgArgs<T>&, int, size_t, cudaStream_t);                  \
  template cudaError_t launch_backsub_pts<T>(const Layout&, const ModelParams&, const T*, const T*,    \
                                             const uint8_t*, const uint8_t*, const int*, const T*,     \
                                             const T*, const T*, const T*, const T*, double, T*,       \
                                             double*, int, cudaStream_t);
BAB_SINST(float)
BAB_SINST(double)

}  // namespace bab
