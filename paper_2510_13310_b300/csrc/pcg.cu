// pcg.cu -- step (d): persistent block-Jacobi PCG on the reduced camera system
// with the point back-substitution (Sec. 4.2 step 3: "preconditioned conjugate
// gradient", then scatter of the compact update).
//
// One cooperative launch runs the whole solve.  The Schur matvec
//   S p = U* p - sum_pts W_p V*_p^-1 (sum_k W_k^T p_c(k))
// streams W once per iteration in point order, one tile of whole points at a
// time.  Each tile (W rows, static metadata and V*^-1 rows) arrives in shared
// memory through bulk asynchronous copies (TMA) into a double buffer, so the
// next tile loads while the current one is computed:
//   1. per observation  a_k = W_k^T p_c(k)
//   2. per point        z_p = V*_p^-1 sum_k a_k
//   3. per observation  v_k = W_k z_p(k)
//   4. per camera run   y_c += sum_k v_k    (the tile's observations pre-sorted
//                                             by camera: fixed-order sums)
// Each block owns a contiguous slice of the free cameras for the vector
// updates and reduces the blocks' partial y in a fixed order after a grid
// barrier.  Dot products are FP64, summed in the same order by every block,
// so every block takes the same convergence decision, and no floating-point
// atomics are used anywhere: runs are bit-reproducible.  Grid barriers and
// mbarrier waits give up after a time limit and raise an error flag.
#include <cuda/atomic>

#include "internal.h"
#include "tma.cuh"

namespace bab {

constexpr int kPcgThreads = 256;
constexpr int kVtRows = kTileObs + 2;

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__host__ __device__ __forceinline__ int pad16(int x) { return (x + 15) & ~15; }

__host__ __device__ __forceinline__ int tile_meta_bytes(int n_obs, int n_pts, int n_runs) {
  return 4 * pad4(n_obs) + 4 * pad4(n_pts + 1) + 4 * pad4(n_runs) + pad16(n_obs);
}
constexpr int kMetaBytes = 4 * kTileObs + 4 * (kTileObs + 4) + 4 * kTileObs + kTileObs;

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
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  cuda::atomic_ref<int, cuda::thread_scope_device> e(*err);
  return (e.load(cuda::memory_order_relaxed) & 1) == 0;  // bit 0: a wait timed out
}

template <typename T>
struct PcgSmem {
  T* W[2];
  unsigned char* M[2];
  T* V[2];
  uint64_t* mbar;
  TileDesc* desc;
  double* dred;
  T* vb;
  T* zt;
  T* osum;
  T* xs;
  T* ys;
  int* lid;
  int* crank;
};

template <typename T>
size_t pcg_smem_bytes(int n, int C, int stages) {
  size_t b = 0;
  b += (size_t)stages * sizeof(T) * kTileObs * 27;  // W rows
  b += (size_t)stages * kMetaBytes;                 // metadata
  b += (size_t)stages * sizeof(T) * kVtRows * 6;    // V*^-1 rows
  b += 2 * sizeof(uint64_t) + 2 * sizeof(TileDesc); // mbarriers, descriptors
  b += sizeof(double) * 32;                         // reduction scratch
  b += sizeof(T) * kTileObs * 9;                    // vb
  b += sizeof(T) * kTileObs * 3;                    // zt
  b += sizeof(T) * kPcgThreads;                     // osum
  b += sizeof(T) * (size_t)n * 2;                   // xs, ys
  b += sizeof(int) * kTileObs;                      // lid
  b += sizeof(int) * (size_t)C;                     // crank
  return (b + 15) & ~size_t(15);
}

template <typename T>
__device__ PcgSmem<T> carve(unsigned char* base, int n, int C, int stages) {
  PcgSmem<T> s;
  unsigned char* p = base;
  for (int i = 0; i < 2; ++i) s.W[i] = reinterpret_cast<T*>(p + (size_t)(i < stages ? i : 0) * sizeof(T) * kTileObs * 27);
  p += (size_t)stages * sizeof(T) * kTileObs * 27;
  for (int i = 0; i < 2; ++i) s.M[i] = p + (size_t)(i < stages ? i : 0) * kMetaBytes;
  p += (size_t)stages * kMetaBytes;
  for (int i = 0; i < 2; ++i) s.V[i] = reinterpret_cast<T*>(p + (size_t)(i < stages ? i : 0) * sizeof(T) * kVtRows * 6);
  p += (size_t)stages * sizeof(T) * kVtRows * 6;
  s.mbar = reinterpret_cast<uint64_t*>(p);
  p += 2 * sizeof(uint64_t);
  s.desc = reinterpret_cast<TileDesc*>(p);
  p += 2 * sizeof(TileDesc);
  s.dred = reinterpret_cast<double*>(p);
  p += sizeof(double) * 32;
  s.vb = reinterpret_cast<T*>(p);
  p += sizeof(T) * kTileObs * 9;
  s.zt = reinterpret_cast<T*>(p);
  p += sizeof(T) * kTileObs * 3;
  s.osum = reinterpret_cast<T*>(p);
  p += sizeof(T) * kPcgThreads;
  s.xs = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)n;
  s.ys = reinterpret_cast<T*>(p);
  p += sizeof(T) * (size_t)n;
  s.lid = reinterpret_cast<int*>(p);
  p += sizeof(int) * kTileObs;
  s.crank = reinterpret_cast<int*>(p);
  return s;
}

// thread 0: start the bulk copies of tile t into stage s
template <typename T>
__device__ void issue_tile(const PcgArgs<T>& a, PcgSmem<T>& sm, int t, int s) {
  TileDesc d = a.descs[t];
  sm.desc[s] = d;
  unsigned wbytes = (unsigned)(pad4(d.n_obs) * 27 * sizeof(T));
  unsigned mbytes = (unsigned)tile_meta_bytes(d.n_obs, d.n_pts, d.n_runs);
  int pb2 = d.pt_begin & ~1, pe2 = (d.pt_begin + d.n_pts + 1) & ~1;
  unsigned vbytes = (unsigned)((pe2 - pb2) * 6 * sizeof(T));
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sm.mbar[s], wbytes + mbytes + vbytes);
  if (wbytes) bulk_g2s(sm.W[s], a.W + 27 * (size_t)d.w_row, wbytes, &sm.mbar[s]);
  bulk_g2s(sm.M[s], a.meta + d.meta_off, mbytes, &sm.mbar[s]);
  bulk_g2s(sm.V[s], a.Vinv + 6 * (size_t)pb2, vbytes, &sm.mbar[s]);
}

// Per-tile work.  MODE 0: Schur matvec contribution into ys.  MODE 1: point
// back-substitution dp = V*^-1 (-g_p - sum_k W_k^T x) and the point part of the
// predicted decrease, returned through pred.
template <typename T, int MODE>
__device__ void tile_compute(const PcgArgs<T>& a, PcgSmem<T>& sm, int s, double& pred) {
  const int tid = threadIdx.x;
  const TileDesc d = sm.desc[s];
  const int nobs = d.n_obs, npts = d.n_pts, nruns = d.n_runs;
  const int* camS = reinterpret_cast<const int*>(sm.M[s]);
  const int* poffS = camS + pad4(nobs);
  const unsigned* runsS = reinterpret_cast<const unsigned*>(poffS + pad4(npts + 1));
  const uint8_t* cpermS = reinterpret_cast<const uint8_t*>(runsS + pad4(nruns));
  const T* Wt = sm.W[s];
  const T* Vt = sm.V[s] + 6 * (d.pt_begin - (d.pt_begin & ~1));
  T* vb = sm.vb;
  // 1. a_k = W_k^T x_c(k)
  for (int i = tid; i < nobs; i += blockDim.x) {
    int cr = sm.crank[camS[i]];
    T s0 = T(0), s1 = T(0), s2 = T(0);
    if (cr >= 0) {
      const T* w = Wt + 27 * i;
      const T* xv = sm.xs + 9 * cr;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        T xq = xv[q];
        s0 += w[3 * q] * xq;
        s1 += w[3 * q + 1] * xq;
        s2 += w[3 * q + 2] * xq;
      }
    }
    vb[9 * i] = s0;
    vb[9 * i + 1] = s1;
    vb[9 * i + 2] = s2;
  }
  __syncthreads();
  if (MODE == 0) {
    // 2. z_p = V*^-1 sum_k a_k
    for (int j = tid; j < npts; j += blockDim.x) {
      T s0 = T(0), s1 = T(0), s2 = T(0);
      for (int i = poffS[j]; i < poffS[j + 1]; ++i) {
        s0 += vb[9 * i];
        s1 += vb[9 * i + 1];
        s2 += vb[9 * i + 2];
        sm.lid[i] = j;
      }
      const T* v = Vt + 6 * j;
      sm.zt[3 * j] = v[0] * s0 + v[1] * s1 + v[2] * s2;
      sm.zt[3 * j + 1] = v[1] * s0 + v[3] * s1 + v[4] * s2;
      sm.zt[3 * j + 2] = v[2] * s0 + v[4] * s1 + v[5] * s2;
    }
    __syncthreads();
    // 3. v_k = W_k z_p(k)
    for (int i = tid; i < nobs; i += blockDim.x) {
      T* o = vb + 9 * i;
      if (sm.crank[camS[i]] < 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) o[q] = T(0);
        continue;
      }
      const T* w = Wt + 27 * i;
      int j = sm.lid[i];
      T z0 = sm.zt[3 * j], z1 = sm.zt[3 * j + 1], z2 = sm.zt[3 * j + 2];
#pragma unroll
      for (int q = 0; q < 9; ++q) o[q] = w[3 * q] * z0 + w[3 * q + 1] * z1 + w[3 * q + 2] * z2;
    }
    __syncthreads();
    // 4. per camera run (distinct cameras in a tile): y_c += sum v_k
    for (int r = tid; r < nruns; r += blockDim.x) {
      unsigned u = runsS[r];
      int cr = sm.crank[u >> 8];
      if (cr < 0) continue;
      int jb = (int)(u & 255u);
      int je = r + 1 < nruns ? (int)(runsS[r + 1] & 255u) : nobs;
      T acc[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q] = T(0);
      for (int j = jb; j < je; ++j) {
        const T* o = vb + 9 * cpermS[j];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] += o[q];
      }
      T* yv = sm.ys + 9 * cr;
#pragma unroll
      for (int q = 0; q < 9; ++q) yv[q] += acc[q];
    }
  } else {
    // back-substitution for the tile's points
    for (int j = tid; j < npts; j += blockDim.x) {
      size_t p = (size_t)d.pt_begin + j;
      double t0 = -(double)a.gp[3 * p], t1 = -(double)a.gp[3 * p + 1], t2 = -(double)a.gp[3 * p + 2];
      for (int i = poffS[j]; i < poffS[j + 1]; ++i) {
        t0 -= (double)vb[9 * i];
        t1 -= (double)vb[9 * i + 1];
        t2 -= (double)vb[9 * i + 2];
      }
      const T* v = Vt + 6 * j;
      T d0 = (T)(v[0] * t0 + v[1] * t1 + v[2] * t2);
      T d1 = (T)(v[1] * t0 + v[3] * t1 + v[4] * t2);
      T d2 = (T)(v[2] * t0 + v[4] * t1 + v[5] * t2);
      a.dp[3 * p] = d0;
      a.dp[3 * p + 1] = d1;
      a.dp[3 * p + 2] = d2;
      const T* vv = a.V + 6 * p;
      double dd[3] = {(double)d0, (double)d1, (double)d2};
      double dg[3] = {fmin(fmax((double)vv[0], 1e-6), 1e32), fmin(fmax((double)vv[3], 1e-6), 1e32),
                      fmin(fmax((double)vv[5], 1e-6), 1e32)};
      for (int i = 0; i < 3; ++i) pred += dd[i] * (a.lambda * dg[i] * dd[i] - (double)a.gp[3 * p + i]);
    }
  }
}

// Walk this block's tiles (t = blockIdx.x + j G) through the copy pipeline.
// `issued` / `consumed` count tiles over the whole launch; stage = count % stages.
template <typename T, int MODE>
__device__ bool walk_tiles(const PcgArgs<T>& a, PcgSmem<T>& sm, int& issued, int& consumed,
                           bool prologue_done, double& pred) {
  const int G = gridDim.x, bid = blockIdx.x;
  const int ntl = bid < a.n_tiles ? (a.n_tiles - bid + G - 1) / G : 0;
  const int S = a.stages;
  if (S == 2 && !prologue_done && ntl > 0) {
    if (threadIdx.x == 0) issue_tile(a, sm, bid, issued % 2);
    ++issued;
  }
  for (int j = 0; j < ntl; ++j) {
    int s = consumed % S;
    unsigned parity = (unsigned)((consumed / S) & 1);
    if (S == 2) {
      if (j + 1 < ntl) {
        if (threadIdx.x == 0) issue_tile(a, sm, bid + (j + 1) * G, issued % 2);
        ++issued;
      }
    } else {
      if (threadIdx.x == 0) issue_tile(a, sm, bid + j * G, 0);
      ++issued;
    }
    if (!mbar_wait(&sm.mbar[s], parity, a.timeout_ns)) {
      atomicOr(a.err, 1);
      mbar_wait(&sm.mbar[s], parity, a.timeout_ns);  // let a late copy land before leaving
      return false;
    }
    tile_compute<T, MODE>(a, sm, s, pred);
    __syncthreads();
    ++consumed;
  }
  return true;
}

// The next walk's first tile can be issued before the block stages its vectors.
template <typename T>
__device__ bool issue_prologue(const PcgArgs<T>& a, PcgSmem<T>& sm, int& issued) {
  const int bid = blockIdx.x;
  if (a.stages == 2 && bid < a.n_tiles) {
    if (threadIdx.x == 0) issue_tile(a, sm, bid, issued % 2);
    ++issued;
    return true;
  }
  return false;
}

__device__ __forceinline__ double sum_dots(const double* region, int slot, int G, double* red) {
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) s += region[4 * g + slot];
  return block_sum(s, red);
}

template <typename T>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg(PcgArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PcgSmem<T> sm = carve<T>(smem_raw, a.n, a.C, a.stages);
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int n = a.n;
  const int f0 = (int)(((long long)a.Cf * bid) / G), f1 = (int)(((long long)a.Cf * (bid + 1)) / G);
  const int e0 = 9 * f0, e1 = 9 * f1, ne = e1 - e0;
  unsigned epoch = 0;
  int issued = 0, consumed = 0;
  double unused = 0.0;

  if (tid == 0) {
    mbar_init(&sm.mbar[0], 1);
    mbar_init(&sm.mbar[1], 1);
    fence_mbar_init();
  }
  for (int c = tid; c < a.C; c += blockDim.x) sm.crank[c] = a.crank[c];
  __syncthreads();

  // ---- r = b, x = 0, z = M^-1 r, p = z; dots r.z and b.b
  double loc_rz = 0.0, loc_bb = 0.0;
  for (int e = e0 + tid; e < e1; e += blockDim.x) {
    int f = e / 9, i = e - 9 * f;
    const T* Mi = a.Dinv + 81 * (size_t)f + 9 * i;
    T zz = T(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) zz += Mi[j] * a.b[9 * f + j];
    T bv = a.b[e];
    a.x[e] = T(0);
    a.r[e] = bv;
    a.z[e] = zz;
    a.p0[e] = zz;
    loc_rz += (double)bv * (double)zz;
    loc_bb += (double)bv * (double)bv;
  }
  // Dot products of consecutive phases alternate between two regions of G x 4
  // doubles: a region is rewritten only after every block passed the barrier
  // that follows its last read.
  int dph = 0;
  auto dregion = [&](int ph) { return a.dots + (size_t)(ph & 1) * 4 * G; };
  {
    double s0 = block_sum(loc_rz, sm.dred);
    double s1 = block_sum(loc_bb, sm.dred);
    if (tid == 0) {
      dregion(dph)[4 * bid + 0] = s0;
      dregion(dph)[4 * bid + 1] = s1;
    }
  }
  if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
  double rz = sum_dots(dregion(dph), 0, G, sm.dred);
  double bb = sum_dots(dregion(dph), 1, G, sm.dred);
  ++dph;
  double bnorm = sqrt(bb);
  int it = 0;
  double rr_last = bb;
  T* pcur = a.p0;
  T* pnext = a.p1;
  double beta = 0.0;
  bool first = true;
  while (bnorm > 0.0 && it < a.max_iters) {
    bool pro = issue_prologue(a, sm, issued);
    // ---- stage p (first: p = z; later: p = z + beta p_old) and clear the partial
    for (int e = tid; e < n; e += blockDim.x) {
      T pv = first ? pcur[e] : (T)((double)a.z[e] + beta * (double)pcur[e]);
      sm.xs[e] = pv;
      sm.ys[e] = T(0);
      if (!first && e >= e0 && e < e1) pnext[e] = pv;
    }
    if (!first) {
      T* tmp = pcur;
      pcur = pnext;
      pnext = tmp;
    }
    first = false;
    __syncthreads();
    if (!walk_tiles<T, 0>(a, sm, issued, consumed, pro, unused)) return;
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
        int e = e0 + base + tid;
        int f = e / 9, i = e - 9 * f;
        const T* ud = a.Ud + 45 * (size_t)f;
        T up = T(0);
#pragma unroll
        for (int j = 0; j < 9; ++j) up += ud[sym9(i, j)] * sm.xs[9 * f + j];
        T qv = up - tot;
        sm.ys[e] = qv;  // owned q kept in shared memory
        loc_pq += (double)sm.xs[e] * (double)qv;
      }
      __syncthreads();
    }
    {
      double s0 = block_sum(loc_pq, sm.dred);
      if (tid == 0) dregion(dph)[4 * bid + 2] = s0;
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double pq = sum_dots(dregion(dph), 2, G, sm.dred);
    ++dph;
    if (!(pq > 0.0) || !isfinite(pq)) {
      if (bid == 0 && tid == 0) atomicOr(a.err, 2);
      break;
    }
    double alpha = rz / pq;
    // ---- owners: x += alpha p, r -= alpha q, z = M^-1 r; r.r and r.z
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
      a.x[e] = (T)((double)a.x[e] + alpha * (double)sm.xs[e]);
      a.r[e] = (T)((double)a.r[e] - alpha * (double)sm.ys[e]);
    }
    __syncthreads();
    double loc_rr = 0.0, loc_rz2 = 0.0;
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
      int f = e / 9, i = e - 9 * f;
      const T* Mi = a.Dinv + 81 * (size_t)f + 9 * i;
      T zz = T(0);
#pragma unroll
      for (int j = 0; j < 9; ++j) zz += Mi[j] * a.r[9 * f + j];
      a.z[e] = zz;
      double rv = (double)a.r[e];
      loc_rr += rv * rv;
      loc_rz2 += rv * (double)zz;
    }
    {
      double s0 = block_sum(loc_rr, sm.dred);
      double s1 = block_sum(loc_rz2, sm.dred);
      if (tid == 0) {
        dregion(dph)[4 * bid + 0] = s0;
        dregion(dph)[4 * bid + 1] = s1;
      }
    }
    if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
    double rr = sum_dots(dregion(dph), 0, G, sm.dred);
    double rz2 = sum_dots(dregion(dph), 1, G, sm.dred);
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

  // ---- back-substitution with the final x: every block needs all of x
  if (!grid_barrier(a.bar, (++epoch) * G, a.err, a.timeout_ns)) return;
  bool pro = issue_prologue(a, sm, issued);
  for (int e = tid; e < n; e += blockDim.x) sm.xs[e] = a.x[e];
  __syncthreads();
  double pred = 0.0;
  if (!walk_tiles<T, 1>(a, sm, issued, consumed, pro, pred)) return;
  double ps = block_sum(pred, sm.dred);
  if (tid == 0) a.pred_parts[bid] = ps;
}

template <typename T>
const void* pcg_kernel_ptr() {
  return reinterpret_cast<const void*>(&k_pcg<T>);
}

template <typename T>
cudaError_t launch_pcg(const PcgArgs<T>& a, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {const_cast<PcgArgs<T>*>(&a)};
  return cudaLaunchCooperativeKernel(pcg_kernel_ptr<T>(), dim3(grid), dim3(kPcgThreads), args, smem, s);
}

int pcg_threads() { return kPcgThreads; }

void build_tile_meta(int n_obs, int n_pts, int n_runs, const int* cams, const int* poff,
                     const unsigned* runs, const uint8_t* cperm, unsigned char* out) {
  int* c = reinterpret_cast<int*>(out);
  for (int i = 0; i < pad4(n_obs); ++i) c[i] = i < n_obs ? cams[i] : 0;
  int* po = c + pad4(n_obs);
  for (int i = 0; i < pad4(n_pts + 1); ++i) po[i] = i <= n_pts ? poff[i] : 0;
  unsigned* r = reinterpret_cast<unsigned*>(po + pad4(n_pts + 1));
  for (int i = 0; i < pad4(n_runs); ++i) r[i] = i < n_runs ? runs[i] : 0u;
  uint8_t* cp = reinterpret_cast<uint8_t*>(r + pad4(n_runs));
  for (int i = 0; i < pad16(n_obs); ++i) cp[i] = i < n_obs ? cperm[i] : 0;
}

int meta_bytes_of(int n_obs, int n_pts, int n_runs) { return tile_meta_bytes(n_obs, n_pts, n_runs); }

template size_t pcg_smem_bytes<float>(int, int, int);
template size_t pcg_smem_bytes<double>(int, int, int);
template const void* pcg_kernel_ptr<float>();
template const void* pcg_kernel_ptr<double>();
template cudaError_t launch_pcg<float>(const PcgArgs<float>&, int, size_t, cudaStream_t);
template cudaError_t launch_pcg<double>(const PcgArgs<double>&, int, size_t, cudaStream_t);

}  // namespace bab
