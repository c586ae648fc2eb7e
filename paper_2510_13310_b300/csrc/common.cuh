// common.cuh -- shared device helpers of the B300 bundle-adjustment library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bab {

constexpr int kTileObs = 256;      // max observations per point-order tile (and per point)
constexpr int kChunkObs = 1024;    // max observations per camera-order chunk
constexpr int kCamStride = 16;     // working camera record: R(9) t(3) f k1 k2 pad
constexpr int kWStride = 28;       // W row: 9x3 block padded to 28 entries (16-byte rows)
constexpr int kBlock = 256;

// Packed upper triangle of a symmetric 9x9 block, row-major over i <= j.
__host__ __device__ constexpr int sym9(int i, int j) {
  return i <= j ? i * 9 - (i * (i - 1)) / 2 + (j - i) : j * 9 - (j * (j - 1)) / 2 + (i - j);
}
// Packed symmetric 3x3: 00 01 02 11 12 22.
__host__ __device__ constexpr int sym3(int i, int j) {
  return i <= j ? i * 3 - (i * (i - 1)) / 2 + (j - i) : j * 3 - (j * (j - 1)) / 2 + (i - j);
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };

// Per-iteration scalars shared between kernels and read back by the host.
struct Scalars {
  double cost[2];        // F over the active set for state slot 0 / 1
  double rmse_sum[2];    // sum |r_uv|^2 over the active set
  double n_act[2];       // active observations counted by the evaluation
  double pred;           // predicted decrease
  double pcg_rel_res;
  double pcg_bnorm;
  int pcg_iters;
  int pcg_error;         // 1: barrier timeout, 2: breakdown (non-positive curvature)
  int changed;           // extraction: something changed in this peel round
  int mask_changed;      // extraction: the final obs mask differs from the previous one
  int n_obs_act;
  int n_cam_free;
  int n_pt_act;
  int n_cam_act;
  int valid_flips;       // evaluation: some validity bit differs from the reference slot's
  unsigned done_eval;    // blocks of the evaluation kernel that have written their partials
  unsigned done_pred;    // blocks of the back-substitution kernel likewise
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one value (all threads get the result).  blockDim multiple of 32.
template <typename T>
__device__ T block_sum(T v, T* red /* >= 32 entries */) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = T(0);
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Last-block-done: every block has written its partials (the writers fence, then
// one atomic increment per block); returns true in the block that arrived last,
// to which all partials are visible (read them with __ldcg).  That block resets
// the counter for the next launch.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// FP64 is scarce on B300 (a small fraction of the FP32 rate), so FP64 sums run
// in one warp only.  warp0_sum2: sum of per-thread values a, b held by threads
// [0, count) (others ignored); every thread gets both results.
// buf: >= 2 * count doubles of shared scratch; out: 2 doubles of shared scratch.
__device__ __forceinline__ void warp0_sum2(double a, double b, int count, double* buf, double* out,
                                           double& ra, double& rb) {
  if ((int)threadIdx.x < count) {
    buf[threadIdx.x] = a;
    buf[count + threadIdx.x] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) {
      sa += buf[i];
      sb += buf[count + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (threadIdx.x == 0) {
      out[0] = sa;
      out[1] = sb;
    }
  }
  __syncthreads();
  ra = out[0];
  rb = out[1];
}

// Sum of slots s0, s1 of the G per-block records (4 doubles each), by warp 0,
// broadcast to the block.  Fixed order: every block gets identical results.
__device__ __forceinline__ void warp0_sum_slots(const double* region, int G, int s0, int s1,
                                                double* out, double& r0, double& r1) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    for (int g = threadIdx.x; g < G; g += 32) {
      a += region[4 * g + s0];
      b += region[4 * g + s1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      out[0] = a;
      out[1] = b;
    }
  }
  __syncthreads();
  r0 = out[0];
  r1 = out[1];
  __syncthreads();
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Index checks of the BA_DEBUG_BOUNDS build, at the gathers that use an index
// loaded from the observation layout or the co-visibility runs.  bidx(i, n, site)
// returns i when 0 <= i < n; otherwise it records the first failure of this
// translation unit as ((site + 1) << 32) | (uint32) i and returns 0, so the access
// stays in bounds and the kernel's control flow (its barriers) is unchanged.
// Release builds compile the checks away.  BA_BOUNDS_QUERY(fn) defines the host
// function reading (and optionally clearing) this translation unit's record.
#ifdef BA_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_fault;
__device__ __forceinline__ int bidx(long long i, long long n, int site) {
  if (i < 0 || i >= n) {
    atomicCAS(&g_bounds_fault, 0ull, ((unsigned long long)(site + 1) << 32) | (unsigned)(i & 0xffffffffLL));
    return 0;
  }
  return (int)i;
}
#define BA_BOUNDS_QUERY(fn)                                                       \
  unsigned long long fn(bool reset) {                                             \
    unsigned long long v = 0;                                                     \
    if (cudaMemcpyFromSymbol(&v, g_bounds_fault, sizeof v) != cudaSuccess) return ~0ull; \
    if (reset) {                                                                  \
      const unsigned long long z = 0;                                             \
      if (cudaMemcpyToSymbol(g_bounds_fault, &z, sizeof z) != cudaSuccess) return ~0ull; \
    }                                                                             \
    return v;                                                                     \
  }
#else
__device__ __forceinline__ int bidx(long long i, long long, int) { return (int)i; }
#define BA_BOUNDS_QUERY(fn) \
  unsigned long long fn(bool) { return 0; }
#endif

}  // namespace bab
