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

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace bab
