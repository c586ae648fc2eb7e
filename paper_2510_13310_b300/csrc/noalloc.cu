// noalloc.cu -- ba_eval_cost_noalloc: the FP64 robust cost of a state without any
// device allocation.
//
// Some callers cannot call cudaMalloc: host code running under a framework that
// owns all device memory and forbids raw allocations (its allocator must account
// for every byte, or the budget is fixed when the process starts, as in embedded
// and real-time pipelines), and latency-critical loops that must not take the
// implicit device-wide synchronisation an allocation can cause.  This entry point evaluates
// F = 1/2 sum rho(|r_k|^2) and the reprojection RMSE from caller-provided
// device arrays, using as scratch only a file-scope device array of fixed
// size that lives as long as the library is loaded.
#include <cstdio>
#include <mutex>

#include "../../include/ba_b300.h"
#include "internal.h"
#include "model.cuh"

namespace bab {

constexpr int kNaMaxCams = 4096;  // largest camera count this entry point accepts
constexpr int kNaBlocks = 1184;   // evaluation grid: 8 blocks per SM on 148 SMs
constexpr int kNaThreads = 256;

// Scratch: kNaMaxCams working camera records (rotation matrix, t, f, k1, k2,
// 16 doubles each) followed by kNaBlocks partial sums (4 doubles each);
// 4096 * 128 B + 1184 * 32 B = 550,400 B on every device that loads the library.
// Host code must not use this name as an address: it is looked up per device
// with cudaGetSymbolAddress below.
static __device__ __align__(256) double g_na_scratch[kNaMaxCams * kCamStride + kNaBlocks * 4];

namespace {

std::mutex g_na_mutex;
double* g_na_ptr[64] = {};  // device address of g_na_scratch, per device ordinal

__global__ void k_na_prep_cams(const double* __restrict__ cams, int C, int model, double* __restrict__ rec) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double r[kCamStride];
  cam_record(cams + 9 * (size_t)c, model, r);
  for (int i = 0; i < kCamStride; ++i) rec[kCamStride * (size_t)c + i] = r[i];
}

// Input-order variant of the FP64 evaluation: every block writes its own partial
// (cost, |r_uv|^2, count), so no scratch entry needs clearing between calls.
// Observations with an index out of range are skipped.
__global__ void k_na_eval(int C, int P, int N, const double* __restrict__ rec,
                          const double* __restrict__ pts, const int32_t* __restrict__ obs_cam,
                          const int32_t* __restrict__ obs_pt, const double* __restrict__ obs_uv,
                          const double* __restrict__ depth, const uint8_t* __restrict__ mask,
                          ModelParams mp, double* __restrict__ partials) {
  __shared__ double red[32];
  double acc_cost = 0.0, acc_e2 = 0.0, acc_n = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
    if (mask && !mask[k]) continue;
    int c = obs_cam[k], p = obs_pt[k];
    if (c < 0 || c >= C || p < 0 || p >= P) continue;
    double d = depth[k];
    bool prior = d > 0.0 && isfinite(d);
    double tau = prior ? 1.0 / d : 0.0;
    double sw = prior ? mp.sw_valid : mp.sw_invalid;
    const double* X = pts + 3 * (size_t)p;
    Eval64 e = eval_obs64(rec + kCamStride * (size_t)c, X[0], X[1], X[2], obs_uv[2 * (size_t)k],
                          obs_uv[2 * (size_t)k + 1], tau, sw, mp.cx, mp.cy);
    double e2 = e.r0 * e.r0 + e.r1 * e.r1;
    acc_cost += huber_loss(e2 + e.r2 * e.r2, mp.huber);
    acc_e2 += e2;
    acc_n += 1.0;
  }
  double s0 = block_sum(acc_cost, red);
  double s1 = block_sum(acc_e2, red);
  double s2 = block_sum(acc_n, red);
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x] = s0;
    partials[4 * blockIdx.x + 1] = s1;
    partials[4 * blockIdx.x + 2] = s2;
  }
}

__global__ void k_na_reduce(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += partials[4 * i];
    b += partials[4 * i + 1];
    c += partials[4 * i + 2];
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  c = block_sum(c, red);
  if (threadIdx.x == 0) {
    out[0] = 0.5 * a;
    out[1] = c > 0.0 ? sqrt(b / c) : 0.0;
    out[2] = c;
  }
}

void fail_msg(const char* fmt, const char* arg) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, arg);
  set_last_error_message(buf);
}

// True when the pointer can be read by kernels on the current device: device or
// managed memory of this device, or page-locked host memory mapped into it whose
// device alias is the pointer itself (unified addressing); the kernels are given
// the pointer as passed, so a host pointer with a different device alias is refused.
bool device_accessible(const void* p, int dev) {
  if (!p) return true;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == dev;
  if (at.type == cudaMemoryTypeManaged) return true;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer == p;
  return false;
}

// Device address of the scratch array on the current device, looked up once per
// device and kept for the life of the process (the first call on a device must
// not happen during stream capture; a device reset in between is not supported).
ba_status scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    fail_msg("ba_eval_cost_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
    return BA_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      fail_msg("ba_eval_cost_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return BA_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return BA_OK;
}

}  // namespace
}  // namespace bab

extern "C" ba_status ba_eval_cost_noalloc(const ba_options* opts, void* stream, int64_t n_cams,
                                          const double* cams, int64_t n_pts, const double* pts,
                                          int64_t n_obs, const int32_t* obs_cam,
                                          const int32_t* obs_pt, const double* obs_uv,
                                          const double* depth, const uint8_t* obs_mask,
                                          double* out) {
  using namespace bab;
  if (!opts || !out || n_cams < 0 || n_pts < 0 || n_obs < 0 || n_obs >= (1LL << 31) ||
      n_pts >= (1LL << 31) || (n_cams && !cams) || (n_pts && !pts) ||
      (n_obs && (!obs_cam || !obs_pt || !obs_uv || !depth))) {
    fail_msg("ba_eval_cost_noalloc: %s", "invalid argument (null pointer or size out of range)");
    return BA_ERR_INVALID_ARG;
  }
  if (n_cams > kNaMaxCams) {
    char buf[160];
    snprintf(buf, sizeof buf, "%lld cameras exceed the fixed scratch limit of %d cameras",
             (long long)n_cams, kNaMaxCams);
    fail_msg("ba_eval_cost_noalloc: %s", buf);
    return BA_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  ba_status st = scratch_for_current_device(&scratch);
  if (st != BA_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  const void* ptrs[] = {cams, pts, obs_cam, obs_pt, obs_uv, depth, obs_mask, out};
  for (const void* p : ptrs)
    if (!device_accessible(p, dev)) {
      fail_msg("ba_eval_cost_noalloc: %s", "every array must be device memory of the current device "
                                             "or mapped page-locked host memory");
      return BA_ERR_INVALID_ARG;
    }
  double* rec = scratch;
  double* partials = scratch + kNaMaxCams * kCamStride;
  ModelParams mp{};
  mp.cx = opts->cx;
  mp.cy = opts->cy;
  mp.huber = opts->huber_delta;
  mp.sw_valid = sqrt(opts->depth_weight);
  mp.sw_invalid = sqrt(opts->invalid_depth_weight);
  cudaStream_t s = (cudaStream_t)stream;
  int C = (int)n_cams, P = (int)n_pts, N = (int)n_obs;
  if (C > 0) k_na_prep_cams<<<(C + 127) / 128, 128, 0, s>>>(cams, C, opts->camera_model == 1 ? 1 : 0, rec);
  int grid = (N + kNaThreads - 1) / kNaThreads;
  grid = grid < 1 ? 1 : (grid > kNaBlocks ? kNaBlocks : grid);
  k_na_eval<<<grid, kNaThreads, 0, s>>>(C, P, N, rec, pts, obs_cam, obs_pt, obs_uv, depth, obs_mask,
                                        mp, partials);
  k_na_reduce<<<1, kNaThreads, 0, s>>>(partials, grid, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fail_msg("ba_eval_cost_noalloc: launch failed: %s", cudaGetErrorString(e));
    return BA_ERR_CUDA;
  }
  return BA_OK;
}
