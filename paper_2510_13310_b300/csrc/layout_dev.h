// layout_dev.h -- the observation layout of ba_create (see layout.h) built on
// the device.  Arrays land in device memory obtained through a caller-supplied
// allocator (so the problem owns and frees them); temporaries are stream-ordered.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "layout.h"

namespace bab {

using DevAlloc = std::function<void*(size_t)>;  // device bytes, or null on failure

struct DevLayout {
  int *po = nullptr, *co = nullptr;          // [N] input index in point / camera order
  int *co_po = nullptr;                      // [N] point-order position of each camera-order observation
  int *po_cam = nullptr, *po_pt = nullptr;   // [N] camera and point of each point-order observation
  int *pt_off = nullptr, *cam_off = nullptr;  // [P + 1], [C + 1]
  TileDesc* descs = nullptr;                 // [n_tiles]
  unsigned char* meta = nullptr;             // tile records (meta_bytes)
  int *chunk_obs = nullptr, *chunk_cam = nullptr, *cam_chunk = nullptr;
  int n_tiles = 0, g_rows = 0, n_chunks = 0;
  size_t meta_bytes = 0;
  uint64_t obs_hash = 0;
  std::vector<int> h_pt_off, h_cam_off;      // host copies of the offsets
};

struct DevCovis {
  int4* runs = nullptr;   // [n_runs] (camera i, camera j, first pair, pair count)
  int2* pairs = nullptr;  // [npairs]
  int n_runs = 0;
  size_t npairs = 0;
};

// d_*: device arrays.  Returns 0; 1 invalid input, 2 CUDA error, 3 out of memory
// (message in *err).  The same checks, messages and layout as build_obs_layout.
// vs (nullable): a second stream on which d_cams, d_pts and d_uv become ready
// (their finiteness is checked there, overlapping the index work on s).
int build_obs_layout_dev(int C, int P, int N, const double* d_cams, const double* d_pts, const double* d_uv,
                         const int32_t* d_oc, const int32_t* d_op, const DevAlloc& alloc, cudaStream_t s,
                         cudaStream_t vs, DevLayout* L, std::string* err);
// The same layout from the observation indices alone (index ranges, duplicate
// pairs and track lengths checked; no value arrays), for problems whose values
// are not BA cameras and pixels (global positioning).
int build_obs_layout_dev_indices(int C, int P, int N, const int32_t* d_oc, const int32_t* d_op,
                                 const DevAlloc& alloc, cudaStream_t s, DevLayout* L, std::string* err);
// Return the layout builders' cached scratch memory to the device.
void release_scratch_pools();
int build_covis_runs_dev(const DevLayout& L, int C, int N, const DevAlloc& alloc, cudaStream_t s, DevCovis* out,
                         std::string* err);

}  // namespace bab
