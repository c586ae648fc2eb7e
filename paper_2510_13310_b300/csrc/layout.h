// layout.h -- host-side construction of the observation layout that ba_create
// builds once: input validation, the point-order and camera-order permutations,
// point tiles with their metadata records, camera chunks, and the co-visibility
// runs of the explicit reduced camera system.
//
// The work runs on a persistent pool of host threads.  Every parallel loop
// writes outputs fixed by its indices alone (no atomics on data, no
// order-dependent accumulation), so the layout depends neither on the number of
// threads nor on their timing.
#pragma once
#include <cuda_runtime.h>  // int2, int4
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "internal.h"

namespace bab {

// Large host buffer, 2 MB aligned and advised for transparent huge pages (one
// first-touch fault per 2 MB instead of per 4 KB); not zero-initialised.
template <typename T>
class HostBuf {
 public:
  HostBuf() = default;
  explicit HostBuf(size_t n) { resize(n); }
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  HostBuf(HostBuf&& o) noexcept : p_(o.p_), n_(o.n_) { o.p_ = nullptr, o.n_ = 0; }
  HostBuf& operator=(HostBuf&& o) noexcept {
    if (this != &o) {
      release();
      p_ = o.p_, n_ = o.n_;
      o.p_ = nullptr, o.n_ = 0;
    }
    return *this;
  }
  ~HostBuf() { release(); }
  void resize(size_t n);  // discards the contents
  T* data() { return p_; }
  const T* data() const { return p_; }
  size_t size() const { return n_; }
  T& operator[](size_t i) { return p_[i]; }
  const T& operator[](size_t i) const { return p_[i]; }

 private:
  void release();
  T* p_ = nullptr;
  size_t n_ = 0;
};

// threads used by the parallel loops: the hardware threads, at most 32, or
// BA_HOST_THREADS when set
int host_threads();
// f(t) for t = 0 .. n-1 on the pool (the calling thread takes part)
void run_pieces(int n, const std::function<void(int)>& f);

// f(t, begin, end) over contiguous pieces [n t / nt, n (t+1) / nt) of [0, n),
// at least `grain` indices per piece
template <class F>
void parallel_for(int64_t n, int64_t grain, F&& f) {
  if (n <= 0) return;
  const int64_t g = grain > 0 ? grain : 1;
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / g));
  run_pieces(nt, [&](int t) { f(t, n * t / nt, n * (t + 1) / nt); });
}

// observation layout (all indices 32-bit; N < 2^31)
struct ObsLayout {
  HostBuf<int> po;                  // [N] input index of each point-order observation
  HostBuf<int> co;                  // [N] input index of each camera-order observation
  HostBuf<int> po_cam, po_pt;       // [N] camera and point of each point-order observation
  HostBuf<int> co_po;               // [N] point-order position of each camera-order observation
  std::vector<int> pt_off, cam_off;  // [P + 1], [C + 1]
  std::vector<int> wr_pt, tile_wr;   // warp ranges (first point of each) and tiles (first range)
  std::vector<TileDesc> descs;       // [n_tiles]
  HostBuf<unsigned char> meta;       // tile metadata records
  std::vector<int> chunk_obs, chunk_cam, cam_chunk;  // camera chunks
  int n_tiles = 0, g_rows = 0;
  uint64_t obs_hash = 0;             // digest of (C, P, observation structure)
};

// Validates the inputs (finite values, index ranges, no duplicate (camera,
// point), at most kTileObs observations per point) and builds the layout.
// Returns 0, or 1 with a message in *err.
// wide_keys: sort with gathered keys even when (point, camera) fits a 32-bit
// packed key (the path taken for more than 2^32 point-camera combinations).
int build_obs_layout(int C, int P, int N, const double* cams, const double* pts, const double* uv,
                     const int32_t* oc, const int32_t* op, ObsLayout* L, std::string* err,
                     bool wide_keys = false);

// Warp ranges and tiles over the points (pt_off: [P + 1] observation offsets);
// descriptors without their camera runs and metadata offsets.
void group_tiles(const int* pt_off, int P, std::vector<int>* wr_pt, std::vector<int>* tile_wr,
                 std::vector<TileDesc>* descs, int* g_rows);

// co-visibility runs: every pair of observations of one point in cameras i < j,
// grouped by (i, j), ascending in point within a run
struct CovisRuns {
  std::vector<int4> runs;  // (camera i, camera j, first pair, pair count)
  HostBuf<int2> pairs;     // (k in i, k2 in j), point-order indices
  size_t npairs = 0;
};
// Returns 0, or 1 with a message in *err (more than 2^31 - 1 pairs).
int build_covis_runs(const ObsLayout& L, int C, int N, CovisRuns* out, std::string* err);

}  // namespace bab
