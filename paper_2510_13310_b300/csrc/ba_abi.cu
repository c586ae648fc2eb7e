// ba_abi.cu -- host side of the C ABI: problem set-up, the LM loop and inspection calls.
//
// The host only orders kernels on the problem's stream, reads back a handful
// of scalars per iteration and keeps the scalar LM bookkeeping (damping and
// the accept decision of Sec. 3.3).  Every array operation of steps (a)-(e)
// runs in the kernels of kernels.cu.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ba_b300.h"
#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "layout.h"
#include "layout_dev.h"

using namespace bab;

namespace {

thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

#define CU(expr)                                                                     \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) {                                                         \
      cudaGetLastError(); /* reported here: not left for the caller's next check */  \
      set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA;             \
    }                                                                                \
  } while (0)

#define ST(expr)                      \
  do {                                \
    ba_status _s = (expr);            \
    if (_s != BA_OK) return _s;       \
  } while (0)

}  // namespace

void bab::set_last_error_message(const char* msg) { g_last_error = msg; }

struct ba_problem {
  ba_options opt{};
  std::vector<int32_t> fixed_list;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  int C = 0, P = 0, N = 0;
  bool fp64 = false;
  Layout L{};
  ModelParams mp{};
  std::vector<void*> allocs;
  int64_t launches = 0;

  // layout arrays (device)
  int *po_cam = nullptr, *po_pt = nullptr, *po_orig = nullptr, *pt_off = nullptr;
  double *po_uv64 = nullptr, *po_tau64 = nullptr;
  float4* po_uvdf = nullptr;  // double-float copies for the FP32 problems' evaluation
  F2* po_taudf = nullptr;
  F2* camdf[2] = {nullptr, nullptr};      // per state slot; current when df_current[slot]
  float4* ptdf[2] = {nullptr, nullptr};
  bool df_current[2] = {false, false};    // written by the candidate kernels with the slot
  void *po_uvw = nullptr, *po_tauw = nullptr, *co_uvw = nullptr, *co_tauw = nullptr;
  int *co_pt = nullptr, *co_po = nullptr, *po_wrow = nullptr;
  int *chunk_obs = nullptr, *chunk_cam = nullptr, *cam_chunk = nullptr;
  TileDesc* descs = nullptr;
  unsigned char* meta = nullptr;
  int w_rows = 0;
  uint8_t* cam_fixed = nullptr;
  int n_tiles = 0, n_chunks = 0;

  // state, two slots (current / candidate)
  double* cams64[2] = {nullptr, nullptr};
  double* pts64[2] = {nullptr, nullptr};
  double* camw64[2] = {nullptr, nullptr};
  // adjoint refinement (FP32 problems, allocated by the first ba_backward): the
  // right-hand side, mu, per-observation rho' J mu, (H mu)_p and camera-chunk partials
  bool reuse_system = false;  // the next explicit solve reuses the formed S^ / dense factor
  double *adj_ac = nullptr, *adj_ap = nullptr, *adj_muc = nullptr, *adj_mup = nullptr, *adj_u = nullptr,
         *adj_hp = nullptr, *adj_part = nullptr;
  void* camw[2] = {nullptr, nullptr};
  void* ptsw[2] = {nullptr, nullptr};
  uint8_t* bits[2] = {nullptr, nullptr};
  int cur = 0;

  // extraction
  uint8_t *alive = nullptr, *valid = nullptr, *obs_act = nullptr, *obs_act_co = nullptr;
  uint8_t *cam_act = nullptr, *pt_act = nullptr, *cam_flags = nullptr;
  int *cam_cnt = nullptr, *crank = nullptr, *cam_map = nullptr, *pt_rank = nullptr, *pt_map = nullptr;
  int *rank_tmp = nullptr, *counts = nullptr;
  int n_rank_tmp = 0;

  // normal equations and solver
  void *W = nullptr, *wsgn = nullptr, *V = nullptr, *gp = nullptr, *Vinv = nullptr, *z0 = nullptr;
  void *Ug = nullptr, *Sg = nullptr, *cam_part = nullptr, *Ud = nullptr, *Dinv = nullptr;
  void *bvec = nullptr, *dampc = nullptr, *x = nullptr, *z = nullptr;
  void *partials = nullptr, *dp = nullptr;
  double *dots = nullptr, *pred_parts = nullptr, *eval_parts = nullptr;
  unsigned* bar = nullptr;
  int* err = nullptr;
  Scalars* sc = nullptr;
  Scalars* h_sc = nullptr;  // pinned
  int pcg_grid = 0, eval_grid = 0, pcg_stages = 2, pcg_own_max = 1;
  int recompute = 0, cam_in_smem = 0, max_tiles_per_block = 1, g_rows = 0;
  // explicit reduced camera system
  bool explicit_S = false;
  bool dense = false;            // explicit S factored on the tensor cores (FP32)
  bool sparse = false;           // explicit S stored as 9x9 blocks of co-visible pairs (block-sparse)
  int* brp = nullptr;            // block rows by camera: [C + 1] offsets into bent
  int2* bent = nullptr;          // (column camera, block slot), ascending column within a row
  void* Bs = nullptr;            // blocks [2 n_runs + C][kBlkStride]: run r at 2r (and 2r+1 transposed), diagonals last
  DenseResult dense_last;
  DenseWork dw;
  unsigned dense_epoch = 0;
  float* dense_b = nullptr;      // [2][n]: scaled right-hand side, scaled solution
  void *Shat = nullptr, *Dblk = nullptr;
  void* Yhat = nullptr;         // [N + 1][kWStride] D^-1 W M per damping value (explicit system)
  void* bs_wx = nullptr;        // [N][3] W_k^T dc of the back-substitution (explicit system)
  int4* covis_runs = nullptr;   // (camera i, camera j, first pair, count), i < j
  int2* covis_pairs = nullptr;  // point-order observations (k in i, k2 in j) of shared points; FP32
                                // explicit systems: camera-order (owner's row, other's row), see CamForm
  CamForm cform;                // FP32 explicit systems: the camera-owned formation (n_blocks > 0)
  float* orec = nullptr;        // FP32 warp-per-run formation: observation records [N][16]
  float* prec = nullptr;        //   point records [P][8] (V*^-1)
  int* pair_pt = nullptr;       //   and the point of every co-visible pair
  int n_covis_runs = 0;
  bool form_lanes = false;      // one lane per co-visibility run (many short runs)
  double* dscale = nullptr;
  int spcg_grid = 0, spcg_rows_in_smem = 0, spcg_vecs_in_smem = 0, bs_grid = 1;
  void* spcg_scratch = nullptr;   // per-block PCG vectors when they do not fit in shared memory
  void* spcg_M = nullptr;         // the preconditioner blocks, one copy for all blocks (with spcg_scratch)
  size_t spcg_scratch_stride = 0;
  size_t spcg_smem = 0;
  unsigned long long* spcg_words = nullptr;  // exchange words of the explicit PCG
  unsigned spcg_tag = 1;                     // next launch's first iteration tag
  size_t pcg_smem = 0;

  // LM bookkeeping
  int iter = 0;
  double lambda = 1e-4, nu = 2.0;
  uint64_t obs_hash = 0;        // FNV-1a of the input index arrays (checkpoint identity)
  bool extracted = false, state_changed = true, linearized = false;
  // the state changed by an accepted step whose validity bits equal those of the
  // state the active set was extracted from: the extraction would not change it
  bool same_validity = false, flips_known = false;
  bool bits_valid[2] = {false, false};
  bool cost_valid[2] = {false, false};
  int n_cam_free = 0, n_pt_act = 0, n_obs_act = 0, n_cam_act = 0;
  bool solved = false;

  cudaEvent_t ev[8] = {};
  cudaEvent_t evk[2] = {};  // around the PCG kernel launch of the latest solve
  bool evk_valid = false;
  cudaEvent_t evf[2] = {};
  // high-priority side stream for work that overlaps the main stream: the camera
  // side of the linearisation (k_cam_accum<0>, k_cam_reduce) next to k_pt_lin,
  // and for the explicit system the Schur-diagonal chain (k_cam_accum<1>,
  // k_cam_reduce, k_schur_diag) next to the formation of S^; `join` marks the
  // chain's end, waited on before anything that reads its outputs
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool join_pending = false;
  // LM step: the camera candidate (FP64 rotation updates, latency-bound) runs on
  // the side stream as soon as dc is known, alongside the point back-substitution
  bool cand_early_ok = false;   // set by the LM step around its solve
  bool cand_cams_done = false;  // launched early for this step; `cand_join` marks its end
  cudaEvent_t cand_fork = nullptr, cand_join = nullptr;  // around the co-visibility product kernel of the latest formation
  bool evf_valid = false;
  // step (c): the first pass of an extraction (begin, one peel round, the
  // finalisation, the scalars back to the host) is a fixed sequence of ~20
  // operations per (drop, state slot); it is captured once into a CUDA graph on
  // `cap` and replayed on `stream` (the same kernels in the same order: the same
  // bits, without a launch gap between them)
  cudaStream_t cap = nullptr;
  cudaGraphExec_t ext_graph[2][2] = {};
  long long ext_graph_launches[2][2] = {};
  bool ext_graph_off = false;  // capture failed once: launch the operations one by one
};

namespace {

// Device memory cache of the process: ba_destroy returns a problem's buffers
// here instead of to the driver, and ba_create takes buffers of the same
// (rounded) size back, so a process that creates problems repeatedly (serving,
// batches of scenes) maps no new device memory after the first.  Keyed by
// (device, size); ba_release_cache() frees everything.  BA_NO_ALLOC_CACHE=1
// disables it.
struct AllocCache {
  std::mutex mu;
  std::multimap<std::pair<int, size_t>, void*> free_blocks;
  std::map<void*, std::pair<int, size_t>> sizes;  // every block handed out, with its key
};
AllocCache& alloc_cache() {
  static AllocCache* c = new AllocCache();  // never destroyed: safe at process exit
  return *c;
}
bool alloc_cache_on() {
  static const bool on = [] {
    const char* v = std::getenv("BA_NO_ALLOC_CACHE");
    return !(v && v[0] && v[0] != '0');
  }();
  return on;
}
size_t cache_round(size_t bytes) { return (std::max<size_t>(bytes, 16) + 511) / 512 * 512; }

// device memory for the current device: from the cache when a block of the
// rounded size is free, else cudaMalloc
cudaError_t cached_malloc(void** q, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t rb = cache_round(bytes);
  if (alloc_cache_on()) {
    AllocCache& c = alloc_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.free_blocks.find({dev, rb});
    if (it != c.free_blocks.end()) {
      *q = it->second;
      c.free_blocks.erase(it);
      return cudaSuccess;
    }
  }
  e = cudaMalloc(q, rb);
  if (e == cudaSuccess && alloc_cache_on()) {
    AllocCache& c = alloc_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.sizes[*q] = {dev, rb};
  }
  return e;
}
// back to the cache (the caller has synchronised every stream that used it)
void cached_free(void* q) {
  if (!q) return;
  if (alloc_cache_on()) {
    AllocCache& c = alloc_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.sizes.find(q);
    if (it != c.sizes.end()) {
      c.free_blocks.insert({it->second, q});
      return;
    }
  }
  cudaFree(q);
}

template <typename X>
ba_status dalloc(ba_problem* pb, X** p, size_t count) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(sizeof(X) * count, 16);
  cudaError_t e = cached_malloc(&q, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return BA_ERR_OOM;
  }
  pb->allocs.push_back(q);
  *p = reinterpret_cast<X*>(q);
  return BA_OK;
}

ba_status dalloc_bytes(ba_problem* pb, void** p, size_t bytes) {
  char* q = nullptr;
  ST(dalloc(pb, &q, bytes));
  *p = q;
  return BA_OK;
}

size_t rsz(const ba_problem* pb) { return pb->fp64 ? sizeof(double) : sizeof(float); }

// Stable counting sort of idx by key (keys in [0, nkeys)).
// device-resident (device or managed) memory; anything else is read on the host
bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// RAII device scratch of ba_create (freed once the device is idle)
struct DevScratch {
  void* p = nullptr;
  ~DevScratch() {
    if (p) {
      cudaDeviceSynchronize();
      cached_free(p);
    }
  }
};


bool finite_opts(const ba_options* o) {
  return std::isfinite(o->cx) && std::isfinite(o->cy) && std::isfinite(o->huber_delta) &&
         std::isfinite(o->depth_weight) && o->depth_weight >= 0 &&
         std::isfinite(o->invalid_depth_weight) && o->invalid_depth_weight >= 0 &&
         std::isfinite(o->min_depth) && std::isfinite(o->lambda0) && o->lambda0 > 0 &&
         std::isfinite(o->pcg_rel_tol) && o->pcg_rel_tol > 0 && o->pcg_max_iters > 0 &&
         o->img_w > 0 && o->img_h > 0 && o->min_cam_obs >= 0 && o->min_pt_obs >= 0 &&
         o->extract_every >= 0 && (o->precision == BA_FP64 || o->precision == BA_FP32) &&
         (o->extract_mode == BA_EXTRACT_DYNAMIC || o->extract_mode == BA_EXTRACT_ONCE) &&
         (o->camera_model == BA_CAMERA_RADIAL || o->camera_model == BA_CAMERA_CENTRE);
}

ba_status sync(ba_problem* pb) {
  CU(cudaStreamSynchronize(pb->stream));
  return BA_OK;
}

#define LAUNCH(n, expr)      \
  do {                       \
    pb->launches += (n);     \
    CU(expr);                \
  } while (0)

// ---------------------------------------------------------------------------
// evaluation and extraction
// ---------------------------------------------------------------------------

// Evaluation pass over a state slot (FP64, or double-float for FP32 problems): validity bits (if bits != null) and the cost over
// the current active set (if with_cost) into sc->cost[slot].  ref_slot >= 0:
// compare the validity bits with that slot's (sc->valid_flips, cleared here).
ba_status eval_state(ba_problem* pb, int slot, bool want_bits, bool with_cost, int ref_slot = -1) {
  const bool cmp = want_bits && ref_slot >= 0 && ref_slot != slot && pb->bits_valid[ref_slot];
  if (cmp) CU(cudaMemsetAsync(&pb->sc->valid_flips, 0, sizeof(int), pb->stream));
  if (pb->fp64)
    LAUNCH(1, launch_eval64(pb->L, pb->mp, pb->camw64[slot], pb->pts64[slot],
                            with_cost ? pb->obs_act : nullptr, want_bits ? pb->bits[slot] : nullptr,
                            cmp ? pb->bits[ref_slot] : nullptr, cmp ? &pb->sc->valid_flips : nullptr,
                            with_cost ? pb->eval_parts : nullptr, pb->sc, slot, pb->eval_grid, pb->stream));
  else
    LAUNCH(pb->df_current[slot] ? 1 : 2,
           launch_eval_df(pb->L, pb->mp, pb->camw64[slot], pb->pts64[slot], pb->camdf[slot], pb->ptdf[slot],
                          !pb->df_current[slot],
                             with_cost ? pb->obs_act : nullptr, want_bits ? pb->bits[slot] : nullptr,
                             cmp ? pb->bits[ref_slot] : nullptr, cmp ? &pb->sc->valid_flips : nullptr,
                             with_cost ? pb->eval_parts : nullptr, pb->sc, slot, pb->eval_grid, pb->stream));
  pb->flips_known = cmp;
  if (!pb->fp64) pb->df_current[slot] = true;
  if (want_bits) pb->bits_valid[slot] = true;
  if (with_cost) pb->cost_valid[slot] = true;
  return BA_OK;
}

ba_status run_extraction(ba_problem* pb, bool drop, int* rounds_out) {
  ba_problem* p = pb;
  int slot = p->cur;
  if (!p->bits_valid[slot]) ST(eval_state(p, slot, true, false));
  int rounds = 0;
  const int max_rounds = p->C + p->P + 2;
  // One peel round, then the finalisation launched speculatively: a single
  // readback covers the common case where the first round changes nothing.
  // If it did change something, peel to the fixed point and finalise again.
  auto peel_round = [&]() -> ba_status {
    ++rounds;
    CU(cudaMemsetAsync(&p->sc->changed, 0, sizeof(int), p->stream));
    LAUNCH(1, launch_peel_points(p->L, p->valid, p->cam_act, p->pt_act, p->cam_cnt, p->opt.min_pt_obs,
                                 p->sc, p->stream));
    LAUNCH(1, launch_peel_cams(p->L, p->cam_act, p->cam_cnt, p->opt.min_cam_obs, p->sc, p->stream));
    return BA_OK;
  };
  auto finalize_enqueue = [&]() -> ba_status {
    CU(cudaMemsetAsync(&p->sc->mask_changed, 0, sizeof(int), p->stream));
    CU(cudaMemsetAsync(&p->sc->n_obs_act, 0, sizeof(int), p->stream));
    CU(cudaMemsetAsync(&p->sc->n_cam_act, 0, sizeof(int), p->stream));
    LAUNCH(2, launch_finalize_obs(p->L, p->valid, p->cam_act, p->pt_act, p->obs_act, p->obs_act_co,
                                  p->sc, p->stream));
    LAUNCH(1, launch_cam_flags(p->L, p->cam_act, p->cam_flags, p->sc, p->stream));
    LAUNCH(3, launch_rank(p->cam_flags, p->C, p->crank, p->cam_map, &p->sc->n_cam_free, p->rank_tmp,
                          p->n_rank_tmp, p->stream));
    LAUNCH(3, launch_rank(p->pt_act, p->P, p->pt_rank, p->pt_map, &p->sc->n_pt_act, p->rank_tmp,
                          p->n_rank_tmp, p->stream));
    CU(cudaMemcpyAsync(p->h_sc, p->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, p->stream));
    return BA_OK;
  };
  auto finalize = [&]() -> ba_status {
    ST(finalize_enqueue());
    return sync(p);
  };
  // the first pass: begin, one peel round, the finalisation launched speculatively
  auto first_pass = [&]() -> ba_status {
    LAUNCH(1, launch_extract_begin(p->L, p->alive, p->bits[slot], p->valid, drop ? 1 : 0, p->stream));
    LAUNCH(1, launch_fill_u8(p->cam_act, 1, p->C, p->stream));
    LAUNCH(1, launch_fill_u8(p->pt_act, 1, p->P, p->stream));
    CU(cudaMemsetAsync(p->cam_cnt, 0, sizeof(int) * std::max(1, p->C), p->stream));
    ST(peel_round());
    return finalize_enqueue();
  };
  cudaGraphExec_t& ge = p->ext_graph[drop ? 1 : 0][slot];
  if (!ge && !p->ext_graph_off) {
    // capture the first pass once (thread-local capture: other threads' CUDA calls
    // are unaffected); on any failure the operations are launched one by one
    if (!p->cap) CU(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    cudaStream_t main_stream = p->stream;
    const long long l0 = p->launches;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      p->stream = p->cap;
      const ba_status st = first_pass();
      p->stream = main_stream;
      ok = cudaStreamEndCapture(p->cap, &graph) == cudaSuccess && st == BA_OK && graph;
    }
    if (ok) ok = cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    p->ext_graph_launches[drop ? 1 : 0][slot] = p->launches - l0;
    p->launches = l0;
    if (!ok) {
      ge = nullptr;
      p->ext_graph_off = true;
      (void)cudaGetLastError();  // the capture's error is not the caller's
    }
  }
  if (ge) {
    p->launches += p->ext_graph_launches[drop ? 1 : 0][slot];
    rounds = 1;
    CU(cudaGraphLaunch(ge, p->stream));
    ST(sync(p));
  } else {
    ST(first_pass());
    ST(sync(p));
  }
  if (p->h_sc->changed) {
    // the speculative pass already compared against the previous masks: keep
    // its outcome (a spurious "changed" only costs a recomputation)
    const int spec_mask_changed = p->h_sc->mask_changed;
    for (;;) {
      ST(peel_round());
      CU(cudaMemcpyAsync(&p->h_sc->changed, &p->sc->changed, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
      ST(sync(p));
      if (!p->h_sc->changed || rounds >= max_rounds) break;
    }
    ST(finalize());
    p->h_sc->mask_changed |= spec_mask_changed;
  }
  p->n_cam_free = p->h_sc->n_cam_free;
  p->n_pt_act = p->h_sc->n_pt_act;
  p->n_obs_act = p->h_sc->n_obs_act;
  p->n_cam_act = p->h_sc->n_cam_act;
  if (p->h_sc->mask_changed) {
    p->cost_valid[0] = p->cost_valid[1] = false;
    p->linearized = false;
  }
  p->extracted = true;
  if (rounds_out) *rounds_out = rounds;
  return BA_OK;
}

// ---------------------------------------------------------------------------
// steps (a)-(d)
// ---------------------------------------------------------------------------

template <typename T>
ba_status linearize_t(ba_problem* pb) {
  int s = pb->cur;
  if (pb->join_pending) {
    CU(cudaStreamWaitEvent(pb->stream, pb->join, 0));
    pb->join_pending = false;
  }
  if (pb->side) CU(cudaEventRecord(pb->fork, pb->stream));
  // W rows are stored when the matvec streams them or the explicit system is formed
  LAUNCH(1, launch_pt_lin<T>(pb->L, pb->mp, (const T*)pb->camw[s], (const T*)pb->ptsw[s], pb->obs_act,
                             (pb->recompute && (!pb->explicit_S || pb->orec)) ? nullptr : (T*)pb->W,
                             pb->recompute ? (T*)pb->wsgn : nullptr, (T*)pb->V, (T*)pb->gp, pb->stream,
                             pb->orec));
  // the camera side reads neither W nor V: it runs on the side stream alongside
  cudaStream_t cs = pb->stream;
  if (pb->side) {
    CU(cudaStreamWaitEvent(pb->side, pb->fork, 0));
    cs = pb->side;
  }
  LAUNCH(1, launch_cam_accum<T>(pb->L, pb->mp, 0, (const T*)pb->camw[s], (const T*)pb->ptsw[s],
                                pb->obs_act_co, pb->cam_act, pb->crank, nullptr, nullptr,
                                (T*)pb->cam_part, cs));
  LAUNCH(1, launch_cam_reduce<T>(pb->L, (const T*)pb->cam_part, (T*)pb->Ug, cs));
  if (cs != pb->stream) {
    CU(cudaEventRecord(pb->join, cs));
    CU(cudaStreamWaitEvent(pb->stream, pb->join, 0));
  }
  pb->linearized = true;
  return BA_OK;
}

template <typename T>
ba_status schur_t(ba_problem* pb, double lambda) {
  int s = pb->cur;
  if (pb->join_pending) {  // a previous chain whose solve did not run (error path)
    CU(cudaStreamWaitEvent(pb->stream, pb->join, 0));
    pb->join_pending = false;
  }
  LAUNCH(1, launch_damp_pts<T>(pb->P, (const T*)pb->V, (const T*)pb->gp, pb->pt_act, lambda, (T*)pb->Vinv,
                               (T*)pb->z0, pb->err, pb->stream, pb->prec));
  cudaStream_t cs = pb->stream;
  if (pb->explicit_S && pb->side) {
    CU(cudaEventRecord(pb->fork, pb->stream));  // after the point damping
    CU(cudaStreamWaitEvent(pb->side, pb->fork, 0));
    cs = pb->side;
    // the Jacobi scaling the formation needs now (it depends on U* only)
    LAUNCH(1, launch_dscale<T>(pb->n_cam_free, pb->cam_map, (const T*)pb->Ug, lambda, pb->dscale, pb->stream,
                               pb->mp.cam_model == BA_CAMERA_CENTRE));
  }
  LAUNCH(1, launch_cam_accum<T>(pb->L, pb->mp, 1, (const T*)pb->camw[s], (const T*)pb->ptsw[s],
                                pb->obs_act_co, pb->cam_act, pb->crank, (const T*)pb->Vinv,
                                (const T*)pb->z0, (T*)pb->cam_part, cs));
  LAUNCH(1, launch_cam_reduce<T>(pb->L, (const T*)pb->cam_part, (T*)pb->Sg, cs));
  LAUNCH(1, launch_schur_diag<T>(pb->n_cam_free, pb->cam_map, (const T*)pb->Ug, (const T*)pb->Sg, lambda,
                                 (T*)pb->Ud, (T*)pb->Dinv, (T*)pb->bvec, (T*)pb->dampc,
                                 pb->explicit_S ? (T*)pb->Dblk : nullptr,
                                 pb->explicit_S && !pb->side ? pb->dscale : nullptr, pb->err, cs, pb->mp.cam_model == BA_CAMERA_CENTRE));
  if (cs != pb->stream) {
    CU(cudaEventRecord(pb->join, cs));
    pb->join_pending = true;
  }
  return BA_OK;
}

// (d) with an explicit reduced camera system: form S^ (scaled), PCG on it, then
// the point back-substitution and the predicted decrease.
template <typename T>
ba_status spcg_t(ba_problem* pb, double lambda) {
  int Cf = pb->n_cam_free, s = pb->cur;
  CU(cudaMemsetAsync(&pb->sc->pcg_iters, 0, sizeof(int), pb->stream));
  CU(cudaMemsetAsync(&pb->sc->pcg_rel_res, 0, sizeof(double), pb->stream));
  if (Cf > 0) {
    if (pb->reuse_system) {
      // S^ (and the dense factor) of the previous solve at the same state and damping
      if (pb->join_pending) CU(cudaStreamWaitEvent(pb->stream, pb->join, 0));
    } else {
      FormRec frec;
      frec.rec = pb->orec;
      frec.pair_pt = pb->pair_pt;
      frec.camw = pb->camw[s];
      frec.prec = pb->prec;
      frec.centre = pb->mp.cam_model == BA_CAMERA_CENTRE;
      LAUNCH(3, launch_form_S<T>(pb->L, pb->n_covis_runs, pb->covis_runs, pb->covis_pairs, (const T*)pb->W,
                                 (const T*)pb->Vinv, pb->crank, (const T*)pb->Ud, (const T*)pb->Dblk, pb->dscale,
                                 Cf, (T*)pb->Yhat, pb->sparse ? (T*)pb->Bs : (T*)pb->Shat, pb->form_lanes,
                                 pb->num_sms, pb->evf[0], pb->evf[1], pb->join_pending ? pb->join : nullptr,
                                 pb->stream, pb->cam_map, pb->sparse, pb->cform.n_blocks ? &pb->cform : nullptr,
                                 pb->orec ? &frec : nullptr));
      pb->evf_valid = true;
    }
    pb->join_pending = false;  // the main stream waits for the chain
    bool solved = false;
    if constexpr (sizeof(T) == 4) {
      if (pb->dense) {
        // b^ = D^-1 b; S^ x^ = b^ by the tensor-core factorisation + CG; x = D^-1 x^
        const int n = 9 * Cf;
        const float* dinv = reinterpret_cast<const float*>(pb->dscale + n);
        float* bh = pb->dense_b;
        float* xh = pb->dense_b + n;
        LAUNCH(1, launch_scale_vec(n, (const float*)pb->bvec, dinv, bh, pb->stream));
        CU(cudaEventRecord(pb->evk[0], pb->stream));
        DenseResult res;
        if (pb->reuse_system) res.flags = pb->dense_last.flags, res.shift = pb->dense_last.shift;
        CU(dense_spd_solve(pb->dw, (const float*)pb->Shat, spcg_row_stride<float>(n), n, bh, xh, pb->opt.pcg_rel_tol,
                           pb->opt.pcg_max_iters, pb->num_sms, pb->stream, &res, pb->reuse_system));
        CU(cudaEventRecord(pb->evk[1], pb->stream));
        pb->evk_valid = true;
        pb->launches += res.launches;
        LAUNCH(1, launch_scale_vec(n, xh, dinv, (float*)pb->x, pb->stream));
        LAUNCH(1, launch_set_pcg_info(pb->sc, res.iters, res.rel_res, pb->err,
                                      ((res.flags & 16) ? 1 : 0) | ((res.flags & 34) ? 2 : 0), pb->stream));
        pb->dense_last = res;
        solved = true;
      }
    }
    if (!solved) {
    SpcgArgs<T> a{};
    a.Shat = (const T*)pb->Shat;
    a.Dinv = (const T*)pb->Dinv;
    a.dscale = pb->dscale;
    a.b = (const T*)pb->bvec;
    a.Cf = Cf;
    a.n = 9 * Cf;
    a.rows_in_smem = pb->spcg_rows_in_smem;
    a.vecs_in_smem = pb->spcg_vecs_in_smem;
    a.scratch = (T*)pb->spcg_scratch;
    a.scratch_stride = pb->spcg_scratch_stride;
    a.Mshared = nullptr;
    if (pb->spcg_M) {
      LAUNCH(1, launch_spcg_precond<T>(Cf, (const T*)pb->Dinv, pb->dscale, (T*)pb->spcg_M, pb->stream));
      a.Mshared = (const T*)pb->spcg_M;
    }
    a.x = (T*)pb->x;
    a.words = pb->spcg_words;
    a.err = pb->err;
    a.sc = pb->sc;
    a.tol = pb->opt.pcg_rel_tol;
    a.max_iters = pb->opt.pcg_max_iters;
    a.timeout_ns = 2000000000LL;
    if (pb->sparse) {
      a.brp = pb->brp;
      a.bent = pb->bent;
      a.Bs = (const T*)pb->Bs;
      a.crank = pb->crank;
      a.cam_map = pb->cam_map;
    }
    // the block-sparse kernel owns whole cameras: at least one per block
    const int grid = std::max(1, std::min(pb->spcg_grid, pb->sparse ? Cf : (a.n + 7) / 8));
    const size_t smem = pb->sparse ? bspcg_smem_bytes<T>(Cf, grid)
                                   : spcg_smem_bytes<T>(a.n, (a.n + grid - 1) / grid, a.rows_in_smem, a.vecs_in_smem, Cf);
    if (smem > pb->spcg_smem) {
      set_error("explicit PCG launch needs %zu B of shared memory (planned %zu)", smem, pb->spcg_smem);
      return BA_ERR_INVALID_ARG;
    }
    // fresh tags for this launch; on wrap-around the words are cleared and tags restart at 1
    const unsigned span = (unsigned)a.max_iters + 3u;
    if (pb->spcg_tag == 0 || pb->spcg_tag > 0xFFFFFFFFu - span) {
      CU(cudaMemsetAsync(pb->spcg_words, 0,
                         sizeof(unsigned long long) * 2 * 9 * (size_t)pb->C * spcg_words_per_value(pb->fp64),
                         pb->stream));
      pb->spcg_tag = 1;
    }
    a.tag_base = pb->spcg_tag;
    pb->spcg_tag += span;
    CU(cudaEventRecord(pb->evk[0], pb->stream));
    if (pb->sparse) LAUNCH(1, launch_bspcg<T>(a, grid, smem, pb->stream));
    else LAUNCH(1, launch_spcg<T>(a, grid, smem, pb->stream));
    CU(cudaEventRecord(pb->evk[1], pb->stream));
    pb->evk_valid = true;
    }
  }
  if (pb->join_pending) {  // no formation ran (no free camera): still join the chain
    CU(cudaStreamWaitEvent(pb->stream, pb->join, 0));
    pb->join_pending = false;
  }
  if (pb->cand_early_ok && pb->side) {
    // dc is final: the camera candidate on the side stream, next to the back-substitution
    int sl = pb->cur, d = 1 - pb->cur;
    CU(cudaEventRecord(pb->cand_fork, pb->stream));
    CU(cudaStreamWaitEvent(pb->side, pb->cand_fork, 0));
    LAUNCH(1, launch_candidate<T>(pb->C, 0, pb->crank, (const T*)pb->x, (const T*)pb->dp, pb->cams64[sl],
                                  pb->pts64[sl], pb->cams64[d], pb->pts64[d], pb->camw64[d],
                                  pb->fp64 ? nullptr : (T*)pb->camw[d], (T*)pb->ptsw[d], pb->camdf[d], pb->ptdf[d],
                                  pb->side, pb->mp.cam_model));
    CU(cudaEventRecord(pb->cand_join, pb->side));
    pb->cand_cams_done = true;
  }
  LAUNCH(2, launch_backsub_pts<T>(pb->L, pb->mp, (const T*)pb->camw[s], (const T*)pb->ptsw[s], pb->obs_act,
                                  pb->pt_act, pb->crank, (const T*)pb->x, (const T*)pb->Vinv, (const T*)pb->V,
                                  (const T*)pb->gp, pb->orec ? nullptr : (const T*)pb->W, lambda, (T*)pb->dp,
                                  (T*)pb->bs_wx, Cf,
                                  pb->cam_map, (const T*)pb->Ug, (const T*)pb->dampc, pb->pred_parts, pb->sc,
                                  pb->bs_grid, pb->stream, pb->orec));
  return BA_OK;
}

// (d): PCG on the reduced camera system, point back-substitution and the
// predicted decrease, for the Schur terms prepared at damping lambda.
template <typename T>
ba_status pcg_t(ba_problem* pb, double lambda) {
  if (pb->explicit_S) return spcg_t<T>(pb, lambda);
  int Cf = pb->n_cam_free;
  PcgArgs<T> a{};
  a.recompute = pb->recompute;
  a.W = (const T*)pb->W;
  a.wsgn = (const T*)pb->wsgn;
  a.ptsw = (const T*)pb->ptsw[pb->cur];
  a.camw = (const T*)pb->camw[pb->cur];
  a.cam_in_smem = pb->cam_in_smem;
  a.sw_valid = pb->mp.sw_valid;
  a.sw_invalid = pb->mp.sw_invalid;
  a.max_tiles_per_block = pb->max_tiles_per_block;
  a.descs = pb->descs;
  a.meta = pb->meta;
  a.n_tiles = pb->n_tiles;
  a.stages = pb->pcg_stages;
  a.Vinv = (const T*)pb->Vinv;
  a.crank = pb->crank;
  a.C = pb->C;
  a.Ud = (const T*)pb->Ud;
  a.Dinv = (const T*)pb->Dinv;
  a.b = (const T*)pb->bvec;
  a.Cf = Cf;
  a.n = 9 * Cf;
  a.own_max = pb->pcg_own_max;
  a.x = (T*)pb->x;
  a.z = (T*)pb->z;
  a.partials = (T*)pb->partials;
  a.dots = pb->dots;
  a.bar = pb->bar;
  a.err = pb->err;
  a.sc = pb->sc;
  a.tol = pb->opt.pcg_rel_tol;
  a.max_iters = pb->opt.pcg_max_iters;
  a.timeout_ns = 2000000000LL;
  a.gp = (const T*)pb->gp;
  a.V = (const T*)pb->V;
  a.lambda = lambda;
  a.dp = (T*)pb->dp;
  a.pred_parts = pb->pred_parts;
  size_t smem = pcg_smem_bytes<T>(a.n, pb->C, pb->pcg_stages, pb->pcg_own_max, pb->recompute,
                                  pb->cam_in_smem, pb->max_tiles_per_block);
  CU(cudaMemsetAsync(pb->bar, 0, sizeof(unsigned), pb->stream));
  CU(cudaEventRecord(pb->evk[0], pb->stream));
  LAUNCH(1, launch_pcg<T>(a, pb->pcg_grid, smem, pb->stream));
  CU(cudaEventRecord(pb->evk[1], pb->stream));
  pb->evk_valid = true;
  LAUNCH(1, launch_pred_cams<T>(Cf, pb->cam_map, (const T*)pb->x, (const T*)pb->Ug, (const T*)pb->dampc,
                                lambda, pb->pred_parts, pb->pcg_grid, pb->stream));
  LAUNCH(1, launch_reduce_pred(pb->pred_parts, pb->pcg_grid + 1, pb->sc, pb->stream));
  return BA_OK;
}

template <typename T>
ba_status candidate_t(ba_problem* pb) {
  int s = pb->cur, d = 1 - pb->cur;
  const bool early = pb->cand_cams_done;
  LAUNCH(early ? 1 : 2, launch_candidate<T>(early ? 0 : pb->C, pb->P, pb->crank, (const T*)pb->x, (const T*)pb->dp,
                                            pb->cams64[s], pb->pts64[s], pb->cams64[d], pb->pts64[d],
                                            pb->camw64[d], pb->fp64 ? nullptr : (T*)pb->camw[d],
                                            (T*)pb->ptsw[d], pb->camdf[d], pb->ptdf[d], pb->stream,
                                            pb->mp.cam_model));
  if (early) CU(cudaStreamWaitEvent(pb->stream, pb->cand_join, 0));
  pb->cand_cams_done = false;
  pb->df_current[d] = !pb->fp64;  // the candidate kernels wrote its double-float copy
  pb->bits_valid[d] = false;
  pb->cost_valid[d] = false;
  return BA_OK;
}

ba_status ensure_extracted(ba_problem* pb) {
  const bool once = pb->opt.extract_mode == BA_EXTRACT_ONCE;
  if (!pb->extracted || (pb->state_changed && !once)) {
    ST(run_extraction(pb, false, nullptr));
    pb->state_changed = false;
  }
  return BA_OK;
}

ba_status ensure_linearized(ba_problem* pb) {
  ST(ensure_extracted(pb));
  if (!pb->linearized) {
    if (pb->fp64) ST(linearize_t<double>(pb));
    else ST(linearize_t<float>(pb));
  }
  return BA_OK;
}

// Damped solve at the current linearisation: (b) Schur terms, (d) PCG + back-substitution.
ba_status solve_damped(ba_problem* pb, double lambda) {
  if (pb->fp64) {
    ST(schur_t<double>(pb, lambda));
    ST(pcg_t<double>(pb, lambda));
  } else {
    ST(schur_t<float>(pb, lambda));
    ST(pcg_t<float>(pb, lambda));
  }
  return BA_OK;
}

// Implicit adjoint: undamped Schur solve of H mu = dL/dtheta (gradient slot
// replaced by -dL/dtheta), then rho'_k (J_k mu) per observation.  FP32 problems
// refine mu against the FP64 residual a - H mu (kAdjRefineSteps corrections, each
// solved by the same FP32 Schur solve), accumulate it in FP64 and form the
// outputs in FP64: the scale direction of a problem with depth priors is too
// weakly determined for a single FP32 solve.
constexpr int kAdjRefineSteps = 4;
template <typename T>
ba_status backward_t(ba_problem* pb, const double* dc, const double* dpts, double* duv, double* dd) {
  const bool refine = !pb->fp64;
  const int C = pb->C, P = pb->P, N = pb->N;
  if (refine && !pb->adj_ac) {
    ST(dalloc(pb, &pb->adj_ac, (size_t)9 * C));
    ST(dalloc(pb, &pb->adj_ap, (size_t)3 * P));
    ST(dalloc(pb, &pb->adj_muc, (size_t)9 * C));
    ST(dalloc(pb, &pb->adj_mup, (size_t)3 * P));
    ST(dalloc(pb, &pb->adj_u, (size_t)3 * N));
    ST(dalloc(pb, &pb->adj_hp, (size_t)3 * P));
    ST(dalloc(pb, &pb->adj_part, (size_t)9 * std::max(1, pb->n_chunks)));
  }
  LAUNCH(1, launch_adjoint_rhs<T>(C, P, pb->cams64[pb->cur], pb->crank, pb->pt_act, dc, dpts, (T*)pb->Ug,
                                  (T*)pb->gp, pb->stream, refine ? pb->adj_ac : nullptr,
                                  refine ? pb->adj_ap : nullptr, pb->mp.cam_model == BA_CAMERA_CENTRE));
  pb->linearized = false;  // the gradient slots now hold the adjoint right-hand side
  ST(schur_t<T>(pb, 0.0));
  ST(pcg_t<T>(pb, 0.0));
  int s = pb->cur;
  if (!refine) {
    LAUNCH(1, launch_adjoint_obs<T>(pb->L, pb->mp, (const T*)pb->camw[s], (const T*)pb->ptsw[s], pb->obs_act,
                                    pb->crank, (const T*)pb->x, (const T*)pb->dp, duv, dd, pb->stream));
    return BA_OK;
  }
  const int Cf = pb->n_cam_free;
  LAUNCH(1, launch_adj_mu_add<T>(Cf, P, (const T*)pb->x, (const T*)pb->dp, pb->adj_muc, pb->adj_mup, true,
                                 pb->stream));
  // the corrections reuse the formed S^ (explicit and block-sparse systems) or the
  // dense factor: only the reduced right-hand side, the PCG and the back-substitution run
  ba_status st = BA_OK;
  for (int r = 0; r < kAdjRefineSteps && st == BA_OK; ++r) {
    LAUNCH(2, launch_adj_hmu(pb->L, pb->mp, pb->camw64[s], pb->pts64[s], pb->obs_act, pb->obs_act_co, pb->crank,
                             pb->adj_muc, pb->adj_mup, pb->adj_u, pb->adj_hp, pb->adj_part, pb->stream));
    LAUNCH(1, launch_adj_residual<T>(C, P, pb->L.cam_chunk, pb->crank, pb->pt_act, pb->adj_part, pb->adj_hp,
                                     pb->adj_ac, pb->adj_ap, (T*)pb->Ug, (T*)pb->gp, pb->stream));
    pb->reuse_system = true;
    st = schur_t<T>(pb, 0.0);
    if (st == BA_OK) st = pcg_t<T>(pb, 0.0);
    pb->reuse_system = false;
    if (st == BA_OK)
      LAUNCH(1, launch_adj_mu_add<T>(Cf, P, (const T*)pb->x, (const T*)pb->dp, pb->adj_muc, pb->adj_mup, false,
                                     pb->stream));
  }
  ST(st);
  LAUNCH(1, launch_adjoint_obs64(pb->L, pb->mp, pb->camw64[s], pb->pts64[s], pb->obs_act, pb->crank, pb->adj_muc,
                                 pb->adj_mup, duv, dd, pb->stream));
  return BA_OK;
}

// NVTX range for the host-side enqueue of one LM phase (visible in Nsight timelines);
// ends at end() or when leaving the scope.
struct NvtxScope {
  bool open = true;
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  void end() {
    if (open) nvtxRangePop();
    open = false;
  }
  ~NvtxScope() { end(); }
};

ba_status lm_step(ba_problem* pb, ba_iter_info* info) {
  const ba_options& o = pb->opt;
  int k = pb->iter;
  // one-shot mode: the active set of the first extraction stays for the whole run
  const bool once = o.extract_mode == BA_EXTRACT_ONCE;
  bool drop = !once && o.extract_every > 0 && o.drop_residual_px > 0 && k > 0 && k % o.extract_every == 0;
  CU(cudaEventRecord(pb->ev[0], pb->stream));
  NvtxScope r_extract("ba: extract");
  if (once && pb->extracted) {
    pb->state_changed = false;
  } else if (pb->extracted && pb->state_changed && pb->same_validity && !drop) {
    // Sec. 4.2: the active set is a function of the validity bits (and the sticky
    // drops, unchanged outside drop iterations); same bits, same active set
    pb->state_changed = false;
  } else if (!pb->extracted || pb->state_changed || drop) {
    ST(run_extraction(pb, drop, nullptr));
    pb->state_changed = false;
  }
  pb->same_validity = false;
  if (!pb->cost_valid[pb->cur]) ST(eval_state(pb, pb->cur, false, true));
  CU(cudaEventRecord(pb->ev[1], pb->stream));
  r_extract.end();
  NvtxScope r_lin("ba: linearize");
  if (!pb->linearized) {
    if (pb->fp64) ST(linearize_t<double>(pb));
    else ST(linearize_t<float>(pb));
  }
  CU(cudaEventRecord(pb->ev[2], pb->stream));
  r_lin.end();
  NvtxScope r_schur("ba: schur terms");
  double lambda = pb->lambda;
  CU(cudaMemsetAsync(pb->err, 0, sizeof(int), pb->stream));
  if (pb->fp64) ST(schur_t<double>(pb, lambda));
  else ST(schur_t<float>(pb, lambda));
  // end of the Schur terms: on the side stream when the chain runs there (the
  // formation of S^ on the main stream overlaps it and is counted in the solve)
  CU(cudaEventRecord(pb->ev[3], pb->join_pending ? pb->side : pb->stream));
  r_schur.end();
  NvtxScope r_solve("ba: solve");
  pb->evk_valid = false;
  pb->evf_valid = false;
  pb->cand_early_ok = true;
  ba_status solve_st = pb->fp64 ? pcg_t<double>(pb, lambda) : pcg_t<float>(pb, lambda);
  pb->cand_early_ok = false;
  if (solve_st != BA_OK && pb->cand_cams_done) {  // the step stops here: settle the early kernel
    CU(cudaStreamWaitEvent(pb->stream, pb->cand_join, 0));
    pb->cand_cams_done = false;
  }
  ST(solve_st);
  CU(cudaEventRecord(pb->ev[4], pb->stream));
  CU(cudaEventRecord(pb->ev[5], pb->stream));
  r_solve.end();
  NvtxScope r_eval("ba: candidate + evaluate");
  if (pb->fp64) ST(candidate_t<double>(pb));
  else ST(candidate_t<float>(pb));
  int nxt = 1 - pb->cur;
  ST(eval_state(pb, nxt, true, true, pb->cur));
  const bool flips_known = pb->flips_known;
  CU(cudaEventRecord(pb->ev[6], pb->stream));
  CU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  int h_err = 0;
  CU(cudaMemcpyAsync(&h_err, pb->err, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
  ST(sync(pb));
  const Scalars& s = *pb->h_sc;
  double F = s.cost[pb->cur], Fc = s.cost[nxt], pred = s.pred;
  double gain = (F - Fc) / pred;
  bool timeout = (h_err & 1) != 0;
  bool ok = std::isfinite(Fc) && std::isfinite(gain) && pred > 0.0 && !timeout;
  bool accept = ok && gain > 1e-3;
  double n_act = s.n_act[pb->cur];
  if (info) {
    memset(info, 0, sizeof *info);
    info->cost = F;
    info->rmse_px = n_act > 0 ? std::sqrt(s.rmse_sum[pb->cur] / n_act) : 0.0;
    info->lambda = lambda;
    info->gain = gain;
    info->pred_decrease = pred;
    info->cand_cost = Fc;
    info->accepted = accept ? 1 : 0;
    info->pcg_iters = s.pcg_iters;
    info->pcg_rel_res = s.pcg_rel_res;
    info->n_cam_act = pb->n_cam_act;
    info->n_pt_act = pb->n_pt_act;
    info->n_obs_act = pb->n_obs_act;
    for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&info->ms[i], pb->ev[i], pb->ev[i + 1]);
    cudaEventElapsedTime(&info->ms[6], pb->ev[0], pb->ev[6]);
    info->ms[4] = 0.f;
    if (pb->evk_valid) cudaEventElapsedTime(&info->ms[4], pb->evk[0], pb->evk[1]);
    if (pb->evf_valid) cudaEventElapsedTime(&info->ms[7], pb->evf[0], pb->evf[1]);
  }
  if (accept) {
    pb->cur = nxt;
    pb->state_changed = true;
    pb->same_validity = flips_known && s.valid_flips == 0;
    pb->linearized = false;
    double t = 2.0 * gain - 1.0;
    pb->lambda = lambda * std::max(1.0 / 3.0, 1.0 - t * t * t);
    pb->nu = 2.0;
  } else {
    pb->lambda = lambda * pb->nu;
    pb->nu *= 2.0;
  }
  pb->iter++;
  pb->solved = true;
  if (timeout) {
    set_error("PCG grid barrier timed out");
    return BA_ERR_TIMEOUT;
  }
  if (!ok) return BA_ERR_NONFINITE;
  if (s.pcg_iters >= o.pcg_max_iters && s.pcg_rel_res > o.pcg_rel_tol) return BA_ERR_NOT_CONVERGED;
  return BA_OK;
}

ba_status create_impl(const ba_options* opts, void* stream, int64_t n_cams, const double* cams,
                      int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                      const int32_t* obs_pt, const double* obs_uv, const double* depth,
                      ba_problem* pb) {
  if (!opts || !finite_opts(opts)) {
    set_error("invalid options");
    return BA_ERR_INVALID_ARG;
  }
  // N < 2^30 keeps every 32-bit index of the kernels plus its grid stride below 2^31
  if (n_cams < 0 || n_pts < 0 || n_obs < 0 || n_cams >= (1LL << 24) || n_pts >= (1LL << 30) ||
      n_obs >= (1LL << 30)) {
    set_error("sizes out of range");
    return BA_ERR_INVALID_ARG;
  }
  if ((n_cams && !cams) || (n_pts && !pts) || (n_obs && (!obs_cam || !obs_pt || !obs_uv || !depth))) {
    set_error("null input array");
    return BA_ERR_INVALID_ARG;
  }
  pb->opt = *opts;
  pb->fixed_list.assign(opts->fixed_cams, opts->fixed_cams + (opts->fixed_cams ? opts->n_fixed : 0));
  pb->opt.fixed_cams = nullptr;
  pb->stream = (cudaStream_t)stream;
  pb->fp64 = opts->precision == BA_FP64;
  pb->lambda = opts->lambda0;
  const int C = (int)n_cams, P = (int)n_pts, N = (int)n_obs;
  pb->C = C;
  pb->P = P;
  pb->N = N;
  CU(cudaGetDevice(&pb->device));
  CU(cudaDeviceGetAttribute(&pb->num_sms, cudaDevAttrMultiProcessorCount, pb->device));

  // ---- inputs on the device: device arrays are used in place, host arrays are
  // uploaded once into scratch
  const bool dev_cams = C && on_device(cams), dev_pts = P && on_device(pts);
  const bool dev_oc = N && on_device(obs_cam), dev_op = N && on_device(obs_pt);
  const bool dev_uv = N && on_device(obs_uv), dev_depth = N && on_device(depth);
  // inputs written by device work on any stream are complete before they are read
  if (dev_cams || dev_pts || dev_oc || dev_op || dev_uv || dev_depth) CU(cudaDeviceSynchronize());
  DevScratch scratch;
  // the values (cameras, points, pixels, depths) upload on a second stream behind
  // the observation indices, overlapping the index sorts of the layout; destroyed
  // (after its copies end) before the scratch they land in
  struct ValueStream {
    cudaStream_t s = nullptr;
    cudaEvent_t idx_done = nullptr;
    ~ValueStream() {
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
      if (idx_done) cudaEventDestroy(idx_done);
    }
  } vals;
  const double *d_cams = cams, *d_pts = pts, *d_uv = obs_uv, *d_depth = depth;
  const int32_t *d_oc = obs_cam, *d_op = obs_pt;
  {
    struct Up {
      const void* src;
      size_t bytes;
      bool dev;
      const void** dst;
      bool value;
    } ups[] = {{obs_cam, sizeof(int32_t) * (size_t)N, dev_oc, (const void**)&d_oc, false},
               {obs_pt, sizeof(int32_t) * (size_t)N, dev_op, (const void**)&d_op, false},
               {cams, sizeof(double) * 9 * (size_t)C, dev_cams, (const void**)&d_cams, true},
               {pts, sizeof(double) * 3 * (size_t)P, dev_pts, (const void**)&d_pts, true},
               {obs_uv, sizeof(double) * 2 * (size_t)N, dev_uv, (const void**)&d_uv, true},
               {depth, sizeof(double) * (size_t)N, dev_depth, (const void**)&d_depth, true}};
    size_t total = 0;
    bool host_values = false;
    for (const Up& u : ups)
      if (!u.dev && u.bytes) {
        total += (u.bytes + 255) / 256 * 256;
        host_values |= u.value;
      }
    if (total) {
      CU(cached_malloc(&scratch.p, total));
      if (host_values) {
        CU(cudaStreamCreateWithFlags(&vals.s, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&vals.idx_done, cudaEventDisableTiming));
      }
      char* at = static_cast<char*>(scratch.p);
      for (int pass = 0; pass < 2; ++pass) {  // the indices, then the values
        if (pass == 1 && vals.s) {
          CU(cudaEventRecord(vals.idx_done, pb->stream));
          CU(cudaStreamWaitEvent(vals.s, vals.idx_done, 0));
        }
        for (const Up& u : ups)
          if (u.value == (pass == 1) && !u.dev && u.bytes) {
            CU(cudaMemcpyAsync(at, u.src, u.bytes, cudaMemcpyHostToDevice, u.value && vals.s ? vals.s : pb->stream));
            *u.dst = at;
            at += (u.bytes + 255) / 256 * 256;
          }
      }
    }
  }
  // ---- validation and the observation layout (device; the grouping of points
  // into tiles on the host)
  auto dev_alloc = [pb](size_t bytes) -> void* {
    void* q = nullptr;
    return dalloc_bytes(pb, &q, bytes) == BA_OK ? q : nullptr;
  };
  DevLayout dl;
  {
    std::string msg;
    const int rc =
        build_obs_layout_dev(C, P, N, d_cams, d_pts, d_uv, d_oc, d_op, dev_alloc, pb->stream, vals.s, &dl, &msg);
    if (rc) {
      set_error("%s", msg.c_str());
      return rc == 1 ? BA_ERR_INVALID_ARG : rc == 3 ? BA_ERR_OOM : BA_ERR_CUDA;
    }
  }
  pb->obs_hash = dl.obs_hash;
  std::vector<uint8_t> h_fixed((size_t)C, 0);
  for (int32_t f : pb->fixed_list) {
    if (f < 0 || f >= C) { set_error("fixed camera %d out of range", f); return BA_ERR_INVALID_ARG; }
    h_fixed[f] = 1;
  }
  pb->n_tiles = dl.n_tiles;
  pb->g_rows = dl.g_rows;
  pb->w_rows = N;
  pb->n_chunks = dl.n_chunks;
  pb->po_orig = dl.po;
  pb->pt_off = dl.pt_off;
  pb->chunk_obs = dl.chunk_obs;
  pb->chunk_cam = dl.chunk_cam;
  pb->cam_chunk = dl.cam_chunk;
  pb->descs = dl.descs;
  pb->meta = dl.meta;
  pb->po_cam = dl.po_cam;
  pb->po_pt = dl.po_pt;
  pb->co_po = dl.co_po;

  // ---- per-observation arrays in both orders, gathered on the device
  ST(dalloc(pb, &pb->po_wrow, (size_t)N));
  ST(dalloc(pb, &pb->co_pt, (size_t)N));
  ST(dalloc(pb, &pb->po_uv64, (size_t)2 * N));
  ST(dalloc(pb, &pb->po_tau64, (size_t)N));
  const size_t Rw = pb->fp64 ? sizeof(double) : sizeof(float);
  if (pb->fp64) {
    pb->po_uvw = pb->po_uv64;
    pb->po_tauw = pb->po_tau64;
  } else {
    ST(dalloc_bytes(pb, &pb->po_uvw, Rw * 2 * (size_t)N));
    ST(dalloc_bytes(pb, &pb->po_tauw, Rw * (size_t)N));
  }
  ST(dalloc_bytes(pb, &pb->co_uvw, Rw * 2 * (size_t)N));
  ST(dalloc_bytes(pb, &pb->co_tauw, Rw * (size_t)N));
  if (N) {
    if (pb->fp64)
      LAUNCH(2, launch_obs_layout<double>(N, d_uv, d_depth, dl.po, dl.co, dl.co_po, dl.po_pt, pb->po_wrow,
                                          pb->po_uv64, pb->po_tau64, nullptr, nullptr, pb->co_pt,
                                          (double*)pb->co_uvw, (double*)pb->co_tauw, pb->stream));
    else
      LAUNCH(2, launch_obs_layout<float>(N, d_uv, d_depth, dl.po, dl.co, dl.co_po, dl.po_pt, pb->po_wrow,
                                         pb->po_uv64, pb->po_tau64, (float*)pb->po_uvw, (float*)pb->po_tauw,
                                         pb->co_pt, (float*)pb->co_uvw, (float*)pb->co_tauw, pb->stream));
  }
  if (!pb->fp64) {
    ST(dalloc(pb, &pb->po_uvdf, (size_t)N));
    ST(dalloc(pb, &pb->po_taudf, (size_t)N));
    for (int sl = 0; sl < 2; ++sl) {
      ST(dalloc(pb, &pb->camdf[sl], (size_t)16 * C));
      ST(dalloc(pb, &pb->ptdf[sl], (size_t)2 * P));
    }
    if (N) LAUNCH(1, launch_obs_df(N, pb->po_uv64, pb->po_tau64, pb->po_uvdf, pb->po_taudf, pb->stream));
  }
  ST(dalloc(pb, &pb->cam_fixed, (size_t)C));
  if (C) CU(cudaMemcpy(pb->cam_fixed, h_fixed.data(), (size_t)C, cudaMemcpyHostToDevice));

  Layout& L = pb->L;
  L.C = C;
  L.P = P;
  L.N = N;
  L.n_tiles = pb->n_tiles;
  L.n_chunks = pb->n_chunks;
  L.po_cam = pb->po_cam;
  L.po_pt = pb->po_pt;
  L.po_orig = pb->po_orig;
  L.po_uv64 = pb->po_uv64;
  L.po_tau64 = pb->po_tau64;
  L.po_uvdf = pb->po_uvdf;
  L.po_taudf = pb->po_taudf;
  L.po_uvw = pb->po_uvw;
  L.po_tauw = pb->po_tauw;
  L.pt_off = pb->pt_off;
  L.co_pt = pb->co_pt;
  L.co_po = pb->co_po;
  L.co_uvw = pb->co_uvw;
  L.co_tauw = pb->co_tauw;
  L.descs = pb->descs;
  L.po_wrow = pb->po_wrow;
  L.chunk_obs = pb->chunk_obs;
  L.chunk_cam = pb->chunk_cam;
  L.cam_chunk = pb->cam_chunk;
  L.cam_fixed = pb->cam_fixed;

  ModelParams& mp = pb->mp;
  mp.cam_model = opts->camera_model;
  mp.cx = opts->cx;
  mp.cy = opts->cy;
  mp.huber = opts->huber_delta;
  mp.sw_valid = std::sqrt(opts->depth_weight);
  mp.sw_invalid = std::sqrt(opts->invalid_depth_weight);
  mp.min_depth = opts->min_depth;
  mp.drop_px = opts->drop_residual_px;
  mp.img_w = opts->img_w;
  mp.img_h = opts->img_h;

  const size_t R = rsz(pb);
  for (int s = 0; s < 2; ++s) {
    ST(dalloc(pb, &pb->cams64[s], (size_t)C * 9));
    ST(dalloc(pb, &pb->pts64[s], (size_t)P * 3));
    ST(dalloc(pb, &pb->camw64[s], (size_t)C * kCamStride));
    if (pb->fp64) pb->camw[s] = pb->camw64[s];
    else ST(dalloc_bytes(pb, &pb->camw[s], R * (size_t)C * kCamStride));
    ST(dalloc_bytes(pb, &pb->ptsw[s], R * ((size_t)P + 2) * 4));
    CU(cudaMemset(pb->ptsw[s], 0, R * ((size_t)P + 2) * 4));
    ST(dalloc(pb, &pb->bits[s], (size_t)N));
  }
  if (C) CU(cudaMemcpyAsync(pb->cams64[0], d_cams, sizeof(double) * 9 * (size_t)C, cudaMemcpyDeviceToDevice, pb->stream));
  if (P) CU(cudaMemcpyAsync(pb->pts64[0], d_pts, sizeof(double) * 3 * (size_t)P, cudaMemcpyDeviceToDevice, pb->stream));
  ST(dalloc(pb, &pb->alive, (size_t)N));
  ST(dalloc(pb, &pb->valid, (size_t)N));
  ST(dalloc(pb, &pb->obs_act, (size_t)N));
  ST(dalloc(pb, &pb->obs_act_co, (size_t)N));
  ST(dalloc(pb, &pb->cam_act, (size_t)C));
  ST(dalloc(pb, &pb->pt_act, (size_t)P));
  ST(dalloc(pb, &pb->cam_flags, (size_t)C));
  ST(dalloc(pb, &pb->cam_cnt, (size_t)C));
  ST(dalloc(pb, &pb->crank, (size_t)C));
  ST(dalloc(pb, &pb->cam_map, (size_t)C));
  ST(dalloc(pb, &pb->pt_rank, (size_t)P));
  ST(dalloc(pb, &pb->pt_map, (size_t)P));
  pb->n_rank_tmp = rank_blocks(std::max(C, P)) + 1;
  ST(dalloc(pb, &pb->rank_tmp, (size_t)pb->n_rank_tmp));
  ST(dalloc(pb, &pb->counts, 8));
  if (N) CU(cudaMemset(pb->alive, 1, (size_t)N));
  if (N) CU(cudaMemset(pb->obs_act, 0, (size_t)N));

  // FP32 recomputes the W blocks inside the Schur matvec from a signed IRLS weight
  // per observation; FP64 stores them (FP64 arithmetic is the scarce resource there)
  pb->recompute = pb->fp64 ? 0 : 1;
  bool auto_sparse_cand = false;
  double auto_t_exp = 1e300, auto_t_imp = 1e300, auto_pairs = 0.0;
  {
    int so = opts->solver;
    if (so != BA_SOLVER_AUTO && so != BA_SOLVER_IMPLICIT && so != BA_SOLVER_EXPLICIT && so != BA_SOLVER_DENSE &&
        so != BA_SOLVER_SPARSE) {
      set_error("unknown solver %d", so);
      return BA_ERR_INVALID_ARG;
    }
    if (so == BA_SOLVER_DENSE && pb->fp64) {
      set_error("BA_SOLVER_DENSE needs BA_FP32 (the factorisation runs on TF32 tensor cores)");
      return BA_ERR_INVALID_ARG;
    }
    // The dense tensor-core solve is opt-in: on the 12M-observation dense
    // workload (2,000 cameras) forming S from 174M co-visible pairs alone costs
    // about as much as the whole implicit block-Jacobi PCG, which converges in
    // 25-46 iterations there; AUTO therefore never picks it.
    const bool dense = so == BA_SOLVER_DENSE;
    pb->dense = dense;
    bool auto_explicit = false;
    if (so == BA_SOLVER_AUTO) {
      if (9 * C <= 4608) {
        auto_explicit = true;  // S^ rows in shared memory: a few microseconds per PCG iteration
      } else {
        // Per-LM-step cost model, constants measured on this part (FP32, 148 SMs):
        // explicit = forming S^ (0.1 ns per co-visible pair, 3 passes of 4 n^2 bytes,
        // 50 ps per observation for Y^) + iterations x (4 n^2 bytes streamed at
        // 4.9 TB/s + 10 us); implicit = iterations x (66 ps per observation +
        // 245 ps per point).  40 iterations assumed (25-70 measured on the
        // large and dense workloads).  A function of the problem's sizes only,
        // so the choice is deterministic.
        double pairs = 0.0;
        for (int p = 0; p < P; ++p) {
          const double t = (double)(dl.h_pt_off[p + 1] - dl.h_pt_off[p]);
          pairs += 0.5 * t * (t - 1.0);
        }
        const double n = 9.0 * C, it = 40.0;
        const double t_exp = pairs * 0.1e-9 + 3.0 * 4.0 * n * n / 6.5e12 + N * 50e-12 +
                             it * (4.0 * n * n / 4.9e12 + 10e-6);
        const double t_imp = it * (N * 66e-12 + P * 245e-12);
        // and only within the explicit system's memory bound below
        const bool exp_fits = (size_t)81 * C * C * (R + 8) <= ((size_t)8 << 30);
        auto_explicit = t_exp < t_imp && exp_fits;
        // the block-sparse system is priced once the co-visibility runs are known
        auto_sparse_cand = true;
        auto_t_exp = exp_fits ? t_exp : 1e300;
        auto_t_imp = t_imp;
        auto_pairs = pairs;
      }
    }
    pb->sparse = so == BA_SOLVER_SPARSE;
    pb->explicit_S = dense || so == BA_SOLVER_EXPLICIT || pb->sparse || auto_explicit || auto_sparse_cand;
    if (pb->explicit_S && !pb->sparse && !auto_sparse_cand &&
        (size_t)81 * C * C * (R + (dense ? 4 : 8)) > ((size_t)(dense ? 24 : 8) << 30)) {
      set_error("explicit reduced camera system of order %d is too large", 9 * C);
      return BA_ERR_INVALID_ARG;
    }
  }
  if (pb->recompute) {
    ST(dalloc_bytes(pb, &pb->wsgn, R * ((size_t)pb->g_rows + 4)));
    CU(cudaMemset(pb->wsgn, 0, R * ((size_t)pb->g_rows + 4)));
  }
  ST(dalloc_bytes(pb, &pb->V, R * 6 * (size_t)P));
  ST(dalloc_bytes(pb, &pb->gp, R * 3 * (size_t)P));
  ST(dalloc_bytes(pb, &pb->Vinv, R * 6 * ((size_t)P + 2)));
  CU(cudaMemset(pb->Vinv, 0, R * 6 * ((size_t)P + 2)));
  ST(dalloc_bytes(pb, &pb->z0, R * 3 * (size_t)P));
  ST(dalloc_bytes(pb, &pb->dp, R * 3 * (size_t)P));
  ST(dalloc_bytes(pb, &pb->Ug, R * 54 * (size_t)C));
  ST(dalloc_bytes(pb, &pb->Sg, R * 54 * (size_t)C));
  ST(dalloc_bytes(pb, &pb->cam_part, R * 54 * (size_t)std::max(1, pb->n_chunks)));
  ST(dalloc_bytes(pb, &pb->Ud, R * 45 * (size_t)C));
  ST(dalloc_bytes(pb, &pb->Dinv, R * 81 * (size_t)C));
  ST(dalloc_bytes(pb, &pb->dampc, R * 9 * (size_t)C));
  for (void** v : {&pb->bvec, &pb->x, &pb->z})
    ST(dalloc_bytes(pb, v, R * 9 * (size_t)C));

  // persistent PCG grid: every block resident (cooperative launch); double-buffered
  // tile copies when the shared memory allows, else a single buffer
  int n_max = 9 * C;
  int dev_smem_optin = 0;
  CU(cudaDeviceGetAttribute(&dev_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pb->device));
  // owned camera slice and tile count per block: at most ceil(x / min(SMs, tiles))
  {
    int gmin = std::max(1, std::min(pb->num_sms, pb->n_tiles));
    pb->pcg_own_max = std::max(1, (C + gmin - 1) / gmin);
    pb->max_tiles_per_block = std::max(1, (pb->n_tiles + gmin - 1) / gmin);
  }
  pb->cam_in_smem = (pb->recompute && R * (size_t)C * kCamStride <= 48 * 1024) ? 1 : 0;
  pb->pcg_stages = pb->recompute ? 3 : 2;
  for (;;) {
    pb->pcg_smem = pb->fp64 ? pcg_smem_bytes<double>(n_max, C, pb->pcg_stages, pb->pcg_own_max, pb->recompute,
                                                     pb->cam_in_smem, pb->max_tiles_per_block)
                            : pcg_smem_bytes<float>(n_max, C, pb->pcg_stages, pb->pcg_own_max, pb->recompute,
                                                    pb->cam_in_smem, pb->max_tiles_per_block);
    if (pb->pcg_smem <= (size_t)dev_smem_optin) break;
    if (pb->cam_in_smem) {
      pb->cam_in_smem = 0;
      continue;
    }
    if (pb->pcg_stages == 1) break;
    pb->pcg_stages -= 1;
  }
  if (pb->pcg_smem > (size_t)dev_smem_optin) {
    // the implicit kernel keeps the camera vectors in shared memory; an explicit
    // system (chosen, or a candidate of AUTO) needs none of it
    if (!pb->explicit_S) {
      set_error("camera system of %d cameras needs %zu B of shared memory per block (limit %d)", C,
                pb->pcg_smem, dev_smem_optin);
      return BA_ERR_INVALID_ARG;
    }
    auto_t_imp = 1e300;
    pb->pcg_grid = 1;
  } else {
    const void* kfn = pb->fp64 ? pcg_kernel_ptr<double>() : pcg_kernel_ptr<float>();
    CU(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pb->pcg_smem));
    int per_sm = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, pcg_threads(), pb->pcg_smem));
    if (per_sm < 1) {
      set_error("PCG kernel cannot be resident");
      return BA_ERR_INVALID_ARG;
    }
    // at most two blocks per SM: fewer blocks means fewer partial vectors to reduce
    pb->pcg_grid = std::max(1, std::min(std::min(per_sm, 2) * pb->num_sms, std::max(1, pb->n_tiles)));
  }
  ST(dalloc_bytes(pb, &pb->partials, R * (size_t)pb->pcg_grid * std::max(1, n_max)));
  // dot-product slots of the implicit PCG kernel: [2 parities][grid][4]
  ST(dalloc(pb, &pb->dots, (size_t)2 * 4 * pb->pcg_grid));
  ST(dalloc(pb, &pb->bar, 1));
  ST(dalloc(pb, &pb->err, 1));
  // co-visibility runs: every pair of observations of one point in cameras i < j,
  // grouped by (i, j), ascending in point within a run (device); the explicit
  // systems are formed over them
  if (pb->explicit_S && n_max > 0) {
    DevCovis cv;
    std::string msg;
    const int rc = build_covis_runs_dev(dl, C, N, dev_alloc, pb->stream, &cv, &msg);
    if (rc) {
      set_error("%s", msg.c_str());
      return rc == 1 ? BA_ERR_INVALID_ARG : rc == 3 ? BA_ERR_OOM : BA_ERR_CUDA;
    }
    pb->covis_pairs = cv.pairs;
    pb->covis_runs = cv.runs;
    pb->n_covis_runs = cv.n_runs;
    // one lane per run when there are enough runs for four blocks of 128 lanes
    // per SM and runs are short (a warp per run would idle in its reduction)
    pb->form_lanes = (long long)cv.n_runs >= 4LL * 128 * pb->num_sms && cv.npairs < 128 * (size_t)cv.n_runs;
    // FP32 with very many short runs (the lane-per-run regime: ~1,000 runs per camera
    // on the 2,000-camera dense workload): camera-owned formation.  With few runs
    // per camera its blocks would hold few live lanes, each walking its run's pairs
    // one dependent gather at a time; the warp-per-run kernel is faster there
    // (0.23 against 0.50 ms on the 200-camera bench workload).
    // FP32 with fewer, longer runs (the warp-per-run kernel): the blocks are formed
    // from observation records (k_form_S_rec) unless BA_FORM_RECORDS=0 keeps the Y^ rows
    const char* frv = std::getenv("BA_FORM_RECORDS");
    if (!pb->fp64 && !pb->form_lanes && cv.n_runs > 0 && !(frv && frv[0] == '0')) {
      ST(dalloc(pb, &pb->orec, (size_t)16 * std::max(N, 1)));
      CU(cudaMemset(pb->orec, 0, sizeof(float) * 16 * (size_t)std::max(N, 1)));
      ST(dalloc(pb, &pb->pair_pt, std::max<size_t>(cv.npairs, 1)));
      ST(dalloc(pb, &pb->prec, (size_t)8 * std::max(P, 1)));
      CU(cudaMemset(pb->prec, 0, sizeof(float) * 8 * (size_t)std::max(P, 1)));
      LAUNCH(1, launch_pair_pt(cv.npairs, cv.pairs, dl.po_pt, pb->pair_pt, pb->stream));
    }
    if (!pb->fp64 && pb->form_lanes) {
      // runs grouped by owner camera, blocks of up to 128 runs
      int* po_co = nullptr;
      ST(dalloc(pb, &po_co, (size_t)N));
      LAUNCH(2, launch_owner_pairs(N, dl.co_po, po_co, cv.n_runs, cv.runs, cv.pairs, pb->stream));
      std::vector<int4> h_runs((size_t)cv.n_runs);
      CU(cudaMemcpy(h_runs.data(), cv.runs, sizeof(int4) * (size_t)cv.n_runs, cudaMemcpyDeviceToHost));
      std::vector<int> own_off((size_t)C + 1, 0), own((size_t)cv.n_runs);
      auto owner = [](const int4& r) { return run_owner_first(r.x, r.y) ? r.x : r.y; };
      for (const int4& r : h_runs) own_off[owner(r) + 1]++;
      for (int c = 0; c < C; ++c) own_off[c + 1] += own_off[c];
      {
        std::vector<int> fill(own_off.begin(), own_off.end() - 1);
        for (int r = 0; r < cv.n_runs; ++r) own[fill[owner(h_runs[r])]++] = r;
      }
      std::vector<int4> blocks;
      for (int c = 0; c < C; ++c)
        for (int g = own_off[c]; g < own_off[c + 1]; g += 128)
          blocks.push_back(make_int4(c, g, std::min(128, own_off[c + 1] - g), 0));
      int* d_own = nullptr;
      int4* d_blocks = nullptr;
      ST(dalloc(pb, &d_own, own.size()));
      ST(dalloc(pb, &d_blocks, blocks.size()));
      CU(cudaMemcpy(d_own, own.data(), sizeof(int) * own.size(), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(d_blocks, blocks.data(), sizeof(int4) * blocks.size(), cudaMemcpyHostToDevice));
      pb->cform.blocks = d_blocks;
      pb->cform.n_blocks = (int)blocks.size();
      pb->cform.own_run = d_own;
      pb->cform.cam_off = dl.cam_off;
      pb->cform.po_co = po_co;
    }
    if (auto_sparse_cand) {
      // AUTO, priced now that the co-visible camera pairs are known: the
      // block-sparse system forms the same blocks and streams its 2 n_runs + C
      // stored blocks per PCG iteration (~4 TB/s from L2 and HBM) + 8 us
      const double nblk = 2.0 * cv.n_runs + C, it = 40.0;
      const double t_sp = auto_pairs * 0.1e-9 + N * 50e-12 + it * (nblk * kBlkStride * R / 4e12 + 8e-6);
      if (t_sp < auto_t_exp && t_sp < auto_t_imp) pb->sparse = true;
      else if (!(auto_t_exp < auto_t_imp)) pb->explicit_S = false;
    }
    if (pb->sparse && (size_t)(2 * (size_t)cv.n_runs + C) * kBlkStride * R > ((size_t)16 << 30)) {
      set_error("block-sparse reduced camera system of %d blocks is too large", 2 * cv.n_runs + C);
      return BA_ERR_INVALID_ARG;
    }
    if (pb->sparse) {
      // block rows by camera: the transposed blocks of runs (j, c) (ascending j < c),
      // the diagonal block, the blocks of runs (c, j) (ascending j > c)
      std::vector<int4> h_runs((size_t)cv.n_runs);
      if (cv.n_runs)
        CU(cudaMemcpy(h_runs.data(), cv.runs, sizeof(int4) * (size_t)cv.n_runs, cudaMemcpyDeviceToHost));
      std::vector<int> rp((size_t)C + 1, 0), fill;
      for (const int4& r : h_runs) rp[r.x + 1]++, rp[r.y + 1]++;
      for (int c = 0; c < C; ++c) rp[c + 1] += rp[c] + 1;
      fill.assign(rp.begin(), rp.end() - 1);
      std::vector<int2> ent((size_t)rp[C]);
      for (int r = 0; r < cv.n_runs; ++r) ent[fill[h_runs[r].y]++] = make_int2(h_runs[r].x, 2 * r + 1);
      for (int c = 0; c < C; ++c) ent[fill[c]++] = make_int2(c, 2 * cv.n_runs + c);
      for (int r = 0; r < cv.n_runs; ++r) ent[fill[h_runs[r].x]++] = make_int2(h_runs[r].y, 2 * r);
      ST(dalloc(pb, &pb->brp, (size_t)C + 1));
      ST(dalloc(pb, &pb->bent, ent.size()));
      CU(cudaMemcpy(pb->brp, rp.data(), sizeof(int) * rp.size(), cudaMemcpyHostToDevice));
      if (!ent.empty()) CU(cudaMemcpy(pb->bent, ent.data(), sizeof(int2) * ent.size(), cudaMemcpyHostToDevice));
      ST(dalloc_bytes(pb, &pb->Bs, R * kBlkStride * (2 * (size_t)cv.n_runs + C)));
    }
  }
  // W rows: streamed by the FP64 matvec, read by the Y^ pass and the
  // back-substitution of explicit systems formed from Y^ (not with records)
  if (!pb->recompute || (pb->explicit_S && !pb->orec)) {
    ST(dalloc_bytes(pb, &pb->W, R * kWStride * ((size_t)pb->w_rows + 1)));
    CU(cudaMemset(pb->W, 0, R * kWStride * ((size_t)pb->w_rows + 1)));
  }
  // explicit reduced camera system (solver option; automatic for up to 512 cameras)
  if (pb->explicit_S && n_max > 0) {
    if (!pb->sparse)
      ST(dalloc_bytes(pb, &pb->Shat, R * (size_t)n_max * (pb->fp64 ? spcg_row_stride<double>(n_max) : spcg_row_stride<float>(n_max))));
    if (!pb->orec) ST(dalloc_bytes(pb, &pb->Yhat, R * (size_t)kWStride * ((size_t)N + 1)));
    ST(dalloc_bytes(pb, &pb->bs_wx, R * 3 * std::max<size_t>(N, 1)));  // W_k^T dc per observation
    ST(dalloc(pb, &pb->dscale, (size_t)2 * n_max));  // D, then 1/D in the working precision
    ST(dalloc_bytes(pb, &pb->Dblk, R * 45 * (size_t)C));
    if (pb->dense) {
      const size_t np = ((size_t)n_max + 127) / 128 * 128;
      ST(dalloc(pb, &pb->dw.A, np * np));
      ST(dalloc(pb, &pb->dw.Linv, np * 128));
      ST(dalloc(pb, &pb->dw.vec, 4 * np));
      ST(dalloc(pb, &pb->dw.part, (size_t)256));
      ST(dalloc(pb, &pb->dw.scal, (size_t)8));
      ST(dalloc(pb, &pb->dw.flags, np / 128));
      CU(cudaMemset(pb->dw.flags, 0, sizeof(unsigned) * (np / 128)));
      ST(dalloc(pb, &pb->dw.err, (size_t)1));
      ST(dalloc(pb, &pb->dense_b, 2 * (size_t)n_max));
      pb->dw.epoch = &pb->dense_epoch;
    }
    // one block per SM, at least 8 rows of S^ per block; rows per block at most
    // ceil(n / grid) for every later (smaller) number of free cameras
    pb->spcg_grid = std::max(1, std::min(pb->num_sms, (n_max + 7) / 8));
    {
      // shared memory, most useful first: p, then r, z, q, x and M^, then the rows
      const int rows_max = std::max(8, (n_max + pb->spcg_grid - 1) / pb->spcg_grid);
      auto bytes = [&](int rows_in, int vecs_in) {
        return pb->fp64 ? spcg_smem_bytes<double>(n_max, rows_max, rows_in, vecs_in, C)
                        : spcg_smem_bytes<float>(n_max, rows_max, rows_in, vecs_in, C);
      };
      pb->spcg_rows_in_smem = pb->spcg_vecs_in_smem = 1;
      if (pb->sparse || bytes(1, 1) > (size_t)dev_smem_optin) pb->spcg_rows_in_smem = 0;
      if (!pb->spcg_rows_in_smem && bytes(0, 1) > (size_t)dev_smem_optin) pb->spcg_vecs_in_smem = 0;
      pb->spcg_smem = bytes(pb->spcg_rows_in_smem, pb->spcg_vecs_in_smem);
      if (pb->spcg_smem > (size_t)dev_smem_optin) {
        set_error("explicit PCG of order %d needs %zu B of shared memory per block (limit %d)", n_max,
                  pb->spcg_smem, dev_smem_optin);
        return BA_ERR_INVALID_ARG;
      }
      if (!pb->spcg_vecs_in_smem) {
        // r, z, q, x per block (the preconditioner blocks are shared: spcg_M)
        pb->spcg_scratch_stride =
            (size_t)4 * (pb->fp64 ? spcg_row_stride<double>(n_max) : spcg_row_stride<float>(n_max));
        ST(dalloc_bytes(pb, &pb->spcg_scratch, R * pb->spcg_scratch_stride * pb->spcg_grid));
        ST(dalloc_bytes(pb, &pb->spcg_M, R * (size_t)kSpcgMStride * std::max(1, C)));
      }
    }
    {
      const size_t nw = (size_t)2 * n_max * spcg_words_per_value(pb->fp64);
      ST(dalloc(pb, &pb->spcg_words, nw));
      CU(cudaMemset(pb->spcg_words, 0, sizeof(unsigned long long) * nw));
    }
    if (pb->sparse) {
      // partitioned PCG: each block keeps its cameras' slices only
      pb->spcg_grid = std::max(1, std::min(pb->num_sms, C));
      pb->spcg_smem = pb->fp64 ? bspcg_smem_bytes<double>(C, pb->spcg_grid) : bspcg_smem_bytes<float>(C, pb->spcg_grid);
    }
    const bool rs = pb->spcg_rows_in_smem != 0;
    const void* sfn = pb->sparse ? (pb->fp64 ? bspcg_kernel_ptr<double>() : bspcg_kernel_ptr<float>())
                                 : (pb->fp64 ? spcg_kernel_ptr<double>(rs) : spcg_kernel_ptr<float>(rs));
    CU(cudaFuncSetAttribute(sfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pb->spcg_smem));
    int sper = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sper, sfn, spcg_threads(), pb->spcg_smem));
    if (sper < 1 || pb->spcg_grid > sper * pb->num_sms) {
      set_error("explicit PCG kernel cannot be resident");
      return BA_ERR_INVALID_ARG;
    }
  }
  pb->bs_grid = std::max(1, std::min(pb->num_sms * 8, (P + 255) / 256));
  ST(dalloc(pb, &pb->pred_parts, (size_t)std::max(pb->pcg_grid, pb->bs_grid) + 1));
  // double-float evaluation (FP32 problems): fewer, longer-lived threads amortise each thread's FP64 tail
  pb->eval_grid = std::max(1, std::min(pb->num_sms * (pb->fp64 ? 8 : 4), (N + kBlock - 1) / kBlock));
  ST(dalloc(pb, &pb->eval_parts, (size_t)3 * pb->eval_grid));
  ST(dalloc(pb, &pb->sc, 1));
  CU(cudaMemset(pb->sc, 0, sizeof(Scalars)));
  CU(cudaMallocHost(&pb->h_sc, sizeof(Scalars)));
  memset(pb->h_sc, 0, sizeof(Scalars));
  for (auto& e : pb->ev) CU(cudaEventCreate(&e));
  {
    int lo = 0, hi = 0;
    CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CU(cudaStreamCreateWithPriority(&pb->side, cudaStreamNonBlocking, hi));
    CU(cudaEventCreateWithFlags(&pb->fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&pb->join, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&pb->cand_fork, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&pb->cand_join, cudaEventDisableTiming));
  }
  for (auto& e : pb->evk) CU(cudaEventCreate(&e));
  for (auto& e : pb->evf) CU(cudaEventCreate(&e));

  // working copies of the initial state (after every upload has landed)
  CU(cudaDeviceSynchronize());
  if (pb->fp64) {
    LAUNCH(1, launch_prep_cams<double>(pb->cams64[0], (double*)pb->camw[0], nullptr, C, pb->stream, pb->mp.cam_model));
    LAUNCH(1, launch_prep_pts<double>(pb->pts64[0], (double*)pb->ptsw[0], P, pb->stream));
  } else {
    LAUNCH(1, launch_prep_cams<float>(pb->cams64[0], (float*)pb->camw[0], pb->camw64[0], C, pb->stream, pb->mp.cam_model));
    LAUNCH(1, launch_prep_pts<float>(pb->pts64[0], (float*)pb->ptsw[0], P, pb->stream));
  }
  ST(sync(pb));
  return BA_OK;
}

void free_problem(ba_problem* pb) {
  if (!pb) return;
  if (pb->stream) cudaStreamSynchronize(pb->stream);
  if (pb->side) {
    cudaStreamSynchronize(pb->side);
    cudaStreamDestroy(pb->side);
  }
  for (auto& row : pb->ext_graph)
    for (cudaGraphExec_t& g : row)
      if (g) cudaGraphExecDestroy(g);
  if (pb->cap) cudaStreamDestroy(pb->cap);
  if (pb->fork) cudaEventDestroy(pb->fork);
  if (pb->join) cudaEventDestroy(pb->join);
  if (pb->cand_fork) cudaEventDestroy(pb->cand_fork);
  if (pb->cand_join) cudaEventDestroy(pb->cand_join);
  for (void* p : pb->allocs) cached_free(p);
  if (pb->h_sc) cudaFreeHost(pb->h_sc);
  for (auto& e : pb->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : pb->evk)
    if (e) cudaEventDestroy(e);
  for (auto& e : pb->evf)
    if (e) cudaEventDestroy(e);
  delete pb;
}

template <typename T>
ba_status copy_out_linearization(ba_problem* pb, double* U, double* V, double* W, double* gc,
                                 double* gp) {
  const int C = pb->C, P = pb->P, N = pb->N;
  // camera blocks and point blocks are small: bring them to the host and unpack
  if (U || gc) {
    std::vector<T> ug((size_t)C * 54);
    if (C) CU(cudaMemcpy(ug.data(), pb->Ug, sizeof(T) * ug.size(), cudaMemcpyDeviceToHost));
    std::vector<double> hU((size_t)C * 81, 0.0), hg((size_t)C * 9, 0.0);
    for (int c = 0; c < C; ++c)
      for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) hU[81 * (size_t)c + 9 * i + j] = ug[54 * (size_t)c + sym9(i, j)];
        hg[9 * (size_t)c + i] = ug[54 * (size_t)c + 45 + i];
      }
    if (U && C) CU(cudaMemcpy(U, hU.data(), sizeof(double) * hU.size(), cudaMemcpyDefault));
    if (gc && C) CU(cudaMemcpy(gc, hg.data(), sizeof(double) * hg.size(), cudaMemcpyDefault));
  }
  if (V || gp) {
    std::vector<T> hv((size_t)P * 6), hgp((size_t)P * 3);
    if (P) {
      CU(cudaMemcpy(hv.data(), pb->V, sizeof(T) * hv.size(), cudaMemcpyDeviceToHost));
      CU(cudaMemcpy(hgp.data(), pb->gp, sizeof(T) * hgp.size(), cudaMemcpyDeviceToHost));
    }
    std::vector<double> oV((size_t)P * 9), og((size_t)P * 3);
    for (int p = 0; p < P; ++p) {
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) oV[9 * (size_t)p + 3 * i + j] = hv[6 * (size_t)p + sym3(i, j)];
        og[3 * (size_t)p + i] = hgp[3 * (size_t)p + i];
      }
    }
    if (V && P) CU(cudaMemcpy(V, oV.data(), sizeof(double) * oV.size(), cudaMemcpyDefault));
    if (gp && P) CU(cudaMemcpy(gp, og.data(), sizeof(double) * og.size(), cudaMemcpyDefault));
  }
  if (W && N) {
    // in recompute mode the W blocks are never stored: form them into a scratch
    // buffer with the same linearization kernel (inspection only)
    T* wsrc = pb->orec ? nullptr : (T*)pb->W;  // W rows are not stored when records are
    T* wtmp = nullptr;
    T* scratch_v = nullptr;
    cudaError_t e = cudaSuccess;
    if (!wsrc) {
      e = cudaMalloc(&wtmp, sizeof(T) * kWStride * ((size_t)N + 1));
      if (e == cudaSuccess) e = cudaMalloc(&scratch_v, sizeof(T) * 9 * ((size_t)P + 1));
      if (e == cudaSuccess) {
        pb->launches += 1;
        e = launch_pt_lin<T>(pb->L, pb->mp, (const T*)pb->camw[pb->cur], (const T*)pb->ptsw[pb->cur],
                             pb->obs_act, wtmp, nullptr, scratch_v, scratch_v + 6 * (size_t)P, pb->stream);
      }
      wsrc = wtmp;
    }
    double* tmp = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(double) * 27 * (size_t)N);
    if (e == cudaSuccess) {
      pb->launches += 1;
      e = launch_permute_rows<T>(pb->po_orig, pb->po_wrow, wsrc, kWStride, tmp, N, 27, pb->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->stream);
    if (e == cudaSuccess) e = cudaMemcpy(W, tmp, sizeof(double) * 27 * (size_t)N, cudaMemcpyDefault);
    cudaFree(tmp);
    cudaFree(wtmp);
    cudaFree(scratch_v);
    CU(e);
  }
  return BA_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

void ba_default_options(ba_options* o) {
  static const int32_t kGauge[1] = {0};
  memset(o, 0, sizeof *o);
  o->precision = BA_FP32;
  o->img_w = 640;
  o->img_h = 480;
  o->cx = 320.0;
  o->cy = 240.0;
  o->huber_delta = 1.0;
  o->depth_weight = 1.0;
  o->invalid_depth_weight = 0.0;
  o->min_depth = 0.1;
  o->extract_every = 0;
  o->drop_residual_px = 0.0;
  o->min_cam_obs = 1;
  o->min_pt_obs = 1;
  o->lambda0 = 1e-4;
  o->pcg_rel_tol = 1e-6;
  o->pcg_max_iters = 500;
  o->fixed_cams = kGauge;
  o->n_fixed = 1;
  o->solver = BA_SOLVER_AUTO;
  o->extract_mode = BA_EXTRACT_DYNAMIC;
}

ba_status ba_create(const ba_options* opts, void* stream, int64_t n_cams, const double* cams,
                    int64_t n_pts, const double* pts, int64_t n_obs, const int32_t* obs_cam,
                    const int32_t* obs_pt, const double* obs_uv, const double* depth,
                    ba_problem** out) {
  if (!out) {
    set_error("null output handle");
    return BA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  ba_problem* pb = new ba_problem();
  ba_status s = create_impl(opts, stream, n_cams, cams, n_pts, pts, n_obs, obs_cam, obs_pt, obs_uv,
                            depth, pb);
  if (s != BA_OK) {
    free_problem(pb);
    return s;
  }
  *out = pb;
  return BA_OK;
}

ba_status ba_lm_step(ba_problem* pb, ba_iter_info* info) {
  if (!pb) return BA_ERR_INVALID_ARG;
  return lm_step(pb, info);
}

ba_status ba_solve(ba_problem* pb, int max_iters, ba_iter_info* log, int* n_done) {
  if (!pb || max_iters < 0) return BA_ERR_INVALID_ARG;
  ba_status worst = BA_OK;
  int i = 0;
  for (; i < max_iters; ++i) {
    ba_status s = lm_step(pb, log ? log + i : nullptr);
    if (s == BA_ERR_NOT_CONVERGED || s == BA_ERR_NONFINITE) {
      worst = s;
      continue;
    }
    if (s != BA_OK) {
      if (n_done) *n_done = i;
      return s;
    }
  }
  if (n_done) *n_done = i;
  return worst == BA_ERR_NONFINITE ? BA_OK : worst;
}

ba_status ba_get_params(ba_problem* pb, double* cams, double* pts) {
  if (!pb) return BA_ERR_INVALID_ARG;
  ST(sync(pb));
  if (cams && pb->C) CU(cudaMemcpy(cams, pb->cams64[pb->cur], sizeof(double) * 9 * (size_t)pb->C, cudaMemcpyDefault));
  if (pts && pb->P) CU(cudaMemcpy(pts, pb->pts64[pb->cur], sizeof(double) * 3 * (size_t)pb->P, cudaMemcpyDefault));
  return BA_OK;
}

ba_status ba_set_params(ba_problem* pb, const double* cams, const double* pts) {
  if (!pb || (!cams && pb->C) || (!pts && pb->P)) return BA_ERR_INVALID_ARG;
  ST(sync(pb));
  std::vector<double> hc((size_t)pb->C * 9), hp((size_t)pb->P * 3);
  if (pb->C) CU(cudaMemcpy(hc.data(), cams, sizeof(double) * hc.size(), cudaMemcpyDefault));
  if (pb->P) CU(cudaMemcpy(hp.data(), pts, sizeof(double) * hp.size(), cudaMemcpyDefault));
  for (double v : hc)
    if (!std::isfinite(v)) return BA_ERR_INVALID_ARG;
  for (double v : hp)
    if (!std::isfinite(v)) return BA_ERR_INVALID_ARG;
  int s = pb->cur;
  if (pb->C) CU(cudaMemcpy(pb->cams64[s], hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice));
  if (pb->P) CU(cudaMemcpy(pb->pts64[s], hp.data(), sizeof(double) * hp.size(), cudaMemcpyHostToDevice));
  if (pb->fp64) {
    LAUNCH(1, launch_prep_cams<double>(pb->cams64[s], (double*)pb->camw[s], nullptr, pb->C, pb->stream, pb->mp.cam_model));
    LAUNCH(1, launch_prep_pts<double>(pb->pts64[s], (double*)pb->ptsw[s], pb->P, pb->stream));
  } else {
    LAUNCH(1, launch_prep_cams<float>(pb->cams64[s], (float*)pb->camw[s], pb->camw64[s], pb->C, pb->stream, pb->mp.cam_model));
    LAUNCH(1, launch_prep_pts<float>(pb->pts64[s], (float*)pb->ptsw[s], pb->P, pb->stream));
  }
  pb->bits_valid[s] = pb->cost_valid[s] = false;
  pb->df_current[s] = false;
  pb->state_changed = true;
  pb->same_validity = false;
  pb->linearized = false;
  ST(sync(pb));
  return BA_OK;
}

namespace {
struct StateHeader {
  uint64_t magic;  // "BAB300ST"
  uint32_t version, precision;
  int64_t C, P, N;
  uint64_t obs_hash;
  int64_t iter;
  double lambda, nu;
};
constexpr uint64_t kStateMagic = 0x5453303033424142ull;
size_t state_bytes(const ba_problem* pb) {
  return sizeof(StateHeader) + sizeof(double) * (9 * (size_t)pb->C + 3 * (size_t)pb->P) + (size_t)pb->N;
}
}  // namespace

ba_status ba_get_state(ba_problem* pb, void* blob, size_t* bytes) {
  if (!pb || !bytes) return BA_ERR_INVALID_ARG;
  const size_t need = state_bytes(pb);
  if (!blob) {
    *bytes = need;
    return BA_OK;
  }
  if (*bytes < need) {
    set_error("ba_get_state: blob of %zu bytes, %zu needed", *bytes, need);
    *bytes = need;
    return BA_ERR_INVALID_ARG;
  }
  ST(sync(pb));
  unsigned char* out = static_cast<unsigned char*>(blob);
  StateHeader h{kStateMagic, 1u, (uint32_t)(pb->fp64 ? BA_FP64 : BA_FP32), pb->C, pb->P, pb->N, pb->obs_hash,
                pb->iter, pb->lambda, pb->nu};
  memcpy(out, &h, sizeof h);
  out += sizeof h;
  const int s = pb->cur;
  if (pb->C) CU(cudaMemcpy(out, pb->cams64[s], sizeof(double) * 9 * (size_t)pb->C, cudaMemcpyDefault));
  out += sizeof(double) * 9 * (size_t)pb->C;
  if (pb->P) CU(cudaMemcpy(out, pb->pts64[s], sizeof(double) * 3 * (size_t)pb->P, cudaMemcpyDefault));
  out += sizeof(double) * 3 * (size_t)pb->P;
  if (pb->N) CU(cudaMemcpy(out, pb->alive, (size_t)pb->N, cudaMemcpyDefault));
  *bytes = need;
  return BA_OK;
}

ba_status ba_set_state(ba_problem* pb, const void* blob, size_t bytes) {
  if (!pb || !blob) return BA_ERR_INVALID_ARG;
  StateHeader h;
  if (bytes < sizeof h) {
    set_error("ba_set_state: blob too short");
    return BA_ERR_INVALID_ARG;
  }
  memcpy(&h, blob, sizeof h);
  if (h.magic != kStateMagic || h.version != 1u) {
    set_error("ba_set_state: not a state blob of this library");
    return BA_ERR_INVALID_ARG;
  }
  if (h.C != pb->C || h.P != pb->P || h.N != pb->N || h.obs_hash != pb->obs_hash ||
      h.precision != (uint32_t)(pb->fp64 ? BA_FP64 : BA_FP32) || bytes < state_bytes(pb)) {
    set_error("ba_set_state: the blob belongs to a different problem (sizes, observations or precision)");
    return BA_ERR_INVALID_ARG;
  }
  if (!(h.lambda > 0.0) || !std::isfinite(h.lambda) || !(h.nu >= 1.0) || !std::isfinite(h.nu) || h.iter < 0) {
    set_error("ba_set_state: invalid damping state");
    return BA_ERR_INVALID_ARG;
  }
  const unsigned char* in = static_cast<const unsigned char*>(blob) + sizeof h;
  const double* cams = reinterpret_cast<const double*>(in);
  const double* pts = cams + 9 * (size_t)pb->C;
  const unsigned char* alive = reinterpret_cast<const unsigned char*>(pts + 3 * (size_t)pb->P);
  ST(ba_set_params(pb, cams, pts));
  if (pb->N) CU(cudaMemcpy(pb->alive, alive, (size_t)pb->N, cudaMemcpyDefault));
  pb->iter = (int)h.iter;
  pb->lambda = h.lambda;
  pb->nu = h.nu;
  pb->extracted = false;
  return BA_OK;
}

ba_status ba_get_active(ba_problem* pb, uint8_t* cam_mask, uint8_t* pt_mask, uint8_t* obs_mask,
                        int32_t* cam_rank, int32_t* pt_rank) {
  if (!pb) return BA_ERR_INVALID_ARG;
  if (!pb->extracted) {
    set_error("no extraction has run yet");
    return BA_ERR_STATE;
  }
  ST(sync(pb));
  if (cam_mask && pb->C) CU(cudaMemcpy(cam_mask, pb->cam_act, (size_t)pb->C, cudaMemcpyDefault));
  if (pt_mask && pb->P) CU(cudaMemcpy(pt_mask, pb->pt_act, (size_t)pb->P, cudaMemcpyDefault));
  if (cam_rank && pb->C) CU(cudaMemcpy(cam_rank, pb->crank, sizeof(int) * (size_t)pb->C, cudaMemcpyDefault));
  if (pt_rank && pb->P) CU(cudaMemcpy(pt_rank, pb->pt_rank, sizeof(int) * (size_t)pb->P, cudaMemcpyDefault));
  if (obs_mask && pb->N) {
    uint8_t* tmp = nullptr;
    CU(cudaMalloc(&tmp, (size_t)pb->N));
    pb->launches += 1;
    cudaError_t e = launch_permute_u8(pb->po_orig, pb->obs_act, tmp, pb->N, pb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->stream);
    if (e == cudaSuccess) e = cudaMemcpy(obs_mask, tmp, (size_t)pb->N, cudaMemcpyDefault);
    cudaFree(tmp);
    CU(e);
  }
  return BA_OK;
}

ba_status ba_selftest_layout(int64_t n_cams, const double* cams, int64_t n_pts, const double* pts, int64_t n_obs,
                             const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv, int with_covis,
                             int* mismatch) {
  if (!mismatch || n_cams < 0 || n_pts < 0 || n_obs < 0 || n_cams >= (1LL << 24) || n_pts >= (1LL << 30) ||
      n_obs >= (1LL << 30) || (n_cams && !cams) || (n_pts && !pts) ||
      (n_obs && (!obs_cam || !obs_pt || !obs_uv))) {
    set_error("ba_selftest_layout: invalid arguments");
    return BA_ERR_INVALID_ARG;
  }
  *mismatch = 0;
  const int C = (int)n_cams, P = (int)n_pts, N = (int)n_obs;
  // reference: the host builder
  ObsLayout H;
  CovisRuns hc;
  std::string herr, derr;
  int hrc = build_obs_layout(C, P, N, cams, pts, obs_uv, obs_cam, obs_pt, &H, &herr);
  if (!hrc && with_covis) hrc = build_covis_runs(H, C, N, &hc, &herr);
  // device builder on uploaded copies; its arrays are freed here
  std::vector<void*> owned;
  struct Free {
    std::vector<void*>& v;
    ~Free() {
      cudaDeviceSynchronize();
      for (void* q : v) cudaFree(q);
    }
  } free_all{owned};
  auto alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    owned.push_back(q);
    return q;
  };
  auto up = [&](const void* src, size_t bytes) -> void* {
    void* q = alloc(bytes);
    if (q && bytes) cudaMemcpy(q, src, bytes, cudaMemcpyHostToDevice);
    return q;
  };
  const double* d_cams = (const double*)up(cams, sizeof(double) * 9 * (size_t)C);
  const double* d_pts = (const double*)up(pts, sizeof(double) * 3 * (size_t)P);
  const double* d_uv = (const double*)up(obs_uv, sizeof(double) * 2 * (size_t)N);
  const int32_t* d_oc = (const int32_t*)up(obs_cam, sizeof(int32_t) * (size_t)N);
  const int32_t* d_op = (const int32_t*)up(obs_pt, sizeof(int32_t) * (size_t)N);
  if (!d_cams || !d_pts || !d_uv || !d_oc || !d_op) {
    set_error("ba_selftest_layout: device allocation failed");
    return BA_ERR_OOM;
  }
  cudaStream_t st = nullptr;
  DevLayout D;
  DevCovis dc;
  int drc = build_obs_layout_dev(C, P, N, d_cams, d_pts, d_uv, d_oc, d_op, alloc, st, nullptr, &D, &derr);
  if (!drc && with_covis) drc = build_covis_runs_dev(D, C, N, alloc, st, &dc, &derr);
  if (drc >= 2) {
    set_error("ba_selftest_layout: %s", derr.c_str());
    return drc == 3 ? BA_ERR_OOM : BA_ERR_CUDA;
  }
  if (hrc || drc) {  // both must reject the input with the same message
    if (hrc != drc || herr != derr) *mismatch |= 128;
    return BA_OK;
  }
  auto same = [&](const void* dev, const void* host, size_t bytes) {
    if (!bytes) return true;
    std::vector<unsigned char> tmp(bytes);
    if (cudaMemcpy(tmp.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return memcmp(tmp.data(), host, bytes) == 0;
  };
  const size_t n4 = sizeof(int) * (size_t)N;
  if (!same(D.po, H.po.data(), n4) || !same(D.co, H.co.data(), n4) || !same(D.co_po, H.co_po.data(), n4) ||
      !same(D.po_cam, H.po_cam.data(), n4) || !same(D.po_pt, H.po_pt.data(), n4))
    *mismatch |= 1;
  if (!same(D.pt_off, H.pt_off.data(), sizeof(int) * H.pt_off.size()) ||
      !same(D.cam_off, H.cam_off.data(), sizeof(int) * H.cam_off.size()))
    *mismatch |= 2;
  if (D.n_tiles != H.n_tiles || D.g_rows != H.g_rows ||
      !same(D.descs, H.descs.data(), sizeof(TileDesc) * H.descs.size()))
    *mismatch |= 4;
  if (D.meta_bytes != H.meta.size() || !same(D.meta, H.meta.data(), H.meta.size())) *mismatch |= 8;
  if (D.n_chunks != (int)H.chunk_cam.size() ||
      !same(D.chunk_obs, H.chunk_obs.data(), sizeof(int) * H.chunk_obs.size()) ||
      !same(D.chunk_cam, H.chunk_cam.data(), sizeof(int) * H.chunk_cam.size()) ||
      !same(D.cam_chunk, H.cam_chunk.data(), sizeof(int) * H.cam_chunk.size()))
    *mismatch |= 16;
  if (D.obs_hash != H.obs_hash) *mismatch |= 32;
  if (with_covis && (dc.npairs != hc.npairs || dc.n_runs != (int)hc.runs.size() ||
                     !same(dc.runs, hc.runs.data(), sizeof(int4) * hc.runs.size()) ||
                     !same(dc.pairs, hc.pairs.data(), sizeof(int2) * hc.npairs)))
    *mismatch |= 64;
  return BA_OK;
}

ba_status ba_extract(ba_problem* pb, int drop, int* n_rounds) {
  if (!pb) return BA_ERR_INVALID_ARG;
  ST(run_extraction(pb, drop != 0, n_rounds));
  pb->state_changed = false;
  return BA_OK;
}

ba_status ba_linearize(ba_problem* pb, double* U, double* V, double* W, double* gc, double* gp) {
  if (!pb) return BA_ERR_INVALID_ARG;
  ST(ensure_linearized(pb));
  ST(sync(pb));
  if (pb->fp64) return copy_out_linearization<double>(pb, U, V, W, gc, gp);
  return copy_out_linearization<float>(pb, U, V, W, gc, gp);
}

ba_status ba_solve_damped(ba_problem* pb, double lambda, double* dc, double* dp,
                          ba_iter_info* info) {
  if (!pb || !(lambda >= 0.0) || !std::isfinite(lambda)) return BA_ERR_INVALID_ARG;
  ST(ensure_linearized(pb));
  CU(cudaMemsetAsync(pb->err, 0, sizeof(int), pb->stream));
  ST(solve_damped(pb, lambda));
  CU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  int h_err = 0;
  CU(cudaMemcpyAsync(&h_err, pb->err, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
  ST(sync(pb));
  if (dc && pb->C) {
    double* tmp = nullptr;
    CU(cudaMalloc(&tmp, sizeof(double) * 9 * (size_t)pb->C));
    pb->launches += 1;
    cudaError_t e = pb->fp64 ? launch_scatter_cams<double>(pb->C, pb->crank, (const double*)pb->x, tmp, pb->stream)
                             : launch_scatter_cams<float>(pb->C, pb->crank, (const float*)pb->x, tmp, pb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->stream);
    if (e == cudaSuccess) e = cudaMemcpy(dc, tmp, sizeof(double) * 9 * (size_t)pb->C, cudaMemcpyDefault);
    cudaFree(tmp);
    CU(e);
  }
  if (dp && pb->P) {
    double* tmp = nullptr;
    CU(cudaMalloc(&tmp, sizeof(double) * 3 * (size_t)pb->P));
    pb->launches += 1;
    cudaError_t e = pb->fp64 ? launch_to_double<double>((const double*)pb->dp, tmp, 3LL * pb->P, pb->stream)
                             : launch_to_double<float>((const float*)pb->dp, tmp, 3LL * pb->P, pb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->stream);
    if (e == cudaSuccess) e = cudaMemcpy(dp, tmp, sizeof(double) * 3 * (size_t)pb->P, cudaMemcpyDefault);
    cudaFree(tmp);
    CU(e);
  }
  if (info) {
    memset(info, 0, sizeof *info);
    info->lambda = lambda;
    info->pcg_iters = pb->h_sc->pcg_iters;
    info->pcg_rel_res = pb->h_sc->pcg_rel_res;
    info->pred_decrease = pb->h_sc->pred;
    info->n_cam_act = pb->n_cam_act;
    info->n_pt_act = pb->n_pt_act;
    info->n_obs_act = pb->n_obs_act;
  }
  if (h_err & 1) {
    set_error("PCG grid barrier timed out");
    return BA_ERR_TIMEOUT;
  }
  return BA_OK;
}

ba_status ba_eval_cost(ba_problem* pb, const double* cams, const double* pts, double* cost,
                       double* rmse_px) {
  if (!pb) return BA_ERR_INVALID_ARG;
  ST(ensure_extracted(pb));
  int slot = pb->cur;
  if (cams || pts) {
    // evaluate in the spare slot without disturbing the solver state
    slot = 1 - pb->cur;
    if (cams && pb->C) CU(cudaMemcpyAsync(pb->cams64[slot], cams, sizeof(double) * 9 * (size_t)pb->C, cudaMemcpyDefault, pb->stream));
    else if (pb->C) CU(cudaMemcpyAsync(pb->cams64[slot], pb->cams64[pb->cur], sizeof(double) * 9 * (size_t)pb->C, cudaMemcpyDeviceToDevice, pb->stream));
    if (pts && pb->P) CU(cudaMemcpyAsync(pb->pts64[slot], pts, sizeof(double) * 3 * (size_t)pb->P, cudaMemcpyDefault, pb->stream));
    else if (pb->P) CU(cudaMemcpyAsync(pb->pts64[slot], pb->pts64[pb->cur], sizeof(double) * 3 * (size_t)pb->P, cudaMemcpyDeviceToDevice, pb->stream));
    LAUNCH(1, launch_prep_cams<double>(pb->cams64[slot], pb->camw64[slot], nullptr, pb->C, pb->stream, pb->mp.cam_model));
    pb->bits_valid[slot] = false;
    pb->df_current[slot] = false;
  }
  ST(eval_state(pb, slot, false, true));
  if (slot != pb->cur) pb->cost_valid[slot] = false;
  CU(cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream));
  ST(sync(pb));
  if (cost) *cost = pb->h_sc->cost[slot];
  if (rmse_px) *rmse_px = pb->h_sc->n_act[slot] > 0 ? std::sqrt(pb->h_sc->rmse_sum[slot] / pb->h_sc->n_act[slot]) : 0.0;
  return BA_OK;
}

ba_status ba_backward(ba_problem* pb, const double* dL_dcams, const double* dL_dpts,
                      double* dL_duv, double* dL_ddepth) {
  if (!pb || !dL_dcams || !dL_dpts || !dL_duv || !dL_ddepth) {
    set_error("ba_backward: NULL argument");
    return BA_ERR_INVALID_ARG;
  }
  ST(ensure_linearized(pb));
  const size_t C = (size_t)pb->C, P = (size_t)pb->P, N = (size_t)pb->N;
  // device staging: dL/dcams, dL/dpts in; dL/duv, dL/ddepth out
  double* buf = nullptr;
  const size_t nb = 9 * C + 3 * P + 3 * N + 1;
  CU(cudaMallocAsync(&buf, sizeof(double) * nb, pb->stream));
  double *dc = buf, *dpv = buf + 9 * C, *duv = dpv + 3 * P, *dd = duv + 2 * N;
  cudaError_t e = cudaSuccess;
  if (C) e = cudaMemcpyAsync(dc, dL_dcams, sizeof(double) * 9 * C, cudaMemcpyDefault, pb->stream);
  if (e == cudaSuccess && P) e = cudaMemcpyAsync(dpv, dL_dpts, sizeof(double) * 3 * P, cudaMemcpyDefault, pb->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pb->err, 0, sizeof(int), pb->stream);
  ba_status st = BA_OK;
  if (e != cudaSuccess) {
    set_error("ba_backward: %s", cudaGetErrorString(e));
    st = BA_ERR_CUDA;
  } else {
    st = pb->fp64 ? backward_t<double>(pb, dc, dpv, duv, dd) : backward_t<float>(pb, dc, dpv, duv, dd);
  }
  int h_err = 0;
  if (st == BA_OK) {
    e = cudaMemcpyAsync(pb->h_sc, pb->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, pb->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, pb->err, sizeof(int), cudaMemcpyDeviceToHost, pb->stream);
    if (e == cudaSuccess && N) e = cudaMemcpyAsync(dL_duv, duv, sizeof(double) * 2 * N, cudaMemcpyDefault, pb->stream);
    if (e == cudaSuccess && N) e = cudaMemcpyAsync(dL_ddepth, dd, sizeof(double) * N, cudaMemcpyDefault, pb->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pb->stream);
    if (e != cudaSuccess) {
      set_error("ba_backward: %s", cudaGetErrorString(e));
      st = BA_ERR_CUDA;
    }
  }
  cudaFreeAsync(buf, pb->stream);
  if (st != BA_OK) return st;
  if (h_err & 1) {
    set_error("ba_backward: PCG grid barrier timed out");
    return BA_ERR_TIMEOUT;
  }
  if (h_err & 14) {
    set_error("ba_backward: the undamped system is singular (flags %d)", h_err);
    return BA_ERR_NONFINITE;
  }
  if (pb->h_sc->pcg_iters >= pb->opt.pcg_max_iters) {
    set_error("ba_backward: PCG reached its iteration cap (relative residual %g)", pb->h_sc->pcg_rel_res);
    return BA_ERR_NOT_CONVERGED;
  }
  return BA_OK;
}

int64_t ba_kernel_launches(const ba_problem* pb) { return pb ? pb->launches : 0; }

int ba_formation_kernel(const ba_problem* pb) {
  if (!pb || !pb->explicit_S || pb->n_covis_runs == 0) return 0;
  return pb->cform.n_blocks ? 3 : pb->form_lanes ? 2 : pb->orec ? 4 : 1;
}

ba_status ba_debug_bounds(int reset, int64_t* site, int64_t* index) {
  if (site) *site = -1;
  if (index) *index = 0;
#ifdef BA_DEBUG_BOUNDS
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("ba_debug_bounds: %s", cudaGetErrorString(cudaGetLastError()));
    return BA_ERR_CUDA;
  }
  unsigned long long first = 0;
  for (unsigned long long v : {bounds_fault_kernels(reset != 0), bounds_fault_schur(reset != 0),
                               bounds_fault_adjoint(reset != 0)}) {
    if (v == ~0ull) {
      set_error("ba_debug_bounds: reading the records failed");
      cudaGetLastError();
      return BA_ERR_CUDA;
    }
    if (!first) first = v;
  }
  if (site) *site = (int64_t)(first >> 32);
  if (index) *index = (int64_t)(int32_t)(first & 0xffffffffull);
#else
  (void)reset;
#endif
  return BA_OK;
}

int ba_solver_kind(const ba_problem* pb) {
  if (!pb) return 0;
  return pb->dense ? BA_SOLVER_DENSE : pb->sparse ? BA_SOLVER_SPARSE : pb->explicit_S ? BA_SOLVER_EXPLICIT
                                                                                    : BA_SOLVER_IMPLICIT;
}

void ba_explicit_layout(const ba_problem* pb, int* rows_in_smem, int* vecs_in_smem, int* grid) {
  const bool e = pb && pb->explicit_S && !pb->dense;
  if (rows_in_smem) *rows_in_smem = e ? pb->spcg_rows_in_smem : 0;
  if (vecs_in_smem) *vecs_in_smem = e ? pb->spcg_vecs_in_smem : 0;
  if (grid) *grid = e ? pb->spcg_grid : 0;
}

void ba_destroy(ba_problem* pb) { free_problem(pb); }

void ba_release_cache(void) {
  AllocCache& c = alloc_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : c.free_blocks) {
    cudaSetDevice(kv.first.first);
    cudaFree(kv.second);
    c.sizes.erase(kv.second);
  }
  c.free_blocks.clear();
  cudaSetDevice(cur);
  release_scratch_pools();
}

const char* ba_status_string(ba_status s) {
  switch (s) {
    case BA_OK: return "ok";
    case BA_ERR_INVALID_ARG: return "invalid argument";
    case BA_ERR_CUDA: return "CUDA error";
    case BA_ERR_OOM: return "out of device memory";
    case BA_ERR_NOT_CONVERGED: return "PCG did not converge";
    case BA_ERR_NONFINITE: return "non-finite cost or step";
    case BA_ERR_STATE: return "call out of order";
    case BA_ERR_TIMEOUT: return "grid barrier timeout";
  }
  return "unknown status";
}

const char* ba_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
