// layout.cu -- host-side construction of the observation layout (see layout.h).
#include "layout.h"
#include "tile_meta.cuh"

#include <stdlib.h>
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdarg>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

namespace bab {

// ---------------------------------------------------------------------------
// host buffers
// ---------------------------------------------------------------------------

template <typename T>
void HostBuf<T>::resize(size_t n) {
  release();
  if (n == 0) return;
  constexpr size_t kHuge = size_t(2) << 20;
  const size_t bytes = (n * sizeof(T) + kHuge - 1) / kHuge * kHuge;
  void* p = nullptr;
  if (posix_memalign(&p, kHuge, bytes) != 0 || !p) throw std::bad_alloc();
  madvise(p, bytes, MADV_HUGEPAGE);  // advisory: ignored where huge pages are off
  p_ = static_cast<T*>(p);
  n_ = n;
}

template <typename T>
void HostBuf<T>::release() {
  free(p_);
  p_ = nullptr;
  n_ = 0;
}

template class HostBuf<int>;
template class HostBuf<unsigned>;
template class HostBuf<unsigned char>;
template class HostBuf<int2>;
template class HostBuf<uint64_t>;

// ---------------------------------------------------------------------------
// worker pool
// ---------------------------------------------------------------------------

int host_threads() {
  if (const char* env = getenv("BA_HOST_THREADS")) {
    const int v = atoi(env);
    if (v > 0) return std::min(v, 256);
  }
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h ? h : 1u, 32u));
}

namespace {

// Persistent workers: a job is n pieces handed out one at a time to the workers
// and the calling thread.  The job's descriptor lives in run()'s frame; a worker
// takes it under the lock and run() returns only once every piece is done and
// no worker holds it, so no worker ever sees a finished job's descriptor.  Jobs
// are serialised by `use_`.  The pool is never destroyed (its threads park on a
// condition variable until the process exits).
class Pool {
 public:
  explicit Pool(int workers) : pid_(getpid()) {
    for (int i = 0; i < workers; ++i) {
      try {
        std::thread(&Pool::loop, this).detach();
      } catch (...) {
        break;  // fewer workers; the caller runs every piece it can take
      }
    }
  }
  pid_t pid() const { return pid_; }
  void run(int n, const std::function<void(int)>& f) {
    std::lock_guard<std::mutex> use(use_);
    Job job;
    job.f = &f;
    job.n = n;
    job.left = n;
    {
      std::lock_guard<std::mutex> lk(m_);
      cur_ = &job;
      ++gen_;
    }
    cv_.notify_all();
    work(&job);
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [&] { return job.left == 0 && job.active == 0; });
    cur_ = nullptr;
  }

 private:
  struct Job {
    const std::function<void(int)>* f = nullptr;
    int n = 0, left = 0, active = 0;  // left, active: guarded by m_
    std::atomic<int> next{0};
  };
  void work(Job* j) {
    int done = 0;
    for (int t; (t = j->next.fetch_add(1)) < j->n;) {
      (*j->f)(t);
      ++done;
    }
    if (done) {
      std::lock_guard<std::mutex> lk(m_);
      j->left -= done;
      if (j->left == 0 && j->active == 0) done_.notify_all();
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      Job* j;
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen && cur_ != nullptr; });
        seen = gen_;
        j = cur_;
        ++j->active;
      }
      work(j);
      std::lock_guard<std::mutex> lk(m_);
      if (--j->active == 0 && j->left == 0) done_.notify_all();
    }
  }
  std::mutex m_, use_;
  std::condition_variable cv_, done_;
  Job* cur_ = nullptr;
  uint64_t gen_ = 0;
  pid_t pid_;
};

Pool* pool() {
  static std::mutex m;
  static Pool* p = nullptr;
  std::lock_guard<std::mutex> lk(m);
  if (!p || p->pid() != getpid()) {  // a forked child starts its own workers
    const unsigned h = std::thread::hardware_concurrency();
    p = new Pool((int)std::max(1u, std::min(h ? h : 1u, 32u)) - 1);
  }
  return p;
}

}  // namespace

void run_pieces(int n, const std::function<void(int)>& f) {
  if (n <= 0) return;
  if (n == 1) {
    f(0);
    return;
  }
  pool()->run(n, f);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

namespace {

int fail(std::string* err, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (err) *err = buf;
  return 1;
}

bool all_finite(const double* v, int64_t n) {
  std::atomic<bool> ok{true};
  parallel_for(n, 1 << 18, [&](int, int64_t b, int64_t e) {
    bool good = true;
    for (int64_t i = b; i < e; ++i) good &= std::isfinite(v[i]);
    if (!good) ok.store(false, std::memory_order_relaxed);
  });
  return ok.load();
}

void atomic_min(std::atomic<int64_t>& a, int64_t v) {
  int64_t cur = a.load();
  while (v < cur && !a.compare_exchange_weak(cur, v)) {
  }
}

int bits_for(int64_t n) {  // bits to hold values 0 .. n-1
  int b = 0;
  while (b < 62 && (int64_t(1) << b) < n) ++b;
  return b;
}

// One stable counting pass of the indices src (or 0..n-1 when src is null) by
// the digit (key[i] >> shift) & (2^bits - 1), over contiguous pieces with
// per-piece histograms.
void radix_pass(const int* src, int* dst, int64_t n, const int32_t* key, int shift, int bits) {
  const int B = 1 << bits, mask = B - 1;
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / (1 << 15)));
  std::vector<int64_t> hist((size_t)nt * B, 0);
  auto lo = [&](int t) { return n * t / nt; };
  run_pieces(nt, [&](int t) {
    int64_t* h = hist.data() + (size_t)t * B;
    for (int64_t i = lo(t); i < lo(t + 1); ++i) h[(key[src ? src[i] : i] >> shift) & mask]++;
  });
  int64_t run = 0;
  for (int d = 0; d < B; ++d)
    for (int t = 0; t < nt; ++t) {
      const int64_t v = hist[(size_t)t * B + d];
      hist[(size_t)t * B + d] = run;
      run += v;
    }
  run_pieces(nt, [&](int t) {
    int64_t* h = hist.data() + (size_t)t * B;
    for (int64_t i = lo(t); i < lo(t + 1); ++i) {
      const int s = src ? src[i] : (int)i;
      dst[h[(key[s] >> shift) & mask]++] = s;
    }
  });
}

// Stable sort of the indices src (0..n-1 when null) by key[i] in [0, nkeys):
// least-significant-digit passes of at most 11 bits.  The result lands in out;
// tmp is scratch of n entries.
void radix_sort(const int* src, int* out, int* tmp, int64_t n, const int32_t* key, int64_t nkeys) {
  const int kb = std::max(1, bits_for(nkeys));
  const int passes = (kb + 10) / 11, per = (kb + passes - 1) / passes;
  // ping-pong so that the last pass writes out
  int* bufs[2] = {(passes & 1) ? out : tmp, (passes & 1) ? tmp : out};
  const int* cur = src;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * per, bits = std::min(per, kb - shift);
    radix_pass(cur, bufs[p & 1], n, key, shift, bits);
    cur = bufs[p & 1];
  }
}

// Stable LSD radix sort of 64-bit items by their key bits [32, 32 + key_bits)
// (the low word is the payload), passes of at most 13 bits; in and tmp swap
// roles between passes and the sorted items are returned (one of the two).
uint64_t* radix_sort_items(uint64_t* in, uint64_t* tmp, int64_t n, int key_bits) {
  const int kb = std::max(1, key_bits);
  const int passes = (kb + 12) / 13, per = (kb + passes - 1) / passes;
  const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n / (1 << 15)));
  auto lo = [&](int t) { return n * t / nt; };
  for (int p = 0; p < passes; ++p) {
    const int shift = 32 + p * per, bits = std::min(per, kb - p * per);
    const int B = 1 << bits;
    const uint64_t mask = (uint64_t)B - 1;
    std::vector<int64_t> hist((size_t)nt * B, 0);
    run_pieces(nt, [&](int t) {
      int64_t* h = hist.data() + (size_t)t * B;
      for (int64_t i = lo(t); i < lo(t + 1); ++i) h[(in[i] >> shift) & mask]++;
    });
    int64_t run = 0;
    for (int d = 0; d < B; ++d)
      for (int t = 0; t < nt; ++t) {
        const int64_t v = hist[(size_t)t * B + d];
        hist[(size_t)t * B + d] = run;
        run += v;
      }
    run_pieces(nt, [&](int t) {
      int64_t* h = hist.data() + (size_t)t * B;
      for (int64_t i = lo(t); i < lo(t + 1); ++i) tmp[h[(in[i] >> shift) & mask]++] = in[i];
    });
    std::swap(in, tmp);
  }
  return in;
}

}  // namespace

// Warp ranges: consecutive whole points with at most 32 observations together,
// or one point with more.  Tiles: up to one warp range per PCG warp, at most
// kTileObs observations and kTileObs points.  Descriptors without their camera
// runs and metadata offsets.
void group_tiles(const int* pt_off, int P, std::vector<int>* wr_pt_out, std::vector<int>* tile_wr_out,
                 std::vector<TileDesc>* descs, int* g_rows) {
  std::vector<int>& wr_pt = *wr_pt_out;
  wr_pt.assign(1, 0);
  {
    int cur_obs = 0;
    for (int p = 0; p < P; ++p) {
      const int len = pt_off[p + 1] - pt_off[p];
      const bool open = wr_pt.back() < p;  // the current range already holds points
      if (open && (len > 32 || cur_obs + len > 32 || p - wr_pt.back() >= 32)) {
        wr_pt.push_back(p);
        cur_obs = 0;
      }
      cur_obs += len;
      if (len > 32) {  // a long point closes its own range
        wr_pt.push_back(p + 1);
        cur_obs = 0;
      }
    }
    if (wr_pt.back() != P) wr_pt.push_back(P);
  }
  const int n_wr_total = (int)wr_pt.size() - 1;
  std::vector<int>& tile_wr = *tile_wr_out;
  tile_wr.assign(1, 0);
  {
    int t_obs = 0, t_pts = 0, t_wr = 0;
    for (int r = 0; r < n_wr_total; ++r) {
      const int r_obs = pt_off[wr_pt[r + 1]] - pt_off[wr_pt[r]], r_pts = wr_pt[r + 1] - wr_pt[r];
      if (t_wr > 0 && (t_wr + 1 > kPcgWarps || t_obs + r_obs > kTileObs || t_pts + r_pts > kTileObs)) {
        tile_wr.push_back(r);
        t_obs = t_pts = t_wr = 0;
      }
      t_obs += r_obs;
      t_pts += r_pts;
      t_wr += 1;
    }
    if (tile_wr.back() != n_wr_total) tile_wr.push_back(n_wr_total);
  }
  const int n_tiles = (int)tile_wr.size() - 1;
  descs->assign((size_t)n_tiles, TileDesc{});
  int rows = 0;
  for (int t = 0; t < n_tiles; ++t) {
    const int pbeg = wr_pt[tile_wr[t]], pend = wr_pt[tile_wr[t + 1]];
    TileDesc d{};
    d.g_row = rows;
    d.w_row = d.obs_begin = pt_off[pbeg];
    d.n_obs = pt_off[pend] - pt_off[pbeg];
    d.pt_begin = pbeg;
    d.n_pts = pend - pbeg;
    rows += (d.n_obs + 3) & ~3;
    (*descs)[t] = d;
  }
  *g_rows = rows;
}

// ---------------------------------------------------------------------------
// validation and layout
// ---------------------------------------------------------------------------

int build_obs_layout(int C, int P, int N, const double* cams, const double* pts, const double* uv,
                     const int32_t* oc, const int32_t* op, ObsLayout* L, std::string* err, bool wide_keys) {
  if (!all_finite(cams, (int64_t)C * 9)) return fail(err, "non-finite camera parameter");
  if (!all_finite(pts, (int64_t)P * 3)) return fail(err, "non-finite point");
  if (!all_finite(uv, (int64_t)N * 2)) return fail(err, "non-finite observation");
  {
    std::atomic<int64_t> first_bad{INT64_MAX};
    parallel_for(N, 1 << 16, [&](int, int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k)
        if (oc[k] < 0 || oc[k] >= C || op[k] < 0 || op[k] >= P) {
          atomic_min(first_bad, k);
          break;
        }
    });
    if (first_bad.load() != INT64_MAX)
      return fail(err, "observation %lld has an index out of range", (long long)first_bad.load());
  }
  {
    // FNV-1a (over 32-bit words) of the sizes and of 256-observation chunk
    // digests, each over its (camera, point) pairs: identifies the observation
    // structure
    constexpr int64_t kHashChunk = 1 << 8;
    auto fnv = [](uint64_t h, int32_t v) { return (h ^ (uint64_t)(uint32_t)v) * 1099511628211ull; };
    const int64_t nch = ((int64_t)N + kHashChunk - 1) / kHashChunk;
    std::vector<uint64_t> dig((size_t)nch);
    parallel_for(nch, 1, [&](int, int64_t b, int64_t e) {
      for (int64_t c = b; c < e; ++c) {
        uint64_t h = 1469598103934665603ull;
        for (int64_t k = c * kHashChunk; k < std::min<int64_t>(N, (c + 1) * kHashChunk); ++k)
          h = fnv(fnv(h, oc[k]), op[k]);
        dig[c] = h;
      }
    });
    uint64_t h = fnv(fnv(1469598103934665603ull, C), P);
    for (uint64_t d : dig) h = fnv(fnv(h, (int32_t)(uint32_t)d), (int32_t)(uint32_t)(d >> 32));
    L->obs_hash = h;
  }
  // ---- point order (by point, then camera, then input index) and camera order
  // (by camera, then point, then input index): stable radix sorts of 64-bit items
  // whose high word is the packed key (point << cb | camera, then camera) and
  // whose low word is the input index; offsets and the duplicate check then read
  // the sorted keys sequentially.
  L->po.resize(N);
  L->co.resize(N);
  L->po_cam.resize(N);
  L->po_pt.resize(N);
  L->co_po.resize(N);
  L->pt_off.assign((size_t)P + 1, 0);
  L->cam_off.assign((size_t)C + 1, 0);
  const int cb = std::max(1, bits_for(C)), pbits = std::max(1, bits_for(P));
  if (N > 0 && (wide_keys || cb + pbits > 32)) {
    // keys too wide to pack: sort the indices with gathered keys instead
    HostBuf<int> a(N), b(N);
    radix_sort(nullptr, a.data(), b.data(), N, oc, C);            // by camera (stable in input index)
    radix_sort(a.data(), L->po.data(), b.data(), N, op, P);        // then stably by point
    radix_sort(L->po.data(), L->co.data(), b.data(), N, oc, C);    // camera order: stably by camera
    std::atomic<int64_t> first_dup{INT64_MAX};
    parallel_for(N, 1 << 16, [&](int, int64_t b0, int64_t e) {
      for (int64_t i = b0; i < e; ++i) {
        const int k = L->po[i], pt = op[k], ppt = i ? op[L->po[i - 1]] : -1;
        for (int q = ppt + 1; q <= pt; ++q) L->pt_off[q] = (int)i;
        if (i && pt == ppt && oc[k] == oc[L->po[i - 1]]) atomic_min(first_dup, i);
        const int cam = oc[L->co[i]], pcam = i ? oc[L->co[i - 1]] : -1;
        for (int q = pcam + 1; q <= cam; ++q) L->cam_off[q] = (int)i;
      }
    });
    for (int q = op[L->po[N - 1]] + 1; q <= P; ++q) L->pt_off[q] = N;
    for (int q = oc[L->co[N - 1]] + 1; q <= C; ++q) L->cam_off[q] = N;
    HostBuf<int> pos(N);
    parallel_for(N, 1 << 16, [&](int, int64_t b0, int64_t e) {
      for (int64_t i = b0; i < e; ++i) {
        const int k = L->po[i];
        L->po_cam[i] = oc[k];
        L->po_pt[i] = op[k];
        pos[k] = (int)i;
      }
    });
    parallel_for(N, 1 << 16, [&](int, int64_t b0, int64_t e) {
      for (int64_t i = b0; i < e; ++i) L->co_po[i] = pos[L->co[i]];
    });
    if (first_dup.load() != INT64_MAX) {
      const int i = (int)first_dup.load();
      return fail(err, "duplicate observation of point %d in camera %d", op[L->po[i]], oc[L->po[i]]);
    }
  } else if (N > 0) {
    HostBuf<uint64_t> A(N), B(N);
    parallel_for(N, 1 << 16, [&](int, int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k)
        A[k] = (uint64_t)(((uint32_t)op[k] << cb) | (uint32_t)oc[k]) << 32 | (uint64_t)k;
    });
    const uint64_t* S = radix_sort_items(A.data(), B.data(), N, cb + pbits);
    const uint32_t cmask = (1u << cb) - 1;
    std::atomic<int64_t> first_dup{INT64_MAX};
    uint64_t* T = S == A.data() ? B.data() : A.data();  // the other buffer: camera-order items
    parallel_for(N, 1 << 16, [&](int, int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        const uint32_t key = (uint32_t)(S[i] >> 32), pkey = i ? (uint32_t)(S[i - 1] >> 32) : 0;
        const int pt = (int)(key >> cb), ppt = i ? (int)(pkey >> cb) : -1;
        L->po[i] = (int)(uint32_t)S[i];
        L->po_cam[i] = (int)(key & cmask);
        L->po_pt[i] = pt;
        T[i] = (uint64_t)(key & cmask) << 32 | (uint64_t)i;  // payload: point-order position
        for (int q = ppt + 1; q <= pt; ++q) L->pt_off[q] = (int)i;  // points ppt+1 .. pt start here
        if (i && key == pkey) atomic_min(first_dup, i);
      }
    });
    for (int q = (int)(S[N - 1] >> 32 >> cb) + 1; q <= P; ++q) L->pt_off[q] = N;
    if (first_dup.load() != INT64_MAX) {
      const int i = (int)first_dup.load();
      return fail(err, "duplicate observation of point %d in camera %d", op[L->po[i]], oc[L->po[i]]);
    }
    const uint64_t* U = radix_sort_items(T, (T == A.data() ? B.data() : A.data()), N, cb);
    parallel_for(N, 1 << 16, [&](int, int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        const int cam = (int)(U[i] >> 32), pcam = i ? (int)(U[i - 1] >> 32) : -1;
        L->co_po[i] = (int)(uint32_t)U[i];
        L->co[i] = L->po[L->co_po[i]];
        for (int q = pcam + 1; q <= cam; ++q) L->cam_off[q] = (int)i;
      }
    });
    for (int q = (int)(U[N - 1] >> 32) + 1; q <= C; ++q) L->cam_off[q] = N;
  }
  const std::vector<int>& pt_off = L->pt_off;
  for (int p = 0; p < P; ++p)
    if (pt_off[p + 1] - pt_off[p] > kTileObs)
      return fail(err, "point %d has %d observations (limit %d)", p, pt_off[p + 1] - pt_off[p], kTileObs);
  group_tiles(pt_off.data(), P, &L->wr_pt, &L->tile_wr, &L->descs, &L->g_rows);
  const int n_tiles = (int)L->descs.size();
  L->n_tiles = n_tiles;
  std::vector<TileDesc>& descs = L->descs;
  const std::vector<int>& wr_pt = L->wr_pt;
  const std::vector<int>& tile_wr = L->tile_wr;
  // Each tile's observations in (camera, local index) order are the camera-order
  // observations whose point-order position falls in the tile, in camera order:
  // a stable counting pass of camera order by tile (per-piece tile histograms)
  // writes them, as camera << 8 | local index, into the tile's own range.
  HostBuf<uint32_t> skey(std::max(N, 1));
  {
    HostBuf<int> po_tile(std::max(N, 1));
    parallel_for(n_tiles, 64, [&](int, int64_t b, int64_t e) {
      for (int64_t t = b; t < e; ++t)
        for (int i = 0; i < descs[t].n_obs; ++i) po_tile[descs[t].obs_begin + i] = (int)t;
    });
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), (int64_t)N / (1 << 15)));
    auto lo = [&](int t) { return (int64_t)N * t / nt; };
    std::vector<int> hist((size_t)nt * n_tiles, 0);
    run_pieces(nt, [&](int t) {
      int* h = hist.data() + (size_t)t * n_tiles;
      for (int64_t q = lo(t); q < lo(t + 1); ++q) h[po_tile[L->co_po[q]]]++;
    });
    parallel_for(n_tiles, 256, [&](int, int64_t b, int64_t e) {
      for (int64_t tile = b; tile < e; ++tile) {
        int run = descs[tile].obs_begin;
        for (int t = 0; t < nt; ++t) {
          const int v = hist[(size_t)t * n_tiles + tile];
          hist[(size_t)t * n_tiles + tile] = run;
          run += v;
        }
      }
    });
    run_pieces(nt, [&](int t) {
      int* h = hist.data() + (size_t)t * n_tiles;
      const int64_t q0 = lo(t), q1 = lo(t + 1);
      int cam = (int)(std::upper_bound(L->cam_off.begin(), L->cam_off.end(), (int)q0) - L->cam_off.begin()) - 1;
      for (int64_t q = q0; q < q1; ++q) {
        while (L->cam_off[cam + 1] <= q) ++cam;
        const int k = L->co_po[q], tile = po_tile[k];
        skey[h[tile]++] = (uint32_t)cam << 8 | (uint32_t)(k - descs[tile].obs_begin);
      }
    });
  }
  parallel_for(n_tiles, 16, [&](int, int64_t b, int64_t e) {
    for (int64_t t = b; t < e; ++t) {
      TileDesc& d = descs[t];
      const uint32_t* key = skey.data() + d.obs_begin;
      int runs = 0;
      for (int j = 0; j < d.n_obs; ++j) runs += (j == 0 || (key[j] >> 8) != (key[j - 1] >> 8));
      d.n_runs = runs;
    }
  });
  size_t meta_total = 0;
  for (int t = 0; t < n_tiles; ++t) {
    descs[t].meta_off = (int)std::min<size_t>(meta_total, (size_t)INT_MAX);
    meta_total += (size_t)tile_meta_bytes(descs[t].n_obs, descs[t].n_pts, descs[t].n_runs);
  }
  if (meta_total >= (size_t)INT_MAX) return fail(err, "tile metadata too large");
  L->meta.resize(meta_total);
  parallel_for(n_tiles, 16, [&](int, int64_t b, int64_t e) {
    std::vector<int> cams_t, poff, wr;
    std::vector<unsigned> runs;
    std::vector<uint8_t> cperm, lid;
    for (int64_t t = b; t < e; ++t) {
      const TileDesc& d = descs[t];
      const int r0 = tile_wr[t], r1 = tile_wr[t + 1], ob = d.obs_begin, nobs = d.n_obs, npts = d.n_pts;
      cams_t.resize(nobs);
      poff.resize(npts + 1);
      wr.resize(r1 - r0 + 1);
      cperm.resize(nobs);
      lid.resize(nobs);
      runs.clear();
      for (int i = 0; i < nobs; ++i) cams_t[i] = L->po_cam[ob + i];
      for (int j = 0; j <= npts; ++j) poff[j] = pt_off[d.pt_begin + j] - ob;
      for (int j = 0; j < npts; ++j)
        for (int i = poff[j]; i < poff[j + 1]; ++i) lid[i] = (uint8_t)j;
      for (int r = r0; r <= r1; ++r) wr[r - r0] = pt_off[wr_pt[r]] - ob;
      const uint32_t* key = skey.data() + ob;
      for (int j = 0; j < nobs; ++j) {
        cperm[j] = (uint8_t)(key[j] & 0xFFu);
        if (j == 0 || (key[j] >> 8) != (key[j - 1] >> 8)) runs.push_back((key[j] >> 8) << 8 | (unsigned)j);
      }
      build_tile_meta(nobs, npts, d.n_runs, r1 - r0, cams_t.data(), poff.data(), runs.data(), wr.data(),
                      cperm.data(), lid.data(), L->meta.data() + d.meta_off);
    }
  });
  // chunks: pieces of one camera's observations
  L->chunk_obs.assign(1, 0);
  L->chunk_cam.clear();
  L->cam_chunk.assign((size_t)C + 1, 0);
  for (int c = 0; c < C; ++c) {
    for (int b = L->cam_off[c]; b < L->cam_off[c + 1]; b += kChunkObs) {
      L->chunk_cam.push_back(c);
      L->chunk_obs.push_back(std::min(b + kChunkObs, L->cam_off[c + 1]));
    }
    L->cam_chunk[c + 1] = (int)L->chunk_cam.size();
  }
  return 0;
}

// ---------------------------------------------------------------------------
// co-visibility runs
// ---------------------------------------------------------------------------

// Row i (first camera i) is built by one task from camera i's observations in
// camera order, which visits the points in ascending order; the partner
// observations of a point follow it in point order (cameras ascending).
int build_covis_runs(const ObsLayout& L, int C, int N, CovisRuns* out, std::string* err) {
  const int* po_cam = L.po_cam.data();
  const int* po_pt = L.po_pt.data();
  const int* co_po = L.co_po.data();
  const int* pt_off = L.pt_off.data();
  auto row_pairs = [&](int i, auto&& emit) {
    for (int q = L.cam_off[i]; q < L.cam_off[i + 1]; ++q) {
      const int k = co_po[q], pend = pt_off[po_pt[k] + 1];
      for (int k2 = k + 1; k2 < pend; ++k2) emit(k, k2, po_cam[k2]);
    }
  };
  std::vector<long long> cnt((size_t)C * C + 1, 0);
  run_pieces(C, [&](int i) {
    long long* row = cnt.data() + 1 + (size_t)i * C;
    row_pairs(i, [&](int, int, int j) { row[j]++; });
  });
  for (size_t q = 0; q < (size_t)C * C; ++q) cnt[q + 1] += cnt[q];
  const size_t npairs = (size_t)cnt[(size_t)C * C];
  if (npairs >= (1ull << 31))
    return fail(err, "too many co-visible observation pairs (%zu) for the explicit system", npairs);
  out->npairs = npairs;
  out->pairs.resize(std::max<size_t>(npairs, 1));
  int2* hp = out->pairs.data();
  run_pieces(C, [&](int i) {
    std::vector<long long> fill(cnt.begin() + (size_t)i * C, cnt.begin() + (size_t)(i + 1) * C);
    row_pairs(i, [&](int k, int k2, int j) { hp[fill[j]++] = make_int2(k, k2); });
  });
  out->runs.clear();
  for (int i = 0; i < C; ++i)
    for (int j = i + 1; j < C; ++j) {
      const size_t q = (size_t)i * C + j;
      if (cnt[q + 1] > cnt[q]) out->runs.push_back(make_int4(i, j, (int)cnt[q], (int)(cnt[q + 1] - cnt[q])));
    }
  return 0;
}

}  // namespace bab
