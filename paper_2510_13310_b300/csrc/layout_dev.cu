// layout_dev.cu -- the observation layout of ba_create (layout.h) built on the
// device: validation, point-order and camera-order permutations by stable radix
// sorts, offsets, tile records and the co-visibility runs.  Only the greedy
// grouping of points into warp ranges and tiles (a sequential scan over the
// point offsets) and the camera chunks run on the host.  The result is the
// host builder's layout bit for bit (tested).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>

#include "layout_dev.h"
#include "tile_meta.cuh"

namespace bab {

namespace {

// ---------------------------------------------------------------------------
// device scratch (stream-ordered allocations, released at scope exit)
// ---------------------------------------------------------------------------

// Stream-ordered scratch from a memory pool of the library's own per device that
// keeps its memory when freed (release threshold: unlimited), so that building a
// second layout maps no new memory; released by release_scratch_pools().
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t scratch_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  g_pools[dev] = pool;
  return pool;
}

struct Scratch {
  cudaStream_t s;
  cudaMemPool_t pool;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st), pool(scratch_pool()) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    if ((pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s)) != cudaSuccess)
      return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

int fail(std::string* err, int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (err) *err = buf;
  return code;
}

#define DCU(expr)                                                                   \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) return fail(err, 2, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

int bits_for(long long n) {  // bits to hold values 0 .. n-1
  int b = 0;
  while (b < 62 && (1LL << b) < n) ++b;
  return b;
}

int grid_for(long long n, int threads) { return (int)std::max(1LL, std::min((n + threads - 1) / threads, 1LL << 20)); }

// ---------------------------------------------------------------------------
// exclusive scan of an int array (in place; optional total)
// ---------------------------------------------------------------------------

constexpr int kScanT = 256, kScanItems = 4, kScanBlock = kScanT * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* total) {
  // sh: kScanT / 32 ints
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) sh[lane] = s;
  }
  __syncthreads();
  const int before = (w ? sh[w - 1] : 0) + x - v;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_tiles(int* data, int m, int* sums) {
  __shared__ int sh[32];
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
  int v[kScanItems], t = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < m ? data[base + i] : 0;
    t += v[i];
  }
  int total;
  int run = block_exclusive_scan(t, sh, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < m) data[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block scans the tile sums (any number: chunked per thread)
__global__ void k_scan_sums(int* sums, int nb, int* total) {
  __shared__ int sh[32];
  const int per = (nb + blockDim.x - 1) / blockDim.x, b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  int t = 0;
  for (int i = b0; i < b1; ++i) t += sums[i];
  int tot;
  int run = block_exclusive_scan(t, sh, &tot);
  for (int i = b0; i < b1; ++i) {
    const int x = sums[i];
    sums[i] = run;
    run += x;
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void k_scan_add(int* data, int m, const int* sums) {
  const int base = blockIdx.x * kScanBlock;
  const int add = sums[blockIdx.x];
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
    if (base + i < m) data[base + i] += add;
}

// exclusive scan of data[0, m); *total (device, nullable) gets the sum
cudaError_t dev_exclusive_scan(int* data, int m, int* total, Scratch& sc, cudaStream_t s) {
  const int nb = std::max(1, (m + kScanBlock - 1) / kScanBlock);
  int* sums = sc.get<int>(nb);
  if (!sums) return cudaErrorMemoryAllocation;
  if (m > 0) k_scan_tiles<<<nb, kScanT, 0, s>>>(data, m, sums);
  else cudaMemsetAsync(sums, 0, sizeof(int), s);
  k_scan_sums<<<1, 1024, 0, s>>>(sums, m > 0 ? nb : 1, total);
  if (m > 0) k_scan_add<<<nb, kScanT, 0, s>>>(data, m, sums);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, payload) on the device, 8-bit digits:
// per pass, block digit histograms, a scan of the (digit, block) counts and a
// stable block scatter (items of a block in slot-major order; within a slot,
// lanes ranked by __match_any_sync, warps by per-warp digit counts)
// ---------------------------------------------------------------------------

constexpr int kSortT = 256, kSortItems = 8, kSortTile = kSortT * kSortItems;

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift, int nb, int* __restrict__ counts) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
#pragma unroll
  for (int sl = 0; sl < kSortItems; ++sl) {
    const int i = base + sl * kSortT + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);  // integer counts: order-free
  }
  __syncthreads();
  counts[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <typename V>
__global__ void k_rs_scatter(const uint32_t* __restrict__ keys, const V* __restrict__ vals, int n, int shift, int nb,
                             const int* __restrict__ offs, uint32_t* __restrict__ keys_out, V* __restrict__ vals_out) {
  __shared__ int run[256];
  __shared__ int wcnt[kSortT / 32][257];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  run[t] = offs[t * nb + blockIdx.x];
  for (int i = t; i < (kSortT / 32) * 257; i += kSortT) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int sl = 0; sl < kSortItems; ++sl) {
    const int i = base + sl * kSortT + t;
    const bool ok = i < n;
    const uint32_t key = ok ? keys[i] : 0u;
    V val{};
    if (ok) val = vals[i];
    const int d = ok ? (int)((key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      int dst = run[d] + rank;
      for (int w = 0; w < warp; ++w) dst += wcnt[w][d];
      keys_out[dst] = key;
      vals_out[dst] = val;
    }
    __syncthreads();
    int sum = 0;
#pragma unroll
    for (int w = 0; w < kSortT / 32; ++w) {
      sum += wcnt[w][t];
      wcnt[w][t] = 0;
    }
    run[t] += sum;
    if (t < kSortT / 32) wcnt[t][256] = 0;
    __syncthreads();
  }
}

// sorts (keys, vals) by the low key_bits bits of the keys; the sorted arrays end
// up in keys/vals (the pointers are swapped with the alternates as needed)
template <typename V>
cudaError_t dev_radix_sort(uint32_t*& keys, V*& vals, uint32_t*& keys_alt, V*& vals_alt, int n, int key_bits,
                           Scratch& sc, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int nb = (n + kSortTile - 1) / kSortTile;
  int* counts = sc.get<int>((size_t)256 * nb);
  if (!counts) return cudaErrorMemoryAllocation;
  for (int shift = 0; shift < std::max(1, key_bits); shift += 8) {
    k_rs_hist<<<nb, kSortT, 0, s>>>(keys, n, shift, nb, counts);
    cudaError_t e = dev_exclusive_scan(counts, 256 * nb, nullptr, sc, s);
    if (e != cudaSuccess) return e;
    k_rs_scatter<V><<<nb, kSortT, 0, s>>>(keys, vals, n, shift, nb, counts, keys_alt, vals_alt);
    std::swap(keys, keys_alt);
    std::swap(vals, vals_alt);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// validation and hash
// ---------------------------------------------------------------------------

struct Flags {
  unsigned long long first_bad;  // first observation with an index out of range
  unsigned long long first_dup;  // first point-order position repeating (point, camera)
  int nonfinite;                 // 1 cameras, 2 points, 4 observations
};

__global__ void k_check_finite(const double* __restrict__ v, long long n, int bit, Flags* fl) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&fl->nonfinite, bit);
}

__global__ void k_check_index(const int32_t* __restrict__ oc, const int32_t* __restrict__ op, int N, int C, int P,
                              Flags* fl) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
    if (oc[k] < 0 || oc[k] >= C || op[k] < 0 || op[k] >= P) atomicMin(&fl->first_bad, (unsigned long long)k);
}

// FNV-1a over 32-bit words of each 256-observation chunk's (camera, point) pairs
// FNV-1a over each 256-observation chunk (camera, point of every observation in
// input order).  Each 64-thread block stages its 16 chunks in shared memory with
// coalesced loads (row stride 257: the 16 hashing threads read distinct banks),
// then one thread per chunk runs the sequential hash.
constexpr int kHashChunks = 16;
__global__ void __launch_bounds__(64) k_hash_chunks(const int32_t* __restrict__ oc, const int32_t* __restrict__ op,
                                                    int N, unsigned long long* __restrict__ dig, int nch) {
  __shared__ int32_t soc[kHashChunks * 257], sop[kHashChunks * 257];
  const long long base = (long long)blockIdx.x * (kHashChunks * 256);
  for (int e = threadIdx.x; e < kHashChunks * 256; e += blockDim.x) {
    const long long k = base + e;
    const int at = (e >> 8) * 257 + (e & 255);
    soc[at] = k < N ? oc[k] : 0;
    sop[at] = k < N ? op[k] : 0;
  }
  __syncthreads();
  const int t = threadIdx.x, c = blockIdx.x * kHashChunks + t;
  if (t >= kHashChunks || c >= nch) return;
  unsigned long long h = 1469598103934665603ull;
  const int n = (int)(min((long long)N, ((long long)c + 1) << 8) - ((long long)c << 8));
  for (int i = 0; i < n; ++i) {
    h = (h ^ (unsigned long long)(unsigned)soc[t * 257 + i]) * 1099511628211ull;
    h = (h ^ (unsigned long long)(unsigned)sop[t * 257 + i]) * 1099511628211ull;
  }
  dig[c] = h;
}

// ---------------------------------------------------------------------------
// orders and offsets
// ---------------------------------------------------------------------------

__global__ void k_keys_from(const int32_t* __restrict__ src, const int* __restrict__ idx, int n,
                            uint32_t* __restrict__ keys, int* __restrict__ vals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = idx ? idx[i] : i;
    keys[i] = (uint32_t)src[k];
    vals[i] = k;
  }
}

// offsets off[0..nkeys] of sorted keys: off[q] = first position with key >= q
__global__ void k_offsets(const uint32_t* __restrict__ keys, int n, int nkeys, int* __restrict__ off) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int kc = (int)keys[i], kp = i ? (int)keys[i - 1] : -1;
    for (int q = kp + 1; q <= kc; ++q) off[q] = i;
    if (i == n - 1)
      for (int q = kc + 1; q <= nkeys; ++q) off[q] = n;
  }
}

// point order: camera and point of each position, duplicate check
__global__ void k_po_fields(const int* __restrict__ po, const uint32_t* __restrict__ pt_sorted,
                            const int32_t* __restrict__ oc, int n, int* __restrict__ po_cam, int* __restrict__ po_pt,
                            Flags* fl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int cam = oc[po[i]], pt = (int)pt_sorted[i];
    po_cam[i] = cam;
    po_pt[i] = pt;
    if (i && pt == (int)pt_sorted[i - 1] && cam == oc[po[i - 1]]) atomicMin(&fl->first_dup, (unsigned long long)i);
  }
}

__global__ void k_co_fields(const int* __restrict__ co_po, const int* __restrict__ po, int n, int* __restrict__ co) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) co[q] = po[co_po[q]];
}

// ---------------------------------------------------------------------------
// tile records (one block per tile; the format of tile_meta.cuh)
// ---------------------------------------------------------------------------

// the tile's observations as camera << 8 | local index, sorted ascending (bitonic)
__device__ void tile_sorted_keys(const TileDesc& d, const int* __restrict__ po_cam, uint32_t* key) {
  for (int i = threadIdx.x; i < kTileObs; i += blockDim.x)
    key[i] = i < d.n_obs ? ((uint32_t)po_cam[d.obs_begin + i] << 8 | (uint32_t)i) : 0xFFFFFFFFu;
  __syncthreads();
  for (int k = 2; k <= kTileObs; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kTileObs; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t a = key[i], b = key[l];
          if (((i & k) == 0) == (a > b)) {
            key[i] = b;
            key[l] = a;
          }
        }
      }
      __syncthreads();
    }
}

__device__ __forceinline__ bool run_start(const uint32_t* key, int j, int n) {
  return j < n && (j == 0 || (key[j] >> 8) != (key[j - 1] >> 8));
}

__global__ void k_tile_runs(TileDesc* __restrict__ descs, const int* __restrict__ po_cam, int* __restrict__ mb) {
  __shared__ uint32_t key[kTileObs];
  TileDesc d = descs[blockIdx.x];
  tile_sorted_keys(d, po_cam, key);
  const int runs = __syncthreads_count(threadIdx.x < kTileObs && run_start(key, threadIdx.x, d.n_obs));
  if (threadIdx.x == 0) {
    descs[blockIdx.x].n_runs = runs;
    mb[blockIdx.x] = tile_meta_bytes(d.n_obs, d.n_pts, runs);
  }
}

__global__ void k_tile_meta_off(TileDesc* __restrict__ descs, const int* __restrict__ off, int n_tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) descs[t].meta_off = off[t];
}

__global__ void k_tile_records(const TileDesc* __restrict__ descs, const int* __restrict__ po_cam,
                               const int* __restrict__ pt_off, const int* __restrict__ wr_pt,
                               const int* __restrict__ tile_wr, unsigned char* __restrict__ meta) {
  __shared__ uint32_t key[kTileObs];
  __shared__ int sh[32];
  const TileDesc d = descs[blockIdx.x];
  tile_sorted_keys(d, po_cam, key);
  const int n = d.n_obs, np = d.n_pts, ob = d.obs_begin;
  int* cam = reinterpret_cast<int*>(meta + d.meta_off);
  int* poff = cam + pad4(n);
  unsigned* runs = reinterpret_cast<unsigned*>(poff + pad4(np + 1));
  int* wr = reinterpret_cast<int*>(runs + pad4(d.n_runs));
  uint8_t* cperm = reinterpret_cast<uint8_t*>(wr + 16);
  uint8_t* lid = cperm + pad16(n);
  for (int i = threadIdx.x; i < pad4(n); i += blockDim.x) cam[i] = i < n ? po_cam[ob + i] : 0;
  for (int j = threadIdx.x; j < pad4(np + 1); j += blockDim.x) poff[j] = j <= np ? pt_off[d.pt_begin + j] - ob : 0;
  // runs of equal cameras: (camera << 8) | first sorted position, compacted by a scan
  const int j = threadIdx.x;  // blockDim.x == kTileObs
  const int f = run_start(key, j, n) ? 1 : 0;
  const int pos = block_exclusive_scan(f, sh, nullptr);
  if (f) runs[pos] = (key[j] >> 8) << 8 | (unsigned)j;
  for (int r = d.n_runs + threadIdx.x; r < pad4(d.n_runs); r += blockDim.x) runs[r] = 0u;
  const int r0 = tile_wr[blockIdx.x], nwr = tile_wr[blockIdx.x + 1] - r0;
  if (threadIdx.x < 16) wr[threadIdx.x] = threadIdx.x <= nwr ? pt_off[wr_pt[r0 + threadIdx.x]] - ob : n;
  for (int i = threadIdx.x; i < pad16(n); i += blockDim.x) cperm[i] = i < n ? (uint8_t)(key[i] & 0xFFu) : 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x)
    for (int i = pt_off[d.pt_begin + p] - ob; i < pt_off[d.pt_begin + p + 1] - ob; ++i) lid[i] = (uint8_t)p;
  for (int i = n + threadIdx.x; i < pad16(n); i += blockDim.x) lid[i] = 0;
}

// ---------------------------------------------------------------------------
// co-visibility runs
// ---------------------------------------------------------------------------

__global__ void k_cv_count(const int* __restrict__ co_po, const int* __restrict__ po_pt, const int* __restrict__ pt_off,
                           int n, int* __restrict__ cnt) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int k = co_po[q];
    cnt[q] = pt_off[po_pt[k] + 1] - k - 1;
  }
}

// pairs in camera order of their first observation (ascending point within each
// first camera), keyed by the camera pair i * C + j
__global__ void k_cv_fill(const int* __restrict__ co_po, const int* __restrict__ po_pt, const int* __restrict__ po_cam,
                          const int* __restrict__ pt_off, const int* __restrict__ off, int n, int C,
                          uint32_t* __restrict__ keys, int2* __restrict__ vals) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int k = co_po[q], pend = pt_off[po_pt[k] + 1], o = off[q];
    const uint32_t ki = (uint32_t)po_cam[k] * (uint32_t)C;
    for (int k2 = k + 1; k2 < pend; ++k2) {
      keys[o + k2 - k - 1] = ki + (uint32_t)po_cam[k2];
      vals[o + k2 - k - 1] = make_int2(k, k2);
    }
  }
}

__global__ void k_cv_flags(const uint32_t* __restrict__ keys, int n, int* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_cv_runs(const uint32_t* __restrict__ keys, const int* __restrict__ rank, int n, int C,
                          int4* __restrict__ runs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (i == 0 || keys[i] != keys[i - 1]) runs[rank[i]] = make_int4((int)(keys[i] / C), (int)(keys[i] % C), i, 0);
}

__global__ void k_cv_counts(int4* __restrict__ runs, int n_runs, int npairs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_runs) runs[r].w = (r + 1 < n_runs ? runs[r + 1].z : npairs) - runs[r].z;
}

}  // namespace

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------

namespace {
int build_obs_layout_impl(int C, int P, int N, const double* d_cams, const double* d_pts, const double* d_uv,
                          const int32_t* d_oc, const int32_t* d_op, bool check_values, const DevAlloc& alloc,
                          cudaStream_t s, DevLayout* L, std::string* err) {
  Scratch sc(s);
  Flags* fl = sc.get<Flags>(1);
  if (!fl) return fail(err, 2, "device scratch allocation failed");
  const int nch = (N + 255) / 256;
  unsigned long long* dig = sc.get<unsigned long long>(nch);
  DCU(cudaMemsetAsync(fl, 0xFF, 2 * sizeof(unsigned long long), s));
  DCU(cudaMemsetAsync(&fl->nonfinite, 0, sizeof(int), s));
  if (C && check_values) k_check_finite<<<grid_for(9LL * C, 256), 256, 0, s>>>(d_cams, 9LL * C, 1, fl);
  if (P && check_values) k_check_finite<<<grid_for(3LL * P, 256), 256, 0, s>>>(d_pts, 3LL * P, 2, fl);
  if (N) {
    if (check_values) k_check_finite<<<grid_for(2LL * N, 256), 256, 0, s>>>(d_uv, 2LL * N, 4, fl);
    k_check_index<<<grid_for(N, 256), 256, 0, s>>>(d_oc, d_op, N, C, P, fl);
    k_hash_chunks<<<(nch + kHashChunks - 1) / kHashChunks, 64, 0, s>>>(d_oc, d_op, N, dig, nch);
  }
  DCU(cudaGetLastError());
  Flags h_fl;
  std::vector<unsigned long long> h_dig((size_t)nch);
  DCU(cudaMemcpyAsync(&h_fl, fl, sizeof(Flags), cudaMemcpyDeviceToHost, s));
  if (nch) DCU(cudaMemcpyAsync(h_dig.data(), dig, sizeof(unsigned long long) * nch, cudaMemcpyDeviceToHost, s));
  DCU(cudaStreamSynchronize(s));
  if (h_fl.nonfinite & 1) return fail(err, 1, "non-finite camera parameter");
  if (h_fl.nonfinite & 2) return fail(err, 1, "non-finite point");
  if (h_fl.nonfinite & 4) return fail(err, 1, "non-finite observation");
  if (h_fl.first_bad != ~0ull) return fail(err, 1, "observation %lld has an index out of range", (long long)h_fl.first_bad);
  {
    auto fnv = [](uint64_t h, int32_t v) { return (h ^ (uint64_t)(uint32_t)v) * 1099511628211ull; };
    uint64_t h = fnv(fnv(1469598103934665603ull, C), P);
    for (uint64_t d : h_dig) h = fnv(fnv(h, (int32_t)(uint32_t)d), (int32_t)(uint32_t)(d >> 32));
    L->obs_hash = h;
  }
  // ---- orders: stably by camera, then stably by point (point order); camera
  // order stably by camera from point order
  auto A = [&](size_t n) { return static_cast<int*>(alloc(sizeof(int) * std::max<size_t>(n, 1))); };
  L->po = A(N), L->co = A(N), L->co_po = A(N), L->po_cam = A(N), L->po_pt = A(N);
  L->pt_off = A((size_t)P + 1), L->cam_off = A((size_t)C + 1);
  if (!L->po || !L->co || !L->co_po || !L->po_cam || !L->po_pt || !L->pt_off || !L->cam_off)
    return fail(err, 3, "device allocation failed");
  uint32_t* k0 = sc.get<uint32_t>(N);
  uint32_t* k1 = sc.get<uint32_t>(N);
  int* v0 = sc.get<int>(N);
  int* v1 = sc.get<int>(N);
  if (!k0 || !k1 || !v0 || !v1) return fail(err, 3, "device scratch allocation failed");
  DCU(cudaMemsetAsync(L->pt_off, 0, sizeof(int) * ((size_t)P + 1), s));
  DCU(cudaMemsetAsync(L->cam_off, 0, sizeof(int) * ((size_t)C + 1), s));
  if (N > 0) {
    const int g = grid_for(N, 256);
    k_keys_from<<<g, 256, 0, s>>>(d_oc, nullptr, N, k0, v0);
    DCU(dev_radix_sort(k0, v0, k1, v1, N, bits_for(C), sc, s));
    // keys: the points of the camera-sorted indices (payload carried into v1)
    k_keys_from<<<g, 256, 0, s>>>(d_op, v0, N, k0, v1);
    std::swap(v0, v1);
    DCU(dev_radix_sort(k0, v0, k1, v1, N, bits_for(P), sc, s));
    DCU(cudaMemcpyAsync(L->po, v0, sizeof(int) * N, cudaMemcpyDeviceToDevice, s));
    k_po_fields<<<g, 256, 0, s>>>(L->po, k0, d_oc, N, L->po_cam, L->po_pt, fl);
    k_offsets<<<g, 256, 0, s>>>(k0, N, P, L->pt_off);
    // camera order: keys = camera of each point-order position, payload = position
    k_keys_from<<<g, 256, 0, s>>>(L->po_cam, nullptr, N, k0, v0);
    DCU(dev_radix_sort(k0, v0, k1, v1, N, bits_for(C), sc, s));
    DCU(cudaMemcpyAsync(L->co_po, v0, sizeof(int) * N, cudaMemcpyDeviceToDevice, s));
    k_co_fields<<<g, 256, 0, s>>>(L->co_po, L->po, N, L->co);
    k_offsets<<<g, 256, 0, s>>>(k0, N, C, L->cam_off);
    DCU(cudaGetLastError());
  }
  // ---- host: offsets back for the duplicate check, tiles and chunks
  std::vector<int> pt_off((size_t)P + 1), cam_off((size_t)C + 1);
  DCU(cudaMemcpyAsync(pt_off.data(), L->pt_off, sizeof(int) * pt_off.size(), cudaMemcpyDeviceToHost, s));
  DCU(cudaMemcpyAsync(cam_off.data(), L->cam_off, sizeof(int) * cam_off.size(), cudaMemcpyDeviceToHost, s));
  DCU(cudaMemcpyAsync(&h_fl, fl, sizeof(Flags), cudaMemcpyDeviceToHost, s));
  DCU(cudaStreamSynchronize(s));
  if (h_fl.first_dup != ~0ull) {
    const long long i = (long long)h_fl.first_dup;
    int pt = 0, cam = 0, k = 0;
    DCU(cudaMemcpy(&pt, L->po_pt + i, sizeof(int), cudaMemcpyDeviceToHost));
    DCU(cudaMemcpy(&k, L->po + i, sizeof(int), cudaMemcpyDeviceToHost));
    DCU(cudaMemcpy(&cam, d_oc + k, sizeof(int), cudaMemcpyDeviceToHost));
    return fail(err, 1, "duplicate observation of point %d in camera %d", pt, cam);
  }
  for (int p = 0; p < P; ++p)
    if (pt_off[p + 1] - pt_off[p] > kTileObs)
      return fail(err, 1, "point %d has %d observations (limit %d)", p, pt_off[p + 1] - pt_off[p], kTileObs);
  std::vector<int> wr_pt{0}, tile_wr{0};
  std::vector<TileDesc> descs;
  int g_rows = 0;
  group_tiles(pt_off.data(), P, &wr_pt, &tile_wr, &descs, &g_rows);
  const int n_tiles = (int)descs.size();
  L->n_tiles = n_tiles;
  L->g_rows = g_rows;
  L->descs = static_cast<TileDesc*>(alloc(sizeof(TileDesc) * std::max(n_tiles, 1)));
  int* d_wr_pt = sc.get<int>(wr_pt.size());
  int* d_tile_wr = sc.get<int>(tile_wr.size());
  int* mb = sc.get<int>((size_t)n_tiles + 1);
  if (!L->descs || !d_wr_pt || !d_tile_wr || !mb) return fail(err, 3, "device allocation failed");
  if (n_tiles) {
    DCU(cudaMemcpyAsync(L->descs, descs.data(), sizeof(TileDesc) * n_tiles, cudaMemcpyHostToDevice, s));
    DCU(cudaMemcpyAsync(d_wr_pt, wr_pt.data(), sizeof(int) * wr_pt.size(), cudaMemcpyHostToDevice, s));
    DCU(cudaMemcpyAsync(d_tile_wr, tile_wr.data(), sizeof(int) * tile_wr.size(), cudaMemcpyHostToDevice, s));
    k_tile_runs<<<n_tiles, kTileObs, 0, s>>>(L->descs, L->po_cam, mb);
    int* d_total = sc.get<int>(1);
    DCU(dev_exclusive_scan(mb, n_tiles, d_total, sc, s));
    k_tile_meta_off<<<(n_tiles + 255) / 256, 256, 0, s>>>(L->descs, mb, n_tiles);
    int total = 0;
    DCU(cudaMemcpyAsync(&total, d_total, sizeof(int), cudaMemcpyDeviceToHost, s));
    DCU(cudaStreamSynchronize(s));
    L->meta_bytes = (size_t)total;
    L->meta = static_cast<unsigned char*>(alloc(std::max<size_t>(L->meta_bytes, 16)));
    if (!L->meta) return fail(err, 3, "device allocation failed");
    k_tile_records<<<n_tiles, kTileObs, 0, s>>>(L->descs, L->po_cam, L->pt_off, d_wr_pt, d_tile_wr, L->meta);
    DCU(cudaGetLastError());
  } else {
    L->meta_bytes = 0;
    L->meta = static_cast<unsigned char*>(alloc(16));
  }
  // ---- camera chunks (host, from the camera offsets)
  std::vector<int> chunk_obs{0}, chunk_cam, cam_chunk((size_t)C + 1, 0);
  for (int c = 0; c < C; ++c) {
    for (int b = cam_off[c]; b < cam_off[c + 1]; b += kChunkObs) {
      chunk_cam.push_back(c);
      chunk_obs.push_back(std::min(b + kChunkObs, cam_off[c + 1]));
    }
    cam_chunk[c + 1] = (int)chunk_cam.size();
  }
  L->n_chunks = (int)chunk_cam.size();
  L->chunk_obs = A(chunk_obs.size()), L->chunk_cam = A(chunk_cam.size()), L->cam_chunk = A(cam_chunk.size());
  if (!L->chunk_obs || !L->chunk_cam || !L->cam_chunk) return fail(err, 3, "device allocation failed");
  DCU(cudaMemcpyAsync(L->chunk_obs, chunk_obs.data(), sizeof(int) * chunk_obs.size(), cudaMemcpyHostToDevice, s));
  if (!chunk_cam.empty())
    DCU(cudaMemcpyAsync(L->chunk_cam, chunk_cam.data(), sizeof(int) * chunk_cam.size(), cudaMemcpyHostToDevice, s));
  DCU(cudaMemcpyAsync(L->cam_chunk, cam_chunk.data(), sizeof(int) * cam_chunk.size(), cudaMemcpyHostToDevice, s));
  L->h_pt_off = std::move(pt_off);
  L->h_cam_off = std::move(cam_off);
  DCU(cudaStreamSynchronize(s));  // host vectors above are released on return
  return 0;
}
}  // namespace

void release_scratch_pools() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto& kv : g_pools) cudaMemPoolTrimTo(kv.second, 0);
}

int build_obs_layout_dev_indices(int C, int P, int N, const int32_t* d_oc, const int32_t* d_op,
                                 const DevAlloc& alloc, cudaStream_t s, DevLayout* L, std::string* err) {
  return build_obs_layout_impl(C, P, N, nullptr, nullptr, nullptr, d_oc, d_op, false, alloc, s, L, err);
}

int build_obs_layout_dev(int C, int P, int N, const double* d_cams, const double* d_pts, const double* d_uv,
                         const int32_t* d_oc, const int32_t* d_op, const DevAlloc& alloc, cudaStream_t s,
                         cudaStream_t vs, DevLayout* L, std::string* err) {
  if (!vs) return build_obs_layout_impl(C, P, N, d_cams, d_pts, d_uv, d_oc, d_op, true, alloc, s, L, err);
  // the value checks run on vs behind the values' uploads while the index work
  // runs on s; their result is read last but reported first (the order of the
  // checks is the same as with one stream)
  Scratch vsc(vs);
  Flags* fl = vsc.get<Flags>(1);
  if (!fl) return fail(err, 2, "device scratch allocation failed");
  DCU(cudaMemsetAsync(&fl->nonfinite, 0, sizeof(int), vs));
  if (C) k_check_finite<<<grid_for(9LL * C, 256), 256, 0, vs>>>(d_cams, 9LL * C, 1, fl);
  if (P) k_check_finite<<<grid_for(3LL * P, 256), 256, 0, vs>>>(d_pts, 3LL * P, 2, fl);
  if (N) k_check_finite<<<grid_for(2LL * N, 256), 256, 0, vs>>>(d_uv, 2LL * N, 4, fl);
  DCU(cudaGetLastError());
  const int rc = build_obs_layout_impl(C, P, N, d_cams, d_pts, d_uv, d_oc, d_op, false, alloc, s, L, err);
  int nonfinite = 0;
  DCU(cudaStreamSynchronize(vs));
  DCU(cudaMemcpy(&nonfinite, &fl->nonfinite, sizeof(int), cudaMemcpyDeviceToHost));
  if (nonfinite & 1) return fail(err, 1, "non-finite camera parameter");
  if (nonfinite & 2) return fail(err, 1, "non-finite point");
  if (nonfinite & 4) return fail(err, 1, "non-finite observation");
  return rc;
}

int build_covis_runs_dev(const DevLayout& L, int C, int N, const DevAlloc& alloc, cudaStream_t s, DevCovis* out,
                         std::string* err) {
  Scratch sc(s);
  out->npairs = 0;
  out->n_runs = 0;
  int* cnt = sc.get<int>((size_t)N + 1);
  int* d_total = sc.get<int>(1);
  if (!cnt || !d_total) return fail(err, 3, "device scratch allocation failed");
  int total = 0;
  if (N > 0) {
    // pair counts in 64-bit first: the total may exceed what the explicit system allows
    k_cv_count<<<grid_for(N, 256), 256, 0, s>>>(L.co_po, L.po_pt, L.pt_off, N, cnt);
    long long total64 = 0;
    {
      // sum of t(t - 1)/2 over points, from the host copy of the point offsets
      for (size_t p = 0; p + 1 < L.h_pt_off.size(); ++p) {
        const long long t = L.h_pt_off[p + 1] - L.h_pt_off[p];
        total64 += t * (t - 1) / 2;
      }
    }
    if (total64 >= (1LL << 30))  // pair indices plus a loop stride stay below 2^31
      return fail(err, 1, "too many co-visible observation pairs (%lld) for the explicit system", total64);
    DCU(dev_exclusive_scan(cnt, N, d_total, sc, s));
    total = (int)total64;
  }
  out->npairs = (size_t)total;
  out->pairs = static_cast<int2*>(alloc(sizeof(int2) * std::max<size_t>(out->npairs, 1)));
  if (!out->pairs) return fail(err, 3, "device allocation failed");
  if (total == 0) {
    out->runs = static_cast<int4*>(alloc(sizeof(int4)));
    return out->runs ? 0 : fail(err, 3, "device allocation failed");
  }
  uint32_t* k0 = sc.get<uint32_t>(total);
  uint32_t* k1 = sc.get<uint32_t>(total);
  int2* v0 = sc.get<int2>(total);
  int2* v1 = sc.get<int2>(total);
  int* flag = sc.get<int>(total);
  if (!k0 || !k1 || !v0 || !v1 || !flag) return fail(err, 3, "device scratch allocation failed");
  k_cv_fill<<<grid_for(N, 256), 256, 0, s>>>(L.co_po, L.po_pt, L.po_cam, L.pt_off, cnt, N, C, k0, v0);
  DCU(dev_radix_sort(k0, v0, k1, v1, total, bits_for((long long)C * C), sc, s));
  DCU(cudaMemcpyAsync(out->pairs, v0, sizeof(int2) * (size_t)total, cudaMemcpyDeviceToDevice, s));
  k_cv_flags<<<grid_for(total, 256), 256, 0, s>>>(k0, total, flag);
  DCU(dev_exclusive_scan(flag, total, d_total, sc, s));
  int n_runs = 0;
  DCU(cudaMemcpyAsync(&n_runs, d_total, sizeof(int), cudaMemcpyDeviceToHost, s));
  DCU(cudaStreamSynchronize(s));
  out->n_runs = n_runs;
  out->runs = static_cast<int4*>(alloc(sizeof(int4) * std::max(n_runs, 1)));
  if (!out->runs) return fail(err, 3, "device allocation failed");
  k_cv_runs<<<grid_for(total, 256), 256, 0, s>>>(k0, flag, total, C, out->runs);
  k_cv_counts<<<(n_runs + 255) / 256, 256, 0, s>>>(out->runs, n_runs, total);
  DCU(cudaGetLastError());
  DCU(cudaStreamSynchronize(s));
  return 0;
}

}  // namespace bab
