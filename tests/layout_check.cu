// Host-side check of the observation layout built by ba_create (csrc/layout.cu):
// invariants against brute-force definitions on random scenes, the input errors,
// and bit-identical layouts for different thread counts and for both sort paths.
// Built and run by tests/test_layout_cpu.py; prints "OK" on success.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <random>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../paper_2510_13310_b300/csrc/layout.h"
#include "../paper_2510_13310_b300/csrc/tile_meta.cuh"

using namespace bab;

static int failures = 0;
#define CHECK(cond, ...)                                   \
  do {                                                     \
    if (!(cond)) {                                         \
      fprintf(stderr, "FAIL %s:%d: ", __FILE__, __LINE__); \
      fprintf(stderr, __VA_ARGS__);                        \
      fprintf(stderr, "\n");                               \
      ++failures;                                          \
      return;                                              \
    }                                                      \
  } while (0)

struct Scene {
  int C, P;
  std::vector<int> oc, op;
  std::vector<double> cams, pts, uv;
  int N() const { return (int)oc.size(); }
};

// random scene: each point seen by a random set of distinct cameras (track
// length in [0, max_track]), observations shuffled into input order
static Scene make(int C, int P, int max_track, unsigned seed) {
  std::mt19937 rng(seed);
  Scene s;
  s.C = C;
  s.P = P;
  std::vector<int> cams(C);
  for (int c = 0; c < C; ++c) cams[c] = c;
  for (int p = 0; p < P; ++p) {
    const int t = (int)(rng() % (unsigned)(std::min(max_track, C) + 1));
    std::shuffle(cams.begin(), cams.end(), rng);
    for (int i = 0; i < t; ++i) {
      s.oc.push_back(cams[i]);
      s.op.push_back(p);
    }
  }
  std::vector<int> perm(s.oc.size());
  for (size_t i = 0; i < perm.size(); ++i) perm[i] = (int)i;
  std::shuffle(perm.begin(), perm.end(), rng);
  std::vector<int> oc2(perm.size()), op2(perm.size());
  for (size_t i = 0; i < perm.size(); ++i) oc2[i] = s.oc[perm[i]], op2[i] = s.op[perm[i]];
  s.oc = oc2;
  s.op = op2;
  s.cams.assign((size_t)C * 9, 0.5);
  s.pts.assign((size_t)P * 3, 0.25);
  s.uv.assign((size_t)s.oc.size() * 2, 100.0);
  return s;
}

static uint64_t digest(const ObsLayout& L, const CovisRuns& cv, int N) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t b) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < b; ++i) h = (h ^ c[i]) * 1099511628211ull;
  };
  mix(L.po.data(), 4 * (size_t)N);
  mix(L.co.data(), 4 * (size_t)N);
  mix(L.co_po.data(), 4 * (size_t)N);
  mix(L.pt_off.data(), 4 * L.pt_off.size());
  mix(L.cam_off.data(), 4 * L.cam_off.size());
  mix(L.descs.data(), sizeof(TileDesc) * L.descs.size());
  mix(L.meta.data(), L.meta.size());
  mix(cv.runs.data(), sizeof(int4) * cv.runs.size());
  mix(cv.pairs.data(), sizeof(int2) * cv.npairs);
  mix(&L.obs_hash, 8);
  return h;
}

static void check_scene(const Scene& s, const char* name) {
  const int N = s.N(), C = s.C, P = s.P;
  ObsLayout L;
  std::string err;
  int rc = build_obs_layout(C, P, N, s.cams.data(), s.pts.data(), s.uv.data(), s.oc.data(), s.op.data(), &L, &err);
  CHECK(rc == 0, "%s: layout failed: %s", name, err.c_str());
  // orders: permutations sorted by (point, camera, index) and (camera, point, index)
  std::vector<int> ref_po(N), ref_co(N);
  for (int k = 0; k < N; ++k) ref_po[k] = ref_co[k] = k;
  std::sort(ref_po.begin(), ref_po.end(), [&](int a, int b) {
    return std::make_tuple(s.op[a], s.oc[a], a) < std::make_tuple(s.op[b], s.oc[b], b);
  });
  std::sort(ref_co.begin(), ref_co.end(), [&](int a, int b) {
    return std::make_tuple(s.oc[a], s.op[a], a) < std::make_tuple(s.oc[b], s.op[b], b);
  });
  for (int i = 0; i < N; ++i) {
    CHECK(L.po[i] == ref_po[i], "%s: po[%d] = %d, expected %d", name, i, L.po[i], ref_po[i]);
    CHECK(L.co[i] == ref_co[i], "%s: co[%d] = %d, expected %d", name, i, L.co[i], ref_co[i]);
    CHECK(L.po_cam[i] == s.oc[L.po[i]] && L.po_pt[i] == s.op[L.po[i]], "%s: po_cam/po_pt at %d", name, i);
    CHECK(L.po[L.co_po[i]] == L.co[i], "%s: co_po at %d", name, i);
  }
  // offsets: number of observations of smaller points (cameras)
  std::vector<int> pc(P + 1, 0), cc(C + 1, 0);
  for (int k = 0; k < N; ++k) pc[s.op[k] + 1]++, cc[s.oc[k] + 1]++;
  for (int p = 0; p < P; ++p) pc[p + 1] += pc[p];
  for (int c = 0; c < C; ++c) cc[c + 1] += cc[c];
  CHECK(L.pt_off == pc, "%s: pt_off", name);
  CHECK(L.cam_off == cc, "%s: cam_off", name);
  // tiles: contiguous whole points, limits, descriptors, camera runs
  int next_pt = 0, g_rows = 0;
  size_t meta_off = 0;
  for (int t = 0; t < L.n_tiles; ++t) {
    const TileDesc& d = L.descs[t];
    CHECK(d.pt_begin == next_pt, "%s: tile %d starts at point %d, expected %d", name, t, d.pt_begin, next_pt);
    CHECK(d.n_pts >= 1 && d.n_pts <= kTileObs && d.n_obs <= kTileObs, "%s: tile %d size", name, t);
    CHECK(d.obs_begin == pc[d.pt_begin] && d.w_row == d.obs_begin &&
              d.n_obs == pc[d.pt_begin + d.n_pts] - pc[d.pt_begin],
          "%s: tile %d observations", name, t);
    CHECK(d.g_row == g_rows, "%s: tile %d g_row", name, t);
    CHECK((size_t)d.meta_off == meta_off, "%s: tile %d meta offset", name, t);
    std::set<int> cams;
    for (int i = 0; i < d.n_obs; ++i) cams.insert(L.po_cam[d.obs_begin + i]);
    CHECK(d.n_runs == (int)cams.size(), "%s: tile %d runs %d, expected %zu", name, t, d.n_runs, cams.size());
    next_pt += d.n_pts;
    g_rows += (d.n_obs + 3) & ~3;
    meta_off += (size_t)tile_meta_bytes(d.n_obs, d.n_pts, d.n_runs);
  }
  CHECK(next_pt == P || (P > 0 && L.n_tiles > 0 && next_pt == P), "%s: tiles cover %d of %d points", name, next_pt, P);
  CHECK(L.g_rows == g_rows, "%s: g_rows", name);
  // chunks: each camera's observations in pieces of at most kChunkObs
  for (int c = 0; c < C; ++c) {
    int b = cc[c];
    for (int q = L.cam_chunk[c]; q < L.cam_chunk[c + 1]; ++q) {
      CHECK(L.chunk_cam[q] == c && L.chunk_obs[q + 1] > b && L.chunk_obs[q + 1] - b <= kChunkObs,
            "%s: chunk %d of camera %d", name, q, c);
      b = L.chunk_obs[q + 1];
    }
    CHECK(b == cc[c + 1], "%s: chunks of camera %d end at %d, expected %d", name, c, b, cc[c + 1]);
  }
  // co-visibility runs against a brute-force enumeration over points
  CovisRuns cv;
  rc = build_covis_runs(L, C, N, &cv, &err);
  CHECK(rc == 0, "%s: covis failed: %s", name, err.c_str());
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> ref;
  for (int p = 0; p < P; ++p)
    for (int k = pc[p]; k < pc[p + 1]; ++k)
      for (int k2 = k + 1; k2 < pc[p + 1]; ++k2) ref[{L.po_cam[k], L.po_cam[k2]}].push_back({k, k2});
  CHECK(cv.runs.size() == ref.size(), "%s: %zu runs, expected %zu", name, cv.runs.size(), ref.size());
  size_t r = 0, total = 0;
  for (const auto& kv : ref) {  // std::map iterates (i, j) ascending, as the runs are
    const int4 rn = cv.runs[r++];
    CHECK(rn.x == kv.first.first && rn.y == kv.first.second && rn.x < rn.y && rn.z == (int)total &&
              rn.w == (int)kv.second.size(),
          "%s: run (%d, %d)", name, rn.x, rn.y);
    for (size_t q = 0; q < kv.second.size(); ++q)
      CHECK(cv.pairs[total + q].x == kv.second[q].first && cv.pairs[total + q].y == kv.second[q].second,
            "%s: pair %zu of run (%d, %d)", name, q, rn.x, rn.y);
    total += kv.second.size();
  }
  CHECK(cv.npairs == total, "%s: %zu pairs, expected %zu", name, cv.npairs, total);
  // the same bits with other thread counts and with the wide-key sort
  const uint64_t h0 = digest(L, cv, N);
  for (int variant = 0; variant < 3; ++variant) {
    setenv("BA_HOST_THREADS", variant == 0 ? "1" : variant == 1 ? "7" : "3", 1);
    ObsLayout L2;
    CovisRuns cv2;
    rc = build_obs_layout(C, P, N, s.cams.data(), s.pts.data(), s.uv.data(), s.oc.data(), s.op.data(), &L2, &err,
                          variant == 2);
    CHECK(rc == 0, "%s: variant %d failed", name, variant);
    rc = build_covis_runs(L2, C, N, &cv2, &err);
    CHECK(rc == 0 && digest(L2, cv2, N) == h0, "%s: variant %d differs", name, variant);
  }
  unsetenv("BA_HOST_THREADS");
}

static void check_errors() {
  Scene s = make(6, 40, 5, 11);
  std::string err;
  auto run = [&](const Scene& t) {
    ObsLayout L;
    err.clear();
    return build_obs_layout(t.C, t.P, t.N(), t.cams.data(), t.pts.data(), t.uv.data(), t.oc.data(), t.op.data(), &L,
                            &err);
  };
  Scene d = s;  // a duplicate (camera, point)
  d.oc.push_back(d.oc[3]);
  d.op.push_back(d.op[3]);
  d.uv.push_back(1.0), d.uv.push_back(2.0);
  CHECK(run(d) == 1 && err.find("duplicate") != std::string::npos, "duplicate not rejected: %s", err.c_str());
  Scene o = s;  // an index out of range
  o.op[7] = o.P;
  CHECK(run(o) == 1 && err.find("out of range") != std::string::npos, "bad index not rejected: %s", err.c_str());
  Scene f = s;  // a non-finite observation
  f.uv[5] = std::nan("");
  CHECK(run(f) == 1 && err.find("non-finite") != std::string::npos, "NaN not rejected: %s", err.c_str());
  Scene lng = make(300, 3, 0, 5);  // a point seen by 257 cameras
  for (int c = 0; c < kTileObs + 1; ++c) lng.oc.push_back(c), lng.op.push_back(1);
  lng.uv.assign(lng.oc.size() * 2, 1.0);
  CHECK(run(lng) == 1 && err.find("limit") != std::string::npos, "long track not rejected: %s", err.c_str());
  Scene ok = make(300, 3, 0, 5);  // exactly 256 is fine
  for (int c = 0; c < kTileObs; ++c) ok.oc.push_back(c), ok.op.push_back(1);
  ok.uv.assign(ok.oc.size() * 2, 1.0);
  CHECK(run(ok) == 0, "a 256-observation point rejected: %s", err.c_str());
}

int main() {
  check_scene(make(7, 50, 7, 1), "small");
  check_scene(make(40, 3000, 40, 2), "long tracks");
  check_scene(make(25, 2000, 3, 3), "short tracks, empty points");
  check_scene(make(300, 400, 12, 4), "many cameras, empty cameras");
  check_scene(make(5, 0, 0, 5), "no points");
  check_scene(make(5, 10, 0, 6), "no observations");
  check_errors();
  if (failures) {
    fprintf(stderr, "%d failure(s)\n", failures);
    return 1;
  }
  printf("OK\n");
  return 0;
}
