// tile_meta.cuh -- the point tiles of the implicit Schur matvec and their
// metadata records: written on the host by the layout builder (layout.cu), read
// by the PCG kernels (pcg.cu).
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace bab {

constexpr int kPcgThreads = 256;
constexpr int kPcgWarps = kPcgThreads / 32;  // warp ranges per tile

__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__host__ __device__ __forceinline__ int pad16(int x) { return (x + 15) & ~15; }

// Metadata record of a tile (16-byte aligned, every field a multiple of 16 B):
//   int  cam[pad4(n_obs)]        camera of each observation
//   int  poff[pad4(n_pts+1)]     tile-local observation offset of each point
//   uint runs[pad4(n_runs)]      (camera << 8) | start, runs of equal cameras in camera order
//   int  wr[16]                  observation offsets of the warp ranges (n_wr + 1 used)
//   u8   cperm[pad16(n_obs)]     tile-local positions sorted by camera
//   u8   lid[pad16(n_obs)]       tile-local point of each observation
__host__ __device__ __forceinline__ int tile_meta_bytes(int n_obs, int n_pts, int n_runs) {
  return 4 * pad4(n_obs) + 4 * pad4(n_pts + 1) + 4 * pad4(n_runs) + 64 + 2 * pad16(n_obs);
}
constexpr int kMetaBytes = 4 * kTileObs + 4 * (kTileObs + 4) + 4 * kTileObs + 64 + 2 * kTileObs;

// Writes one tile's record (tile_meta_bytes(n_obs, n_pts, n_runs) bytes at out).
inline void build_tile_meta(int n_obs, int n_pts, int n_runs, int n_wr, const int* cams, const int* poff,
                     const unsigned* runs, const int* wr, const uint8_t* cperm, const uint8_t* lid,
                     unsigned char* out) {
  int* c = reinterpret_cast<int*>(out);
  for (int i = 0; i < pad4(n_obs); ++i) c[i] = i < n_obs ? cams[i] : 0;
  int* po = c + pad4(n_obs);
  for (int i = 0; i < pad4(n_pts + 1); ++i) po[i] = i <= n_pts ? poff[i] : 0;
  unsigned* r = reinterpret_cast<unsigned*>(po + pad4(n_pts + 1));
  for (int i = 0; i < pad4(n_runs); ++i) r[i] = i < n_runs ? runs[i] : 0u;
  int* w = reinterpret_cast<int*>(r + pad4(n_runs));
  for (int i = 0; i < 16; ++i) w[i] = i <= n_wr ? wr[i] : n_obs;
  uint8_t* cp = reinterpret_cast<uint8_t*>(w + 16);
  for (int i = 0; i < pad16(n_obs); ++i) cp[i] = i < n_obs ? cperm[i] : 0;
  uint8_t* li = cp + pad16(n_obs);
  for (int i = 0; i < pad16(n_obs); ++i) li[i] = i < n_obs ? lid[i] : 0;
}


}  // namespace bab
