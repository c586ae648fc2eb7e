// internal.h -- device views and kernel launchers shared by the library's host code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "df.cuh"

namespace bab {

// One tile of whole points in point order.  W rows of the tile start at w_row
// (a multiple of 4, so every tile starts on a 16-byte boundary); its static
// metadata (camera of each observation, point offsets, camera runs, positions in
// camera order) is a 16-byte aligned record at meta_off.
struct TileDesc {
  int w_row, n_obs, pt_begin, n_pts;
  int meta_off, n_runs, obs_begin, g_row;  // g_row: first row of per-observation arrays
                                           // padded to 4 rows per tile (16-byte aligned)
};

// Immutable observation layout built by ba_create.  "po" = point order (sorted by
// point, then camera), "co" = camera order (sorted by camera, then point).
struct Layout {
  int C, P, N;
  int n_tiles, n_chunks;
  const int* po_cam;       // [N]
  const int* po_pt;        // [N]
  const int* po_orig;      // [N] input index
  const double* po_uv64;   // [N][2]
  const double* po_tau64;  // [N] inverse-depth target m/d (0 without prior)
  const void* po_uvw;      // [N][2] working precision
  const void* po_tauw;     // [N]
  const int* pt_off;       // [P+1]
  const int* co_pt;        // [N]
  const int* co_po;        // [N] point-order index of each camera-order observation
  const void* co_uvw;      // [N][2]
  const void* co_tauw;     // [N]
  const TileDesc* descs;   // [n_tiles]
  const int* po_wrow;      // [N] W row of each point-order observation
  const int* chunk_obs;    // [n_chunks+1]
  const int* chunk_cam;    // [n_chunks]
  const int* cam_chunk;    // [C+1] chunk range of each camera
  const uint8_t* cam_fixed;  // [C]
  const float4* po_uvdf;   // [N] (u, v) as double-float pairs (FP32 problems; else null)
  const F2* po_taudf;      // [N] tau as a double-float pair (FP32 problems; else null)
};

// model constants of the double-float evaluation as (hi, lo) pairs
struct EvalDFConst {
  F2 cx, cy, huber, huber2, two_huber, sw_valid, sw_invalid, min_depth, img_w, img_h, drop2;
};

struct ModelParams {
  int cam_model;   // 0 radial, 1 centre + rotation + focal (model.cuh)
  double cx, cy, huber, sw_valid, sw_invalid, min_depth, drop_px;
  int img_w, img_h;
};

template <typename T>
struct PcgArgs {
  int recompute;                // 1: recompute Jacobian blocks from wsgn, points and cameras
  const T* W;                   // stored W rows (recompute == 0)
  const T* wsgn;                // signed IRLS weight per observation (recompute == 1)
  const T* ptsw;                // working points [P+2][4] (recompute == 1)
  const T* camw;                // working cameras [C][16] (recompute == 1)
  int cam_in_smem;              // stage the camera table in shared memory
  double sw_valid, sw_invalid;  // square roots of the depth-row weights
  int max_tiles_per_block;
  const TileDesc* descs;
  const unsigned char* meta;    // tile metadata records
  int n_tiles;
  int stages;                   // 2: double-buffered tile copies, 1: single buffer
  const T* Vinv;                // [P+2][6]
  const int* crank;
  int C;
  const T* Ud;
  const T* Dinv;
  const T* b;
  int Cf, n;
  int own_max;                  // largest owned camera slice of a block
  T *x, *z;
  T* partials;
  double* dots;                 // [2][G][4]
  unsigned* bar;
  int* err;
  Scalars* sc;
  double tol;
  int max_iters;
  long long timeout_ns;
  // back-substitution
  const T* gp;
  const T* V;
  double lambda;
  T* dp;
  double* pred_parts;           // [G] (+1 slot for the camera part)
};

template <typename T>
struct SpcgArgs {
  const T* Shat;                // scaled reduced camera system [n][n]
  const T* Dinv;                // unscaled block-Jacobi inverses [Cf][81]
  const double* dscale;         // D = sqrt(diag U*) [n], then 1/D in T
  const T* b;                   // Schur right-hand side [n]
  int Cf, n, rows_in_smem, vecs_in_smem;
  T* x;                         // solution [n]
  const T* Mshared;              // preconditioner blocks shared by all blocks (nullable)
  T* scratch;                   // per-block vectors when not in shared memory
  size_t scratch_stride;        // elements per block of scratch
  unsigned long long* words;    // exchange words [2][replicas][n][sizeof(T)/4]
  unsigned tag_base;            // first iteration tag of this launch (>= 1)
  int* err;
  Scalars* sc;
  double tol;
  int max_iters;
  long long timeout_ns;
  // block-sparse S^ (nullable otherwise): block rows by camera, entries (column
  // camera, block slot), blocks of kBlkStride entries; ranks and their cameras
  const int* brp;
  const int2* bent;
  const T* Bs;
  const int* crank;
  const int* cam_map;
};
// entries per stored 9x9 block of the block-sparse system (row-major, padded to
// 16 bytes in FP32)
constexpr int kBlkStride = 84;

// message returned by ba_last_error() for the calling thread
void set_last_error_message(const char* msg);
cudaError_t tc_gemm_nt(const float* A, long long lda, const float* B, long long ldb, float* C, long long ldc,
                       int M, int N, int K, float alpha, float beta, bool lower_only, int* err, cudaStream_t s);
cudaError_t dense_cholesky_tc(float* A, long long lda, int np, float* Linv, int* err, cudaStream_t s,
                              long long* launches);

// Work buffers of the dense solver (np = n rounded up to 128):
// A [np][np] factor, Linv [np/128][128][128], vec [4][np], part [256], scal [8],
// flags [np/128], err [1]; *epoch increases by one per triangular solve.
struct DenseWork {
  float* A = nullptr;
  float* Linv = nullptr;
  float* vec = nullptr;
  double* part = nullptr;
  double* scal = nullptr;
  unsigned* flags = nullptr;
  int* err = nullptr;
  unsigned* epoch = nullptr;  // host counter
};
struct DenseResult {
  int iters = 0;
  double rel_res = 0.0;
  int flags = 0;       // 2 breakdown, 16 pipeline timeout, 32 non-positive pivot (after the retries)
  double shift = 0.0;  // diagonal shift of the factored matrix (0 unless a pivot failed)
  long long launches = 0;
};
cudaError_t dense_trsv(bool back, const float* L, long long ld, const float* Linv, const float* rhs, float* out,
                       int T, unsigned* flags, unsigned epoch, int* err, int num_sms, cudaStream_t s);
// reuse_factor: S and the factor in w.A are those of the previous call (whose
// result *res still holds); only the preconditioned CG runs
cudaError_t dense_spd_solve(const DenseWork& w, const float* S, long long ld_s, int n, const float* b, float* x,
                            double tol, int max_iters, int num_sms, cudaStream_t s, DenseResult* res,
                            bool reuse_factor = false);
cudaError_t launch_scale_vec(int n, const float* a, const float* d, float* out, cudaStream_t s);
cudaError_t launch_set_pcg_info(Scalars* sc, int iters, double rel, int* err, int errbits, cudaStream_t s);

// ---- launchers (return cudaGetLastError of the launch) ----
template <typename T>
cudaError_t launch_prep_cams(const double* cams64, T* camw, double* camw64, int C, cudaStream_t s,
                             int model = 0);  // camera model of the working records (model.cuh)
template <typename T>
cudaError_t launch_prep_pts(const double* pts64, T* ptsw, int P, cudaStream_t s);
// uv and inverse-depth priors in point order and camera order (and the W row of
// each point-order observation) from the caller's arrays (uv, depth: input order)
// through the permutations po and co; the working-precision point-order arrays
// are skipped when po_uvw is null
template <typename T>
cudaError_t launch_obs_layout(int N, const double* uv, const double* depth, const int* po, const int* co,
                              const int* co_po, const int* po_pt, int* po_wrow, double* po_uv64, double* po_tau64,
                              T* po_uvw, T* po_tauw, int* co_pt, T* co_uvw, T* co_tauw, cudaStream_t s);

// partials (nullable): per-block sums; the last block reduces them into
// sc->cost[slot], rmse_sum[slot], n_act[slot]
cudaError_t launch_eval64(const Layout& L, const ModelParams& mp, const double* camw64,
                          const double* pts64, const uint8_t* act, uint8_t* bits,
                          const uint8_t* ref_bits, int* flips, double* partials, Scalars* sc, int slot, int grid,
                          cudaStream_t s);
// double-float evaluation of FP32 problems (same outputs as launch_eval64);
// camdf [C][16] and ptdf [P][2]: the state slot as double-float pairs
cudaError_t launch_eval_df(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                           F2* camdf, float4* ptdf, bool convert, const uint8_t* act, uint8_t* bits,
                           const uint8_t* ref_bits, int* flips, double* partials, Scalars* sc, int slot, int grid,
                           cudaStream_t s);  // convert: fill camdf/ptdf from camw64/pts64 first
cudaError_t launch_obs_df(int N, const double* uv64, const double* tau64, float4* uvdf, F2* taudf, cudaStream_t s);

cudaError_t launch_extract_begin(const Layout& L, uint8_t* alive, const uint8_t* bits,
                                 uint8_t* valid, int drop, cudaStream_t s);
cudaError_t launch_fill_u8(uint8_t* p, uint8_t v, int n, cudaStream_t s);
cudaError_t launch_peel_points(const Layout& L, const uint8_t* valid, const uint8_t* cam_act,
                               uint8_t* pt_act, int* cam_cnt, int min_pt, Scalars* sc,
                               cudaStream_t s);
cudaError_t launch_peel_cams(const Layout& L, uint8_t* cam_act, int* cam_cnt, int min_cam,
                             Scalars* sc, cudaStream_t s);
cudaError_t launch_finalize_obs(const Layout& L, const uint8_t* valid, const uint8_t* cam_act,
                                const uint8_t* pt_act, uint8_t* obs_act, uint8_t* obs_act_co,
                                Scalars* sc, cudaStream_t s);
cudaError_t launch_cam_flags(const Layout& L, const uint8_t* cam_act, uint8_t* flags, Scalars* sc, cudaStream_t s);
// ranks of nonzero flags: rank[i] (-1 if zero), map[rank] = i, *count
cudaError_t launch_rank(const uint8_t* flags, int n, int* rank, int* map, int* count,
                        int* block_tmp, int n_block_tmp, cudaStream_t s);
int rank_blocks(int n);

template <typename T>
cudaError_t launch_pt_lin(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                          const uint8_t* obs_act, T* W, T* wsgn, T* V, T* gp, cudaStream_t s,
                          float* orec = nullptr);  // FP32 explicit systems: observation records [N][16]
template <typename T>
cudaError_t launch_cam_accum(const Layout& L, const ModelParams& mp, int mode, const T* camw,
                             const T* ptsw, const uint8_t* act_co, const uint8_t* cam_act,
                             const int* crank, const T* Vinv, const T* z0, T* partials,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_cam_reduce(const Layout& L, const T* partials, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_damp_pts(int P, const T* V, const T* gp, const uint8_t* pt_act, double lambda,
                            T* Vinv, T* z0, int* err, cudaStream_t s,
                            float* prec = nullptr);      // FP32: point records [P][8] (V*^-1, 0, 0)
template <typename T>
cudaError_t launch_schur_diag(int Cf, const int* cam_map, const T* Ug, const T* Sg, double lambda,
                              T* Ud, T* Dinv, T* b, T* dampc, T* Dblk, double* dscale, int* err,
                              cudaStream_t s,
                              int kfix = 0);  // dscale (nullable): D and 1/D of the explicit system
// Camera-owned formation of the explicit system (FP32): every co-visibility run
// (i, j) is summed by its owner camera (run_owner_first), whose Y^ rows, stored in
// camera order, are staged in shared memory chunk by chunk; pairs hold (owner's
// camera-order row, other's camera-order row).  Block d covers blocks[d] =
// (camera, first index into own_run, run count, 0).
struct CamForm {
  const int4* blocks = nullptr;
  int n_blocks = 0;
  const int* own_run = nullptr;  // runs grouped by owner camera
  const int* cam_off = nullptr;  // [C + 1] camera-order offsets
  const int* po_co = nullptr;    // [N] camera-order position of each point-order observation
};
__host__ __device__ constexpr bool run_owner_first(int i, int j) { return ((i + j) & 1) == 0; }
cudaError_t launch_owner_pairs(int N, const int* co_po, int* po_co, int n_runs, const int4* runs, int2* pairs,
                               cudaStream_t s);

// FP32 warp-per-run formation from observation records (k_form_S_rec): the
// records written by the point-side linearisation, the point of every pair, the
// working camera records
struct FormRec {
  const float* rec = nullptr;      // [N][16] observation records
  const int* pair_pt = nullptr;    // [npairs]
  const void* camw = nullptr;      // working cameras [C][kCamStride] (FP32)
  const float* prec = nullptr;     // [P][8] point records: V*^-1 (6), 0, 0
  bool centre = false;             // the camera model of Sec. 3.2 (centre, rotation, focal)
};
cudaError_t launch_pair_pt(size_t npairs, const int2* pairs, const int* po_pt, int* pair_pt, cudaStream_t s);
template <typename T>
cudaError_t launch_form_S(const Layout& L, int n_runs, const int4* runs, const int2* pairs, const T* W,
                          const T* Vinv, const int* crank, const T* Ud, const T* Dblk, double* dscale,
                          int Cf, T* Y, T* Shat, bool lanes, int num_sms, cudaEvent_t ev0, cudaEvent_t ev1,
                          cudaEvent_t join, cudaStream_t s,   // join (nullable): waited on before the
                                                              // diagonal blocks are written
                          const int* cam_map = nullptr,       // sparse: Shat is the block storage
                          bool sparse = false,
                          const CamForm* cf = nullptr,        // FP32: camera-owned formation
                          const FormRec* fr = nullptr);       // FP32: formation from observation records
template <typename T>
cudaError_t launch_dscale(int Cf, const int* cam_map, const T* Ug, double lambda, double* dscale, cudaStream_t s, int kfix = 0);
template <typename T>
size_t spcg_smem_bytes(int n, int rows, int rows_in_smem, int vecs_in_smem, int Cf);
// row stride of S^: FP32 rows padded to a multiple of 4 entries (zeros)
template <typename T>
__host__ __device__ inline int spcg_row_stride(int n) {
  return sizeof(T) == 4 ? (n + 3) & ~3 : n;
}
template <typename T>
__host__ __device__ size_t spcg_vec_elems(int n, int Cf);
template <typename T>
const void* spcg_kernel_ptr(bool rows_in_smem);
template <typename T>
cudaError_t launch_spcg(const SpcgArgs<T>& a, int grid, size_t smem, cudaStream_t s);
// partitioned PCG on the block-sparse system (each block owns a slice of cameras)
template <typename T>
cudaError_t launch_bspcg(const SpcgArgs<T>& a, int grid, size_t smem, cudaStream_t s);
template <typename T>
size_t bspcg_smem_bytes(int Cf, int grid);
template <typename T>
const void* bspcg_kernel_ptr();
// the explicit PCG's preconditioner blocks into M [Cf][kSpcgMStride], for a shared copy
constexpr int kSpcgMStride = 84;
template <typename T>
cudaError_t launch_spcg_precond(int Cf, const T* Dinv, const double* dscale, T* M, cudaStream_t s);
int spcg_threads();
int spcg_words_per_value(bool fp64);
template <typename T>
cudaError_t launch_backsub_pts(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                               const uint8_t* act_po, const uint8_t* pt_act, const int* crank, const T* x,
                               const T* Vinv, const T* V, const T* gp, const T* Wst, double lambda, T* dp,
                               T* wx, int Cf, const int* cam_map, const T* Ug, const T* dampc, double* pred_parts,
                               Scalars* sc, int grid, cudaStream_t s,  // also sc->pred (points and cameras)
                               const float* orec = nullptr);  // FP32: W^T x from the observation records
template <typename T>
cudaError_t launch_pcg(const PcgArgs<T>& a, int grid, size_t smem, cudaStream_t s);
template <typename T>
size_t pcg_smem_bytes(int n, int C, int stages, int own_max, int recompute, int cam_in_smem,
                      int max_tiles_per_block);
template <typename T>
const void* pcg_kernel_ptr();
int pcg_threads();
int pcg_max_stages();
template <typename T>
cudaError_t launch_pred_cams(int Cf, const int* cam_map, const T* x, const T* Ug, const T* dampc,
                             double lambda, double* pred_parts, int offset, cudaStream_t s);
cudaError_t launch_reduce_pred(const double* parts, int n, Scalars* sc, cudaStream_t s);
template <typename T>
cudaError_t launch_candidate(int C, int P, const int* crank, const T* x, const T* dp,
                             const double* cams_src, const double* pts_src, double* cams_dst,
                             double* pts_dst, double* camw64_dst, T* camw_dst, T* ptsw_dst,
                             F2* camdf_dst, float4* ptdf_dst, cudaStream_t s,  // *df_dst nullable
                             int model = 0);
template <typename T>
cudaError_t launch_scatter_cams(int C, const int* crank, const T* x, double* dc, cudaStream_t s);
// a_c [9C], a_p [3P] (nullable): the right-hand side dL/dtheta in the solve's coordinates, FP64
template <typename T>
cudaError_t launch_adjoint_rhs(int C, int P, const double* cams64, const int* crank, const uint8_t* pt_act,
                               const double* dL_dc, const double* dL_dp, T* Ug, T* gp, cudaStream_t s,
                               double* a_c = nullptr, double* a_p = nullptr, int kfix = 0);
// FP64-residual refinement of the adjoint solve (adjoint.cu): H mu in FP64 from the
// FP64 state (u_obs [3N] point order, hmu_p [3P], part [9 n_chunks]), the residual
// a - H mu into the gradient slots, mu accumulation, and the outputs from mu
cudaError_t launch_adj_hmu(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                           const uint8_t* act_po, const uint8_t* act_co, const int* crank, const double* mu_c,
                           const double* mu_p, double* u_obs, double* hmu_p, double* part, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_residual(int C, int P, const int* cam_chunk, const int* crank, const uint8_t* pt_act,
                                const double* part, const double* hmu_p, const double* a_c, const double* a_p,
                                T* Ug, T* gp, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_mu_add(int Cf, int P, const T* x, const T* dp, double* mu_c, double* mu_p, bool first,
                              cudaStream_t s);
cudaError_t launch_adjoint_obs64(const Layout& L, const ModelParams& mp, const double* camw64, const double* pts64,
                                 const uint8_t* act_po, const int* crank, const double* mu_c, const double* mu_p,
                                 double* duv, double* ddepth, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_obs(const Layout& L, const ModelParams& mp, const T* camw, const T* ptsw,
                               const uint8_t* act_po, const int* crank, const T* x, const T* dp, double* duv,
                               double* ddepth, cudaStream_t s);
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t s);
cudaError_t launch_permute_u8(const int* orig, const uint8_t* src, uint8_t* dst, int N,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_permute_rows(const int* orig, const int* row, const T* src, int src_stride,
                                double* dst, int N, int width, cudaStream_t s);

// first index-check failure of each translation unit in BA_DEBUG_BOUNDS builds
// (((site + 1) << 32) | index, 0 if none; ~0 if it could not be read), cleared
// when reset; 0 in release builds
unsigned long long bounds_fault_kernels(bool reset);
unsigned long long bounds_fault_schur(bool reset);
unsigned long long bounds_fault_adjoint(bool reset);

}  // namespace bab
