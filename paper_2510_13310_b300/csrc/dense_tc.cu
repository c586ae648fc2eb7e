// dense_tc.cu -- dense symmetric positive definite factorisation of the reduced
// camera system on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// When many cameras see the same points the Schur complement S (Eq. LM, Schur
// form) is dense, and a direct factorisation replaces hundreds of PCG
// iterations.  S^ = L L^T is computed by a blocked right-looking Cholesky:
// 128 x 128 tiles, panels of kPanelTiles tile columns.  Per tile column j the
// diagonal tile is factored and inverted on CUDA cores in FP32 (k_potrf_tile);
// the tiles below it become L_ij = A_ij L_jj^-T, a product with the explicit
// inverse; the remaining tile columns of the panel are updated with K = 128.
// After each panel the trailing matrix takes one rank-(128 kPanelTiles) update
// A_il -= L_i,P L_l,P^T, the bulk of the n^3/3 flops.  All three products run
// in k_tc_gemm_nt: operands streamed by TMA (128-byte swizzle) through a
// 4-stage mbarrier ring, tcgen05.mma issued by one thread, FP32 accumulators in
// tensor memory, read back with tcgen05.ld for the epilogue.  Operands are FP32
// in memory and enter the tensor cores as TF32 (10-bit mantissa); the factor is
// used as a preconditioner, so the solution is recovered to FP32 accuracy by
// the conjugate-gradient refinement in dense_solve.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdarg.h>
#include <stdio.h>

#include "../../include/ba_b300.h"
#include "internal.h"
#include "tma.cuh"

namespace bab {

constexpr int kTcBM = 128;      // output tile rows (UMMA M)
constexpr int kTcBN = 256;      // output tile columns (UMMA N)
constexpr int kTcBK = 32;       // K per pipeline stage: 32 FP32 = one 128-byte swizzle row
constexpr int kTcStages = 4;
constexpr int kTcThreads = 128;
constexpr int kTcStageBytes = (kTcBM + kTcBN) * kTcBK * 4;  // 48 KB
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long kTcTimeoutNs = 1000000000LL;

cudaError_t tc_gemm_nt(const float* A, long long lda, const float* B, long long ldb, float* C, long long ldc,
                       int M, int N, int K, float alpha, float beta, bool lower_only, int* err, cudaStream_t s);

// ---------------------------------------------------------------------------
// tcgen05 / TMA inline PTX
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzled
// layout TMA writes: rows of 128 B, 8-row groups 1024 B apart (SBO), leading
// offset unused for this layout, descriptor version 1, swizzle mode 128B.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// mbarrier arrives once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns: thread i of the warp gets lane
// (lane base + i), columns [col, col + 32).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// C = alpha A B^T + beta C over a grid of 128 x 256 output tiles.
// A: M x K, B: N x K, both row-major FP32 (K contiguous), seen through tensor
// maps with boxes {32, 128} and {32, 256}; rows and columns past M, N, K read
// as zero.  C row-major, ldc.  lower_only: tiles wholly above the diagonal
// (first row > last column... i.e. row tile end <= column tile start) are
// skipped; used for symmetric updates of the lower triangle.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm_nt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float* C,
                 long long ldc, int M, int N, int K, float alpha, float beta, int tiles_n, int lower_only,
                 int vec_ok, int* err) {
  extern __shared__ unsigned char tc_smem_raw[];
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x - (blockIdx.x / tiles_n) * tiles_n;
  const int row0 = tm * kTcBM, col0 = tn * kTcBN;
  if (lower_only && row0 + kTcBM <= col0) return;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kTcStages * kTcStageBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, kTcBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nk = (K + kTcBK - 1) / kTcBK;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      if (kb >= kTcStages && !mbar_wait(&empty[s], ((kb / kTcStages) & 1) ^ 1, kTcTimeoutNs)) {
        ok = false;
        break;
      }
      unsigned char* sa = base + s * kTcStageBytes;
      unsigned char* sb = sa + kTcBM * kTcBK * 4;
      mbar_arrive_expect_tx(&full[s], kTcStageBytes);
      tma_load_2d(sa, &tmA, kb * kTcBK, row0, &full[s]);
      tma_load_2d(sb, &tmB, kb * kTcBK, col0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: 4 x (128 x 256 x 8) per stage
    constexpr uint32_t idesc = umma_idesc_tf32(kTcBM, kTcBN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kTcStages;
      if (!mbar_wait(&full[s], (kb / kTcStages) & 1, kTcTimeoutNs)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(base + s * kTcStageBytes);
      const uint32_t sb = sa + kTcBM * kTcBK * 4;
#pragma unroll
      for (int kk = 0; kk < kTcBK / 8; ++kk)
        umma_tf32(tmem, umma_desc_sw128(sa + kk * 32), umma_desc_sw128(sb + kk * 32), idesc,
                  (kb > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(done);
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes [32w, 32w + 32) = tile rows
  if (!mbar_wait(done, 0, kTcTimeoutNs)) ok = false;
  tc_fence_after();
  const int r = row0 + warp * 32 + lane;
  for (int c = 0; c < kTcBN / 32; ++c) {
    float v[32];
    tmem_ld_32x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
    const int cc = col0 + c * 32;
    if (!ok || r >= M || cc >= N) continue;
    float* crow = C + (size_t)r * ldc + cc;
    if (cc + 32 <= N && vec_ok) {
      float4* c4 = reinterpret_cast<float4*>(crow);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (beta != 0.f) o = c4[q];
        o.x = alpha * v[4 * q] + beta * o.x;
        o.y = alpha * v[4 * q + 1] + beta * o.y;
        o.z = alpha * v[4 * q + 2] + beta * o.z;
        o.w = alpha * v[4 * q + 3] + beta * o.w;
        c4[q] = o;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q)
        if (cc + q < N) crow[q] = alpha * v[q] + (beta != 0.f ? beta * crow[q] : 0.f);
    }
  }
  if (!ok && lane == 0) atomicOr(err, 16);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcBN);
}

// ---------------------------------------------------------------------------
// One 128 x 128 diagonal tile: L = chol(A) in place (lower triangle; the upper
// triangle is left as it was) and its inverse L^-1 (lower, zeros above) into a
// separate 128 x 128 buffer.  FP32, one block of 256 threads, right-looking over
// four 32-column blocks: one warp factors the 32 x 32 diagonal block and
// inverts it in registers (row per lane for the factor, column per lane for the
// inverse; pivots through rsqrt, so no divisions); the rows below become
// T_b = A_b L_bb^-T, a product with that inverse; the trailing part takes the
// rank-32 update.  The off-diagonal blocks of L^-1 follow by distance:
// X_ij = -X_ii sum_k L_ik X_kj.  The products use 4-wide and 4 x 4 register
// tiles (independent FMA chains).  A pivot <= 0 (not positive definite in FP32)
// sets err bit 32 and is replaced by a tiny positive value, keeping outputs finite.
// ---------------------------------------------------------------------------
constexpr int kPt = 128;
constexpr int kPtLd = kPt + 1;
constexpr int kPtThreads = 256;  // the warp-0 register work needs > 128 registers
constexpr int kPtSmem = (2 * kPt * kPtLd + 3 * 32 * 33 + kPt) * 4;

// One pivot step of the 32 x 32 register factorisation (lane = row): pivot K,
// scale column K, rank-1 update of the columns after K.  Template recursion keeps
// every register index static.  dinv[K] receives 1 / L_KK.
template <int K>
__device__ __forceinline__ void chol32_step(float (&R)[32], int lane, bool& bad, float* dinv) {
  float dkk = __shfl_sync(0xffffffffu, R[K], K);
  if (!(dkk > 0.f)) {
    bad = true;
    dkk = 1e-30f;
  }
  const float rs = rsqrtf(dkk);
  const float lik = lane == K ? dkk * rs : (lane > K ? R[K] * rs : 0.f);
  if (lane == 0) dinv[K] = rs;
  R[K] = lik;
  // every L_jK first (independent shuffles issued back to back), then the updates
  float lj[32];
#pragma unroll
  for (int j = K + 1; j < 32; ++j) lj[j] = __shfl_sync(0xffffffffu, lik, j);
#pragma unroll
  for (int j = K + 1; j < 32; ++j)
    if (lane >= j) R[j] -= lik * lj[j];
  if constexpr (K + 1 < 32) chol32_step<K + 1>(R, lane, bad, dinv);
}

// Row I of column `lane` of L^-1 (forward substitution), L read from shared
// memory (every lane reads the same entries: broadcasts).
template <int I>
__device__ __forceinline__ void inv32_step(float (&Xc)[32], int lane, const float* Lb, const float* dinv) {
  float acc = I == lane ? 1.f : 0.f;
#pragma unroll
  for (int l = 0; l < I; ++l) acc -= Lb[I * kPtLd + l] * Xc[l];
  Xc[I] = acc * dinv[I];
  if constexpr (I + 1 < 32) inv32_step<I + 1>(Xc, lane, Lb, dinv);
}

// row index ti >= tj of the t-th 4 x 4 tile of a lower-triangular tile grid
__device__ __forceinline__ void tri_decode(int t, int& ti, int& tj) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(kPtThreads) k_potrf_tile(float* __restrict__ A, long long lda,
                                                          float* __restrict__ Linv, int* err) {
  extern __shared__ float pt_smem[];
  float* T = pt_smem;               // [128][129] factor
  float* X = T + kPt * kPtLd;       // [128][129] inverse
  float* Sc = X + kPt * kPtLd;      // [3][32][33] scratch
  float* Dv = Sc + 3 * 32 * 33;     // [128] 1 / L_ii
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // A: 16-byte aligned rows (lda a multiple of 4)
#pragma unroll 4
  for (int q = tid; q < kPt * (kPt / 4); q += kPtThreads) {
    const int r = q >> 5, c = 4 * (q & 31);
    const float4 v = *reinterpret_cast<const float4*>(A + (size_t)r * lda + c);
    float* t = T + r * kPtLd + c;
    t[0] = c <= r ? v.x : 0.f;
    t[1] = c + 1 <= r ? v.y : 0.f;
    t[2] = c + 2 <= r ? v.z : 0.f;
    t[3] = c + 3 <= r ? v.w : 0.f;
    float* x = X + r * kPtLd + c;
    x[0] = x[1] = x[2] = x[3] = 0.f;
  }
  __syncthreads();
  bool bad = false;
  for (int b = 0; b < 4; ++b) {
    const int c0 = 32 * b;
    if (warp == 0) {
      float R[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) R[j] = j <= lane ? T[(c0 + lane) * kPtLd + c0 + j] : 0.f;
      chol32_step<0>(R, lane, bad, Dv + c0);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j <= lane) T[(c0 + lane) * kPtLd + c0 + j] = R[j];
      __syncwarp();
      float Xc[32];
      inv32_step<0>(Xc, lane, T + c0 * kPtLd + c0, Dv + c0);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j >= lane) X[(c0 + j) * kPtLd + c0 + lane] = Xc[j];
    }
    __syncthreads();
    const int r0 = c0 + 32, nr = kPt - r0;
    if (nr > 0) {
      // rows below: T[r][c0 + j] = sum_l A[r][c0 + l] X_bb[j][l]; items = (row, 4 columns)
      float out[3][4];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int it = tid + kPtThreads * m;
#pragma unroll
        for (int i = 0; i < 4; ++i) out[m][i] = 0.f;
        if (it < nr * 8) {
          const int r = r0 + (it >> 3), j0 = 4 * (it & 7);
          const float* ar = T + r * kPtLd + c0;
          const float* x0 = X + (c0 + j0) * kPtLd + c0;
#pragma unroll 8
          for (int l = 0; l < 32; ++l) {
            const float a = ar[l];
            out[m][0] += a * x0[l];
            out[m][1] += a * x0[kPtLd + l];
            out[m][2] += a * x0[2 * kPtLd + l];
            out[m][3] += a * x0[3 * kPtLd + l];
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int it = tid + kPtThreads * m;
        if (it < nr * 8) {
          float* t = T + (r0 + (it >> 3)) * kPtLd + c0 + 4 * (it & 7);
#pragma unroll
          for (int i = 0; i < 4; ++i) t[i] = out[m][i];
        }
      }
      __syncthreads();
      // trailing rank-32 update of the lower triangle, 4 x 4 register tiles
      const int nt = nr / 4, ntiles = nt * (nt + 1) / 2;
      for (int t = tid; t < ntiles; t += kPtThreads) {
        int ti, tj;
        tri_decode(t, ti, tj);
        const float* a0 = T + (r0 + 4 * ti) * kPtLd + c0;
        const float* b0 = T + (r0 + 4 * tj) * kPtLd + c0;
        float acc[4][4] = {};
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          float av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            av[i] = a0[i * kPtLd + l];
            bv[i] = b0[i * kPtLd + l];
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (ti != tj || j <= i) T[(r0 + 4 * ti + i) * kPtLd + r0 + 4 * tj + j] -= acc[i][j];
      }
      __syncthreads();
    }
  }
  // off-diagonal blocks of the inverse, by distance d = bi - bj, 4 x 4 register tiles
  for (int d = 1; d < 4; ++d) {
    const int nb = 4 - d;
    for (int it = tid; it < nb * 64; it += kPtThreads) {
      const int blk = it >> 6, e = it & 63, r = 4 * (e >> 3), c = 4 * (e & 7);
      const int bi = d + blk, bj = bi - d;
      float acc[4][4] = {};
      for (int l = 32 * bj; l < 32 * bi; ++l) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = T[(32 * bi + r + i) * kPtLd + l];
          bv[i] = X[l * kPtLd + 32 * bj + c + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Sc[blk * 32 * 33 + (r + i) * 33 + c + j] = acc[i][j];
    }
    __syncthreads();
    for (int it = tid; it < nb * 64; it += kPtThreads) {
      const int blk = it >> 6, e = it & 63, r = 4 * (e >> 3), c = 4 * (e & 7);
      const int bi = d + blk, bj = bi - d;
      float acc[4][4] = {};
      for (int l = 0; l < r + 4; ++l) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = X[(32 * bi + r + i) * kPtLd + 32 * bi + l];  // zero above the diagonal
          bv[i] = Sc[blk * 32 * 33 + l * 33 + c + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) X[(32 * bi + r + i) * kPtLd + 32 * bj + c + j] = -acc[i][j];
    }
    __syncthreads();
  }
#pragma unroll 4
  for (int q = tid; q < kPt * (kPt / 4); q += kPtThreads) {
    const int r = q >> 5, c = 4 * (q & 31);
    const float* t = T + r * kPtLd + c;
    const float* x = X + r * kPtLd + c;
    float* a = A + (size_t)r * lda + c;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (c + i <= r) a[i] = t[i];
    float4 o = make_float4(c <= r ? x[0] : 0.f, c + 1 <= r ? x[1] : 0.f, c + 2 <= r ? x[2] : 0.f,
                           c + 3 <= r ? x[3] : 0.f);
    *reinterpret_cast<float4*>(Linv + (size_t)r * kPt + c) = o;
  }
  if (bad) atomicOr(err, 32);
}

constexpr int kPanelTiles = 8;  // 1024-column panels: trailing updates with K = 1024

// Blocked Cholesky of the lower triangle of A (np x np, np a multiple of 128,
// lda a multiple of 4, 16-byte aligned), in place; Linv receives the inverses of
// the np/128 diagonal tiles.  Rows/columns past the problem size must hold the
// identity.  Returns the number of kernels launched in *launches.
cudaError_t dense_cholesky_tc(float* A, long long lda, int np, float* Linv, int* err, cudaStream_t s,
                              long long* launches) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_potrf_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kPtSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int T = np / kPt;
  long long nl = 0;
  // Look-ahead of depth one: after panel p is factored (A_p), the trailing update
  // is split into the next panel's columns (B_p, right behind A_p, so that panel
  // p + 1 is factored next) and the columns beyond (C_p), which runs while panel
  // p + 1 is factored.  A and B run on a high-priority stream, C on a low-priority
  // one, so the block scheduler gives the factorisation's small launches the SMs
  // that C's tiles free.  B_{p+1} touches columns C_p also updates and waits for
  // it; C_{p+1} follows C_p and waits for A_{p+1}.  Both streams fork from and
  // join the caller's stream s.
  const cudaStream_t s_in = s;
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_a = nullptr, ev_c = nullptr;
  int prio_lo = 0, prio_hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio_lo);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_c, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev_a, s_in);  // fork: the inputs are ready on s_in
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_a, 0);
  bool c_pending = false;  // a C update was enqueued on s2 since s last waited for it
  for (int p0 = 0; p0 < T && e == cudaSuccess; p0 += kPanelTiles) {
    const int p1 = min(T, p0 + kPanelTiles);
    // A_p: the panel's diagonal tiles, the tiles below them, the in-panel updates
    for (int j = p0; j < p1 && e == cudaSuccess; ++j) {
      float* Ajj = A + (size_t)j * kPt * lda + (size_t)j * kPt;
      float* Lj = Linv + (size_t)j * kPt * kPt;
      k_potrf_tile<<<1, kPtThreads, kPtSmem, s>>>(Ajj, lda, Lj, err);
      ++nl;
      e = cudaGetLastError();
      const int below = T - j - 1;
      if (e != cudaSuccess || below <= 0) continue;
      float* Aij = Ajj + (size_t)kPt * lda;
      // L_ij = A_ij L_jj^-T (each block reads all of its rows before writing them)
      e = tc_gemm_nt(Aij, lda, Lj, kPt, Aij, lda, below * kPt, kPt, kPt, 1.f, 0.f, false, err, s);
      ++nl;
      const int wcols = p1 - j - 1;
      if (e == cudaSuccess && wcols > 0) {
        e = tc_gemm_nt(Aij, lda, Aij, lda, Aij + kPt, lda, below * kPt, wcols * kPt, kPt, -1.f, 1.f, true, err, s);
        ++nl;
      }
    }
    const int rest = T - p1;
    if (e != cudaSuccess || rest <= 0) continue;
    const int p2 = min(T, p1 + kPanelTiles);
    const float* Lp = A + (size_t)p1 * kPt * lda + (size_t)p0 * kPt;  // rows p1.., panel p's columns
    const int K = (p1 - p0) * kPt;
    // C_p: columns p2.. (rows p2..), on s2 once A_p is done
    if (p2 < T) {
      e = cudaEventRecord(ev_a, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, ev_a, 0);
      const float* Lq = Lp + (size_t)(p2 - p1) * kPt * lda;
      float* Cq = A + (size_t)p2 * kPt * lda + (size_t)p2 * kPt;
      if (e == cudaSuccess)
        e = tc_gemm_nt(Lq, lda, Lq, lda, Cq, lda, (T - p2) * kPt, (T - p2) * kPt, K, -1.f, 1.f, true, err, s2);
      ++nl;
    }
    // B_p: columns p1..p2 (rows p1..), on s, after the previous C (same columns)
    if (e == cudaSuccess && c_pending) e = cudaStreamWaitEvent(s, ev_c, 0);
    c_pending = false;
    if (e == cudaSuccess) {
      float* Cb = A + (size_t)p1 * kPt * lda + (size_t)p1 * kPt;
      e = tc_gemm_nt(Lp, lda, Lp, lda, Cb, lda, rest * kPt, (p2 - p1) * kPt, K, -1.f, 1.f, true, err, s);
      ++nl;
    }
    if (e == cudaSuccess && p2 < T) {
      e = cudaEventRecord(ev_c, s2);
      c_pending = true;
    }
  }
  // join: the caller's stream waits for the last C update and for the factorisation
  if (e == cudaSuccess && c_pending) e = cudaStreamWaitEvent(s, ev_c, 0);
  if (e == cudaSuccess) e = cudaEventRecord(ev_a, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev_a, 0);
  if (ev_a) cudaEventDestroy(ev_a);
  if (ev_c) cudaEventDestroy(ev_c);
  if (s2) cudaStreamDestroy(s2);  // released once its work completes
  if (s != s_in) cudaStreamDestroy(s);
  if (launches) *launches += nl;
  return e;
}

// ---------------------------------------------------------------------------
// Triangular solves with the blocked factor, L y = r (forward) and L^T x = y
// (backward), each in one cooperative launch.  Block b takes tiles b, b + G, ...
// in solve order; tile i waits for the tiles it depends on (a flag per tile,
// set with release semantics after the tile's values are stored), accumulates
// r_i - sum_j L_ij y_j as they arrive, and finishes with the diagonal tile's
// inverse: y_i = L_ii^-1 acc.  Dependencies only point to tiles earlier in
// every block's order, so with all blocks resident the solve cannot deadlock;
// waits are bounded (err bit 1 on timeout).
// ---------------------------------------------------------------------------
constexpr int kTrThreads = 256;

__device__ __forceinline__ bool wait_flag(const unsigned* flag, unsigned epoch, long long timeout_ns) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
  if (v == epoch) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v == epoch) return true;
    if ((long long)(globaltimer_ns() - t0) > timeout_ns) return false;
  }
}

__device__ __forceinline__ void set_flag(unsigned* flag, unsigned epoch) {
  __threadfence();
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(epoch) : "memory");
}

// Forward (!BACK): L y = r.  Backward (BACK): L^T x = y.  rhs, out: np vectors
// (np = 128 T, 16-byte aligned); L: np x np row-major lower factor (ld); Linv:
// the T diagonal-tile inverses; flags: T words, epoch unique per call.
//
// Block b takes the tile rows b, b + G, ... in solve order.  Within a tile row,
// warp w owns tile rows [16 w, 16 w + 16) and lane l the float4 column chunk l,
// so every load instruction reads whole 512-byte rows.  Forward: each lane keeps
// 16 row partials over its 4 columns; backward (transposed tiles): 4 column
// partials over the warp's 16 rows.  The dependency tiles stream through
// registers one tile ahead of the arithmetic, each warp polls the dependencies'
// flags itself (no block barrier per dependency), and the diagonal inverse is
// copied into shared memory at the start of the row.  Partials are reduced
// across lanes (forward) or warps (backward) once per tile row.
template <bool BACK>
__global__ void __launch_bounds__(kTrThreads) k_trsv_tiles(const float* __restrict__ L, long long ld,
                                                           const float* __restrict__ Linv, const float* rhs,
                                                           float* out, int T, unsigned* flags, unsigned epoch,
                                                           long long timeout_ns, int* err) {
  extern __shared__ __align__(16) float trsv_dyn[];
  float* inv = trsv_dyn;                          // [kPt * kPt] the diagonal tile's inverse (dynamic)
  __shared__ __align__(16) float sv[kPt];         // r_i - sum_j (...) for the tile row
  __shared__ float red[8][kPt];                   // backward: per-warp column partials
  __shared__ volatile int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = blockIdx.x; k < T && !bad; k += gridDim.x) {
    const int i = BACK ? T - 1 - k : k;
    // the diagonal inverse, asynchronously into shared memory (16 x 16 bytes per thread)
    {
      const float* src = Linv + (size_t)i * kPt * kPt;
#pragma unroll
      for (int u = 0; u < (kPt * kPt) / (4 * kTrThreads); ++u) {
        const int e = 4 * (tid + u * kTrThreads);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(inv + e);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + e) : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int jn = BACK ? T - 1 - i : i;  // number of dependencies
    // tile of dependency d: forward L_ij (j = d), backward L_ji (j = T - 1 - d), both
    // read as 16 rows x one float4 column chunk per lane
    auto tile_ptr = [&](int d) -> const float* {
      const int j = BACK ? T - 1 - d : d;
      return BACK ? L + (size_t)j * kPt * ld + (size_t)i * kPt : L + (size_t)i * kPt * ld + (size_t)j * kPt;
    };
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.f;
    float4 cur[16];
    if (jn > 0) {
      const float* t = tile_ptr(0) + (size_t)(16 * warp) * ld + 4 * lane;
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) cur[rr] = __ldcs(reinterpret_cast<const float4*>(t + (size_t)rr * ld));
    }
    for (int d = 0; d < jn; ++d) {
      float4 nxt[16];
      if (d + 1 < jn) {
        const float* t = tile_ptr(d + 1) + (size_t)(16 * warp) * ld + 4 * lane;
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) nxt[rr] = __ldcs(reinterpret_cast<const float4*>(t + (size_t)rr * ld));
      }
      const int j = BACK ? T - 1 - d : d;
      // every lane waits for the dependency itself (acquire), bounded
      if (!wait_flag(&flags[j], epoch, timeout_ns)) bad = 1;
      if (bad) break;
      const float* y = out + (size_t)j * kPt;
      if (!BACK) {
        const float4 v = *reinterpret_cast<const float4*>(y + 4 * lane);
#pragma unroll
        for (int rr = 0; rr < 16; ++rr)
          acc[rr] = fmaf(cur[rr].x, v.x, fmaf(cur[rr].y, v.y, fmaf(cur[rr].z, v.z, fmaf(cur[rr].w, v.w, acc[rr]))));
      } else {
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const float vr = y[16 * warp + rr];
          acc[0] = fmaf(cur[rr].x, vr, acc[0]);
          acc[1] = fmaf(cur[rr].y, vr, acc[1]);
          acc[2] = fmaf(cur[rr].z, vr, acc[2]);
          acc[3] = fmaf(cur[rr].w, vr, acc[3]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) cur[rr] = nxt[rr];
    }
    // s = r_i - the sum, for the tile row
    if (!BACK) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const float t = warp_sum(acc[rr]);
        if (lane == 0) sv[16 * warp + rr] = rhs[(size_t)i * kPt + 16 * warp + rr] - t;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) red[warp][4 * lane + c] = acc[c];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (bad) break;
    if (BACK && tid < kPt) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += red[w][tid];
      sv[tid] = rhs[(size_t)i * kPt + tid] - t;
    }
    if (BACK) __syncthreads();
    // out_i = Linv_i s (forward) or Linv_i^T s (backward), from shared memory
    if (!BACK) {
      const float4 v = *reinterpret_cast<const float4*>(sv + 4 * lane);
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const float4 m = *reinterpret_cast<const float4*>(inv + (16 * warp + rr) * kPt + 4 * lane);
        const float t = warp_sum(m.x * v.x + m.y * v.y + m.z * v.z + m.w * v.w);
        if (lane == 0) out[(size_t)i * kPt + 16 * warp + rr] = t;
      }
    } else {
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const float4 m = *reinterpret_cast<const float4*>(inv + (16 * warp + rr) * kPt + 4 * lane);
        const float vr = sv[16 * warp + rr];
        o[0] = fmaf(m.x, vr, o[0]);
        o[1] = fmaf(m.y, vr, o[1]);
        o[2] = fmaf(m.z, vr, o[2]);
        o[3] = fmaf(m.w, vr, o[3]);
      }
      __syncthreads();  // red is rewritten
#pragma unroll
      for (int c = 0; c < 4; ++c) red[warp][4 * lane + c] = o[c];
      __syncthreads();
      if (tid < kPt) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w][tid];
        out[(size_t)i * kPt + tid] = t;
      }
    }
    __syncthreads();
    if (tid == 0) set_flag(&flags[i], epoch);
  }
  if (tid == 0 && bad) atomicOr(err, 1);
}

cudaError_t dense_trsv(bool back, const float* L, long long ld, const float* Linv, const float* rhs, float* out,
                       int T, unsigned* flags, unsigned epoch, int* err, int num_sms, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  constexpr int kTrSmem = kPt * kPt * 4;  // the diagonal inverse
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_trsv_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_trsv_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int grid = std::min(T, num_sms);
  long long timeout = 1000000000LL;
  void* args[] = {(void*)&L, (void*)&ld, (void*)&Linv, (void*)&rhs, (void*)&out, (void*)&T, (void*)&flags,
                  (void*)&epoch, (void*)&timeout, (void*)&err};
  const void* fn = back ? reinterpret_cast<const void*>(&k_trsv_tiles<true>)
                        : reinterpret_cast<const void*>(&k_trsv_tiles<false>);
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTrThreads), args, kTrSmem, s);
}

// ---------------------------------------------------------------------------
// Dense preconditioned CG on S^ x = b with M = (L L^T)^-1 from the tensor-core
// factor.  The factor carries TF32-level error, so it is used as a
// preconditioner and CG recovers the FP32 solution; when the damped system is
// nearly singular the iteration count grows rather than the accuracy dropping.
// Dots in FP64 with a fixed-order two-level reduction; alpha, beta on the
// device; one host readback per iteration for the stopping test.
// ---------------------------------------------------------------------------
constexpr int kDotBlocks = 256;

// padded work matrix: rows/columns n..np the identity, diagonal of the leading
// block shifted by `shift` (a retry after a non-positive TF32 pivot)
__global__ void k_pad_shift(float* A, long long ld, int n, int np, float shift) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)np * np;
       q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / np), c = (int)(q % np);
    if (r >= n || c >= n) A[(size_t)r * ld + c] = r == c ? 1.f : 0.f;
    else if (r == c && shift != 0.f) A[(size_t)r * ld + c] += shift;
  }
}

// out[blockIdx] = partial sums of a.b over a grid-stride range (fixed order)
__global__ void k_dot_partial(const float* __restrict__ a, const float* __restrict__ b, int n, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_dot_final(const double* part, int np, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// y = S x over rows [0, n), S row-major with ld (one warp per row)
__global__ void k_gemv_rows(const float* __restrict__ S, long long ld, const float* __restrict__ x, float* y,
                            int n) {
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += (gridDim.x * blockDim.x) >> 5) {
    const float* row = S + (size_t)r * ld;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int c = lane;
    for (; c + 96 < n; c += 128) {
      a0 += row[c] * x[c];
      a1 += row[c + 32] * x[c + 32];
      a2 += row[c + 64] * x[c + 64];
      a3 += row[c + 96] * x[c + 96];
    }
    for (; c < n; c += 32) a0 += row[c] * x[c];
    const float t = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) y[r] = t;
  }
}

// sc: [0] rz, [1] pq, [2] rr, [3] rz_new, [4] alpha, [5] beta
__global__ void k_cg_alpha(double* sc) {
  sc[4] = sc[1] > 0.0 ? sc[0] / sc[1] : 0.0;
}
__global__ void k_cg_beta(double* sc) {
  sc[5] = sc[0] != 0.0 ? sc[3] / sc[0] : 0.0;
  sc[0] = sc[3];
}
// x += alpha p; r -= alpha q
__global__ void k_cg_xr(float* x, float* r, const float* p, const float* q, const double* sc, int n) {
  const float al = (float)sc[4];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    r[i] -= al * q[i];
  }
}
// p = z + beta p (first: p = z)
__global__ void k_cg_p(float* p, const float* z, const double* sc, int n, int first) {
  const float be = first ? 0.f : (float)sc[5];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = z[i] + be * p[i];
}

__global__ void k_scale_vec(int n, const float* __restrict__ a, const float* __restrict__ d, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] * d[i];
}
cudaError_t launch_scale_vec(int n, const float* a, const float* d, float* out, cudaStream_t s) {
  if (n > 0) k_scale_vec<<<std::min((n + 255) / 256, 1024), 256, 0, s>>>(n, a, d, out);
  return cudaGetLastError();
}
__global__ void k_set_pcg_info(Scalars* sc, int iters, double rel, int* err, int errbits) {
  sc->pcg_iters = iters;
  sc->pcg_rel_res = rel;
  if (errbits) atomicOr(err, errbits);
}
cudaError_t launch_set_pcg_info(Scalars* sc, int iters, double rel, int* err, int errbits, cudaStream_t s) {
  k_set_pcg_info<<<1, 1, 0, s>>>(sc, iters, rel, err, errbits);
  return cudaGetLastError();
}

cudaError_t dense_dot(const float* a, const float* b, int n, double* part, double* out, cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, 256, 0, s>>>(a, b, n, part);
  k_dot_final<<<1, 256, 0, s>>>(part, kDotBlocks, out);
  return cudaGetLastError();
}

// Factor S^ (n x n, ld_s) into the padded work matrix and solve S^ x = b.
cudaError_t dense_spd_solve(const DenseWork& w, const float* S, long long ld_s, int n, const float* b, float* x,
                            double tol, int max_iters, int num_sms, cudaStream_t s, DenseResult* res,
                            bool reuse_factor) {
  const int np = (n + kPt - 1) / kPt * kPt, T = np / kPt;
  res->iters = 0;
  res->rel_res = 0.0;
  if (reuse_factor) {
    res->flags &= 32;  // the factor of the previous call stands, with its shift and pivot flag
  } else {
    res->flags = 0;
    res->shift = 0.0;
  }
  long long nl = 0;
  cudaError_t e = cudaSuccess;
  for (int attempt = 0; attempt < 3 && !reuse_factor; ++attempt) {
    const float shift = attempt == 0 ? 0.f : (attempt == 1 ? 1e-3f : 1e-1f);
    e = cudaMemsetAsync(w.err, 0, sizeof(int), s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(w.A, sizeof(float) * np, S, sizeof(float) * ld_s, sizeof(float) * n, n,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const long long tot = (long long)np * np;
    k_pad_shift<<<(unsigned)std::min<long long>((tot + 255) / 256, 65535), 256, 0, s>>>(w.A, np, n, np, shift);
    ++nl;
    e = dense_cholesky_tc(w.A, np, np, w.Linv, w.err, s, &nl);
    if (e != cudaSuccess) return e;
    int h = 0;
    e = cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    res->flags = h;
    res->shift = shift;
    if (!(h & 32)) break;
  }
  if (res->flags & 16) {
    res->launches += nl;
    return cudaSuccess;  // pipeline timeout: reported through flags
  }
  // vectors live in padded length np; entries n..np stay zero
  float *r = w.vec, *z = w.vec + np, *p = w.vec + 2 * (size_t)np, *q = w.vec + 3 * (size_t)np;
  e = cudaMemsetAsync(w.vec, 0, sizeof(float) * 4 * (size_t)np, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, sizeof(float) * n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r, b, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  const int vgrid = std::min((np + 255) / 256, 4 * num_sms);
  auto precond = [&](const float* in, float* outv) -> cudaError_t {
    // z = L^-T (L^-1 in): forward into q as scratch, then backward
    cudaError_t e2 = dense_trsv(false, w.A, np, w.Linv, in, q, T, w.flags, ++*w.epoch, w.err, num_sms, s);
    if (e2 == cudaSuccess) e2 = dense_trsv(true, w.A, np, w.Linv, q, outv, T, w.flags, ++*w.epoch, w.err, num_sms, s);
    nl += 2;
    return e2;
  };
  double* sc = w.scal;
  double h[3] = {0, 0, 0};
  e = dense_dot(b, b, n, w.part, sc + 2, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  nl += 2;
  const double bnorm = std::sqrt(h[0]);
  if (!(bnorm > 0.0)) {
    res->launches += nl;
    return cudaSuccess;
  }
  e = precond(r, z);
  if (e == cudaSuccess) e = dense_dot(r, z, n, w.part, sc + 0, s);
  if (e == cudaSuccess) k_cg_p<<<vgrid, 256, 0, s>>>(p, z, sc, np, 1);
  nl += 3;
  int it = 0;
  double rr = h[0];
  while (e == cudaSuccess && it < max_iters) {
    k_gemv_rows<<<std::min((n + 7) / 8, 32 * num_sms), 256, 0, s>>>(S, ld_s, p, q, n);
    e = dense_dot(p, q, n, w.part, sc + 1, s);
    k_cg_alpha<<<1, 1, 0, s>>>(sc);
    k_cg_xr<<<vgrid, 256, 0, s>>>(x, r, p, q, sc, n);
    if (e == cudaSuccess) e = dense_dot(r, r, n, w.part, sc + 2, s);
    nl += 7;
    ++it;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, sc, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    rr = h[2];
    if (!(h[1] > 0.0) || !std::isfinite(rr)) {
      res->flags |= 2;
      break;
    }
    if (std::sqrt(rr) <= tol * bnorm) break;
    e = precond(r, z);
    if (e == cudaSuccess) e = dense_dot(r, z, n, w.part, sc + 3, s);
    k_cg_beta<<<1, 1, 0, s>>>(sc);
    k_cg_p<<<vgrid, 256, 0, s>>>(p, z, sc, np, 0);
    nl += 4;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  res->iters = it;
  res->rel_res = std::sqrt(rr) / bnorm;
  res->launches += nl;
  return e;
}

// ---------------------------------------------------------------------------
// host: tensor maps and launches
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// rows x cols FP32, row stride ld (elements, multiple of 4; base 16-byte aligned), box {32, box_rows}
static cudaError_t make_map(CUtensorMap* m, const float* ptr, long long rows, long long cols, long long ld,
                            int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  if ((ld & 3) || (reinterpret_cast<uintptr_t>(ptr) & 15)) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_gemm_nt(const float* A, long long lda, const float* B, long long ldb, float* C, long long ldc,
                       int M, int N, int K, float alpha, float beta, bool lower_only, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ma, mb;
  cudaError_t e = make_map(&ma, A, M, K, lda, kTcBM);
  if (e == cudaSuccess) e = make_map(&mb, B, N, K, ldb, kTcBN);
  if (e != cudaSuccess) return e;
  const int tiles_m = (M + kTcBM - 1) / kTcBM, tiles_n = (N + kTcBN - 1) / kTcBN;
  const int vec_ok = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
  k_tc_gemm_nt<<<tiles_m * tiles_n, kTcThreads, kTcSmem, s>>>(ma, mb, C, ldc, M, N, K, alpha, beta, tiles_n,
                                                             lower_only ? 1 : 0, vec_ok, err);
  return cudaGetLastError();
}

}  // namespace bab

// ---------------------------------------------------------------------------
// C ABI: the dense kernels on their own
// ---------------------------------------------------------------------------
namespace {

void dense_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  bab::set_last_error_message(buf);
}

__global__ void k_pad_identity(float* A, long long ld, int n, int np) {
  // rows and columns n..np of the padded matrix: identity
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long tot = (long long)np * (np - n);
  if (q >= tot) return;
  const int r = (int)(q / (np - n)), c = n + (int)(q % (np - n));
  A[(size_t)r * ld + c] = r == c ? 1.f : 0.f;       // columns n..np of every row
  A[(size_t)c * ld + r] = r == c ? 1.f : 0.f;       // rows n..np of every column
}

__global__ void k_zero_upper(float* A, long long ld, int n) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  if (c > r) A[(size_t)r * ld + c] = 0.f;
}

}  // namespace

extern "C" {

ba_status ba_tc_gemm_nt(void* stream, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float beta, float* C, int64_t ldc) {
  if (M < 0 || N < 0 || K < 0 || M >= (1LL << 31) || N >= (1LL << 31) || K >= (1LL << 31) || !A || !B || !C ||
      lda < K || ldb < K || ldc < N || (lda & 3) || (ldb & 3) ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) {
    dense_error("ba_tc_gemm_nt: invalid sizes, strides or pointers (lda, ldb multiples of 4, A, B 16-byte aligned)");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = bab::tc_gemm_nt(A, lda, B, ldb, C, ldc, (int)M, (int)N, (int)K, alpha, beta, false, err, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (err) cudaFreeAsync(err, s);
  if (e != cudaSuccess) {
    dense_error("ba_tc_gemm_nt: %s", cudaGetErrorString(e));
    return BA_ERR_CUDA;
  }
  if (h & 16) {
    dense_error("ba_tc_gemm_nt: pipeline wait timed out");
    return BA_ERR_TIMEOUT;
  }
  return BA_OK;
}

ba_status ba_dense_cholesky(void* stream, int64_t n, const float* A, int64_t lda, float* L, int64_t ldl,
                            int* flags) {
  if (n < 0 || n > 65536 || !A || !L || lda < n || ldl < n) {
    dense_error("ba_dense_cholesky: invalid size or pointers");
    return BA_ERR_INVALID_ARG;
  }
  if (flags) *flags = 0;
  if (n == 0) return BA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int np = (int)((n + 127) / 128 * 128);
  float *Ap = nullptr, *Li = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync(&Ap, sizeof(float) * (size_t)np * np, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&Li, sizeof(float) * (size_t)np * 128, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(Ap, sizeof(float) * np, A, sizeof(float) * lda, sizeof(float) * n, n, cudaMemcpyDefault, s);
  if (e == cudaSuccess && np > n) {
    const long long tot = (long long)np * (np - n);
    k_pad_identity<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Ap, np, (int)n, np);
    e = cudaGetLastError();
  }
  long long nl = 0;
  if (e == cudaSuccess) e = bab::dense_cholesky_tc(Ap, np, np, Li, err, s, &nl);
  if (e == cudaSuccess) {
    const long long tot = (long long)n * n;
    k_zero_upper<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Ap, np, (int)n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(L, sizeof(float) * ldl, Ap, sizeof(float) * np, sizeof(float) * n, n, cudaMemcpyDefault, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (Ap) cudaFreeAsync(Ap, s);
  if (Li) cudaFreeAsync(Li, s);
  if (err) cudaFreeAsync(err, s);
  if (e != cudaSuccess) {
    dense_error("ba_dense_cholesky: %s", cudaGetErrorString(e));
    return BA_ERR_CUDA;
  }
  if (flags) *flags = h;
  if (h & 16) {
    dense_error("ba_dense_cholesky: pipeline wait timed out");
    return BA_ERR_TIMEOUT;
  }
  if (h & 32) {
    dense_error("ba_dense_cholesky: not positive definite in FP32/TF32");
    return BA_ERR_NONFINITE;
  }
  return BA_OK;
}

// Diagnostic of the bounded waits every cross-block kernel of this library uses:
// one block waits, with the given limit, on a device flag that nothing sets.
__global__ void k_wait_selftest(const unsigned* flag, long long timeout_ns, int* out) {
  if (threadIdx.x == 0) *out = bab::wait_flag(flag, 1u, timeout_ns) ? 1 : 2;
}

ba_status ba_selftest_wait_timeout(void* stream, double timeout_ms) {
  if (!(timeout_ms > 0.0) || timeout_ms > 5000.0) {
    dense_error("ba_selftest_wait_timeout: limit must be in (0, 5000] ms");
    return BA_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* flag = nullptr;
  int* out = nullptr;
  cudaError_t e = cudaMallocAsync(&flag, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&out, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(flag, (long long)(timeout_ms * 1e6), out);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, out, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (flag) cudaFreeAsync(flag, s);
  if (out) cudaFreeAsync(out, s);
  if (e != cudaSuccess) {
    dense_error("ba_selftest_wait_timeout: %s", cudaGetErrorString(e));
    return BA_ERR_CUDA;
  }
  if (h == 2) {
    dense_error("ba_selftest_wait_timeout: the wait gave up after %.3f ms, as intended", timeout_ms);
    return BA_ERR_TIMEOUT;
  }
  dense_error("ba_selftest_wait_timeout: unexpected outcome %d", h);
  return BA_ERR_STATE;
}

}  // extern "C"
