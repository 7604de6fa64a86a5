// tc_gemm.cu -- the batched deformation product of the Krylov vectors on the fifth-generation
// tensor cores: C[s][n][m] = sum_{k in split s} A[m][k] B[n][k] with A the (Toeplitz) kernel
// matrix and B the vectors, both float32 and K-major, in TF32 with a three-term split
//   A = A_hi + A_lo, B = B_hi + B_lo,  A_hi = tf32(A) (low 13 mantissa bits zero), A_lo = A - A_hi,
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi  (relative error about 2^-21, float32 accumulation),
// so that the tensor-core product carries float32-class accuracy (Sec. 3.3.1: the deformation
// sum of the film; the Krylov products only, the residual keeps its float64 sum).
//
// One CTA (4 warps) per 128 x 128 output tile and K-split: thread 0 streams the four 128 x 32
// float32 operand tiles of a K step into shared memory with TMA (128-byte swizzle) through a
// 3-stage mbarrier ring; thread 32 issues 4 x 3 tcgen05.mma (kind::tf32, M = N = 128, K = 8)
// per stage into a 128-column TMEM accumulator and frees the stage with tcgen05.commit; after
// the last stage the four warps read their 32 TMEM lanes each (tcgen05.ld 32x32b) and store
// the tile transposed (C[n][m], coalesced along m).  Every wait is bounded: a wait that runs out
// sets *err, and the CTA still releases its TMEM and leaves.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ehl_internal.h"
#include "tc_gemm.h"

namespace ehl {

namespace {

constexpr int BM = 128, BN = 128, BK = 32;       // BK float32 = one 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 4;           // 16 KB (BN == BM)
constexpr int STAGE_BYTES = 4 * TILE_BYTES;       // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 128;
constexpr uint32_t TMEM_COLS = BN;                // float32 accumulator: 128 lanes x BN columns
constexpr long long kSpin = 1ll << 22;            // iterations of a bounded wait
// instruction descriptor: D float32, A and B tf32, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// wait for the phase with the given parity to complete; false if the wait ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle: rows of 128 bytes,
// groups of 8 rows 1024 bytes apart (SBO); the leading offset is not used by this layout
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              float* __restrict__ C, int ldc, size_t split_stride, int M, int Nv, int ktiles_per_split, int ktiles,
              int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* consumed = reinterpret_cast<volatile int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kt0 = blockIdx.z * ktiles_per_split;
  const int kt1 = min(ktiles, kt0 + ktiles_per_split);
  const int nk = max(0, kt1 - kt0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int issued = 0;
  bool ok = true;
  if (threadIdx.x == 0) {
    // producer: the four operand tiles of each K step
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES, u = i / STAGES;
      if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1)) {
        ok = false;
        break;
      }
      unsigned char* st = smem + s * STAGE_BYTES;
      const int kx = (kt0 + i) * BK;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load_2d(st, &ta_hi, &full[s], kx, m0);
      tma_load_2d(st + TILE_BYTES, &ta_lo, &full[s], kx, m0);
      tma_load_2d(st + 2 * TILE_BYTES, &tb_hi, &full[s], kx, n0);
      tma_load_2d(st + 3 * TILE_BYTES, &tb_lo, &full[s], kx, n0);
      issued = i + 1;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: 4 K=8 steps per 128-byte row, three products each
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % STAGES, u = i / STAGES;
      if (!mbar_wait(&full[s], u & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 8; ++k) {
        const uint32_t off = (uint32_t)k * 32u;
        const uint64_t ah = sdesc(base + off), al = sdesc(base + TILE_BYTES + off);
        const uint64_t bh = sdesc(base + 2 * TILE_BYTES + off), bl = sdesc(base + 3 * TILE_BYTES + off);
        mma_tf32(tmem, ah, bh, (i > 0 || k > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, 1u);
        mma_tf32(tmem, al, bh, 1u);
      }
      mma_commit(&empty[s]);
    }
    *consumed = i;
    mma_commit(done);  // arrives once every MMA issued above has completed
  }
  // epilogue: every warp reads its 32 TMEM lanes (rows m) and stores C[n][m]
  const bool got = __syncthreads_and(mbar_wait(done, 0)) != 0;  // CTA-uniform: the TMEM loads are warp-collective
  if (!got) ok = false;
  tc_fence_after();
  float* Cs = C + blockIdx.z * split_stride;
  const int m = m0 + warp * 32 + lane;
  if (got && nk > 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < Nv) Cs[(size_t)n * ldc + m] = v[j];
        }
      }
    }
  } else if (nk == 0 && m < M) {
    for (int j = 0; j < BN; ++j) {
      const int n = n0 + j;
      if (n < Nv) Cs[(size_t)n * ldc + m] = 0.0f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    // copies issued but never consumed (a wait ran out): let them land before the CTA leaves
    for (int i = *consumed; i < issued; ++i) mbar_wait(&full[i % STAGES], (i / STAGES) & 1);
  }
  if (!ok) atomicExch(err, 1);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// hi = x rounded to tf32 (low 13 mantissa bits zero), lo = x - hi (exact in float32)
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7f800000u) != 0x7f800000u) b = (b + 0x1000u) & 0xffffe000u;  // ties away from zero
  hi = __uint_as_float(b);
  lo = x - hi;
}

__global__ void k_tc_split(const double* __restrict__ X, int xstride, int rows, int cols, float* __restrict__ hi,
                           float* __restrict__ lo, int ld) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    float h, l;
    tf32_split((float)X[(size_t)r * xstride + c], h, l);
    hi[(size_t)r * ld + c] = h;
    lo[(size_t)r * ld + c] = l;
  }
  (void)rows;
}

// the Toeplitz kernel matrix A[m][k] = T[|m - k|] as tf32 hi / lo parts
__global__ void k_tc_toeplitz(const double* __restrict__ T, int N, float* __restrict__ hi, float* __restrict__ lo,
                              int ld) {
  const int m = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    float h, l;
    tf32_split((float)T[m > k ? m - k : k - m], h, l);
    hi[(size_t)m * ld + k] = h;
    lo[(size_t)m * ld + k] = l;
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    cudaGetLastError();
  });
  return fn;
}

// a [rows][ld] float32 matrix with `cols` valid columns: 128-row x 32-column boxes, 128-byte swizzle,
// zero fill outside
bool make_map(CUtensorMap* map, const float* base, int rows, int cols, int ld) {
  EncodeTiled enc = encode_fn();
  if (!enc || ((uintptr_t)base % 16) != 0 || (ld % 4) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t elem[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, elem,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_ld(int cols) { return (cols + 3) / 4 * 4; }

cudaError_t tc_gemm_init(TcGemm& g, const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int M,
                         int Nv, int K, int lda, int ldb, float* C, int ldc, int splits) {
  g.M = M;
  g.Nv = Nv;
  g.K = K;
  g.C = C;
  g.ldc = ldc;
  g.ktiles = (K + BK - 1) / BK;
  g.splits = splits < 1 ? 1 : (splits > g.ktiles ? g.ktiles : splits);
  g.per = (g.ktiles + g.splits - 1) / g.splits;
  g.splits = (g.ktiles + g.per - 1) / g.per;
  if (!make_map(&g.a_hi, Ahi, M, K, lda) || !make_map(&g.a_lo, Alo, M, K, lda) || !make_map(&g.b_hi, Bhi, Nv, K, ldb) ||
      !make_map(&g.b_lo, Blo, Nv, K, ldb))
    return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t tc_gemm_run(const TcGemm& g, int* err, cudaStream_t st) {
  const dim3 grid((g.M + BM - 1) / BM, (g.Nv + BN - 1) / BN, g.splits);
  k_tc_gemm<<<grid, 128, SMEM_BYTES, st>>>(g.a_hi, g.a_lo, g.b_hi, g.b_lo, g.C, g.ldc, (size_t)g.Nv * g.ldc, g.M, g.Nv,
                                           g.per, g.ktiles, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tc_split(const double* X, int xstride, int rows, int cols, float* hi, float* lo, int ld, cudaStream_t st) {
  const int bx = (cols + 255) / 256 < 8 ? (cols + 255) / 256 : 8;
  k_tc_split<<<dim3(bx, rows), 256, 0, st>>>(X, xstride, rows, cols, hi, lo, ld);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tc_toeplitz(const double* T, int N, float* hi, float* lo, int ld, cudaStream_t st) {
  const int bx = (N + 255) / 256 < 8 ? (N + 255) / 256 : 8;
  k_tc_toeplitz<<<dim3(bx, N), 256, 0, st>>>(T, N, hi, lo, ld);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ehl
