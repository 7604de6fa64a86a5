// tc_gemm.h -- TF32x3 tensor-core (tcgen05) product of the Krylov vectors with the kernel matrix.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace ehl {

// C[s][n][m] = sum over the K steps of split s of A[m][k] B[n][k] (m < M, n < Nv, k < K): A [M][lda]
// and B [Nv][ldb] float32, K-major, each given as tf32 hi / lo parts (tc_split, tc_toeplitz);
// C [splits][Nv][ldc]; the splits' partial sums are added by the caller.  The operand arrays
// must be 16-byte aligned with lda, ldb multiples of 4 (tc_ld).
struct TcGemm {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  int M = 0, Nv = 0, K = 0, ldc = 0, ktiles = 0, splits = 1, per = 1;
  float* C = nullptr;
};

int tc_ld(int cols);
// tensor maps of the operands (the pointers are fixed for the plan's life) and the kernel's
// shared-memory size; splits: requested K-splits (reduced so that every split has K steps)
cudaError_t tc_gemm_init(TcGemm& g, const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int M,
                         int Nv, int K, int lda, int ldb, float* C, int ldc, int splits);
// err: device int set to 1 if a bounded wait of the kernel ran out (its output is then invalid)
cudaError_t tc_gemm_run(const TcGemm& g, int* err, cudaStream_t st);
// hi / lo tf32 parts of rows x cols float64 values X[r][c] (row stride xstride) into [rows][ld]
cudaError_t tc_split(const double* X, int xstride, int rows, int cols, float* hi, float* lo, int ld, cudaStream_t st);
// hi / lo parts of the symmetric Toeplitz matrix A[m][k] = T[|m - k|], N x N, into [N][ld]
cudaError_t tc_toeplitz(const double* T, int N, float* hi, float* lo, int ld, cudaStream_t st);

}  // namespace ehl
