// gemm.h -- the tensor-core BF16 GEMM of the TTGT contractions (gemm.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ttc {

// Why (A, lda, B, ldb, M, N, K) cannot run on gemm_bf16, or null if it can:
// M, N >= 1, K >= 0 (K = 0 writes beta * C), extents below 2^31, row pitches
// >= K and multiples of 8 elements (16 bytes), operands 16-byte aligned.
const char* gemm_bf16_check(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t N,
                            int64_t K);

// C[rowoff[m] + coloff[n]] (FP32) = alpha * sum_k A[m, k] B[n, k] + beta *
// the same, for m < M, n < N, where A and B are K-major BF16 matrices: row m
// of A and row n of B each hold K consecutive elements, at pitches lda and
// ldb; rowoff (M entries) and coloff (N entries) are device arrays of element
// offsets (a column-major C with leading dimension ldc: rowoff[m] = m,
// coloff[n] = n * ldc).  Asynchronous on s (one persistent launch).  A
// tensor-core wait that gives up sets *err (device memory) to 1 and the
// result is not valid.
cudaError_t gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, const int64_t* rowoff,
                      const int64_t* coloff, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      cudaStream_t s);

}  // namespace ttc
