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

// Tile shapes of gemm_bf16: GEMM_SINGLE / _192 / _128 -- one CTA per 128 x
// 256, 128 x 192 or 128 x 128 output tile; GEMM_PAIR_256 / _192 / _128 --
// a cluster of two CTAs per 256 x 256, 256 x 192 or 256 x 128 tile
// (tensor-core MMAs spanning both SMs); GEMM_AUTO picks by gemm_bf16_pick.
enum GemmVariant : int {
  GEMM_AUTO = 0,
  GEMM_SINGLE = 1,
  GEMM_PAIR_256 = 2,
  GEMM_PAIR_128 = 3,
  GEMM_SINGLE_192 = 4,
  GEMM_SINGLE_128 = 5,
  GEMM_PAIR_192 = 6
};

// The tile shape GEMM_AUTO runs for M x N x K on `sms` SMs of which `pairs`
// CTA pairs are co-resident: the least rounds of tiles weighted by each
// shape's measured cost per tile, plus the exposed last epilogue.
int gemm_bf16_pick(int64_t M, int64_t N, int64_t K, int sms, int pairs);

// C[rowoff[m] + coloff[n]] (FP32) = alpha * sum_k A[m, k] B[n, k] + beta *
// the same, for m < M, n < N, where A and B are K-major BF16 matrices: row m
// of A and row n of B each hold K consecutive elements, at pitches lda and
// ldb; rowoff (M entries) and coloff (N entries) are device arrays of element
// offsets (a column-major C with leading dimension ldc: rowoff[m] = m,
// coloff[n] = n * ldc).  Asynchronous on s (one persistent launch of the
// tile shape `variant`; *used, if not null, receives the shape run: K = 0
// always runs GEMM_SINGLE).  A tensor-core wait that gives up sets *err
// (device memory) to 1 and the result is not valid.
cudaError_t gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, const int64_t* rowoff,
                      const int64_t* coloff, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      int variant, int* used, cudaStream_t s);

}  // namespace ttc
