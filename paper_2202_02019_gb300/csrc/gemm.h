// Internal contraction engine of the ladder library.
//
//   out[n * ldo + m]  (=|+=)  sum_{k < K} A[m][k] * B[n][k]      (m < M, n < N)
//
// Both operands are K-major ("TN"): A is M x K, B is N x K, K contiguous.
// The output is written transposed (M contiguous) so that a warp's lanes,
// which hold consecutive rows m of the accumulator, store coalesced.
// K is split into chunks of `kchunk`; each chunk is accumulated on its own
// (FP32 in TMEM on the mixed path, FP64 on the FP64 path) and added into the
// FP64 output with an atomic add when more than one chunk exists or when
// `atomic` is set (the caller zeroes the output first).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ccl {

struct GemmOp {
  // A: rows a_rows (>= M is not required: rows past a_rows read as zero),
  //    a_cols valid columns (columns past it read as zero), row pitch lda
  //    elements; split-BF16 pieces are a_piece elements apart.
  const void* A = nullptr;
  int64_t lda = 0, a_rows = 0, a_cols = 0, a_piece = 0;
  const void* B = nullptr;
  int64_t ldb = 0, b_rows = 0, b_cols = 0, b_piece = 0;
  int64_t M = 0, N = 0, K = 0;  // K: loop extent, a multiple of 32
  double* out = nullptr;
  int64_t ldo = 0;
  int atomic = 0;
  int64_t kchunk = 0;  // multiple of 32; 0 = whole K in one chunk
  Status* status = nullptr;
  uint64_t timeout_ns = 2000000000ull;
};

// Returns 0 or a negative CC_ERR_* code.
int gemm_mixed(const GemmOp& op, cudaStream_t stream);
int gemm_f64(const GemmOp& op, cudaStream_t stream);

// Launch counter shared by every kernel launch of the library.
void count_launch(int n = 1);

}  // namespace ccl
