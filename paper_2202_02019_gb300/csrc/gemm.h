// Internal contraction engine of the ladder library.
//
//   out[n * ldo + m]  (= | +=)  sum_{k < K} A[m][k] * B[n][k]      (m < M, n < N)
//
// Both operands are K-major ("TN"): A is M x K, B is N x K, K contiguous.
// The output is written transposed (M contiguous) so that a warp's lanes,
// which hold consecutive rows m of the accumulator, store coalesced.
//
// Mixed paths (gemm_mixed): split operands (3 BF16 or 2 scaled FP16 pieces), 128 x 128 output
// tiles each computed by one CTA over the whole K, float-float output (float2
// hi/lo) either stored (OUT_FF_STORE) or added to what is there (OUT_FF_ACCUM,
// a plain read-modify-write: tiles are owned by one CTA).  Up to
// GEMM_MAX_PROBLEMS independent problems of the same piece scheme run in one
// persistent launch whose CTAs pull tiles from a device queue; problems of one
// launch must not write overlapping outputs.
// FP64 path (gemm_f64): FP64 operands and output; K may be split into
// chunks that are added with FP64 atomics (OUT_F64_ATOMIC, caller zeroes).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ccl {

enum OutMode { OUT_F64_STORE = 0, OUT_F64_ATOMIC = 1, OUT_FF_STORE = 2, OUT_FF_ACCUM = 3 };

constexpr int GEMM_MAX_PROBLEMS = 64;  // problems per mixed launch (kernel parameter space)

struct GemmOp {
  // A: rows a_rows (rows past it read as zero), a_cols valid columns
  //    (columns past it read as zero), row pitch lda elements; split-BF16
  //    pieces are a_piece elements apart.
  const void* A = nullptr;
  int64_t lda = 0, a_rows = 0, a_cols = 0, a_piece = 0;
  const void* B = nullptr;
  int64_t ldb = 0, b_rows = 0, b_cols = 0, b_piece = 0;
  int64_t M = 0, N = 0, K = 0;  // K: loop extent, a multiple of 32
  void* out = nullptr;          // double* (FP64 modes) or float2* (FF modes)
  int64_t ldo = 0;
  int mode = OUT_F64_STORE;
  int64_t kchunk = 0;           // FP64 path only: K per CTA (0 = whole K)
  int pieces = 3;               // mixed path: 3 BF16 pieces or 2 scaled FP16 pieces
  const float* scale_a = nullptr;  // FP16 pieces: device scales of A and B (the output is
  const float* scale_b = nullptr;  // divided by their product), else null
  int64_t tri = 0;                 // mixed path: > 0 skips output tiles whose rows all lie in blocks of
                                   // `tri` rows past every column block (only the upper block triangle of a
                                   // symmetric product is read later); the skipped output is left unwritten
  Status* status = nullptr;
  int* queue = nullptr;         // mixed path: device int, the launch's tile counter (zeroed by the launch)
  uint64_t timeout_ns = 2000000000ull;
};

// Returns 0 or a negative CC_ERR_* code.  ops[0].status and ops[0].queue
// serve the whole mixed launch.
int gemm_mixed(const GemmOp* ops, int nops, cudaStream_t stream);
int gemm_f64(const GemmOp& op, cudaStream_t stream);

// C_J = X_J + alpha * A B_J for J < nb, FP64 (csrc/t1.cu).  Element (m, k) of
// A (shared by every J) is at m * a_sm + k * a_sk; element (k, n) of B_J at
// J * b_sj + k * b_sk + n * b_sn; (m, n) of X_J and C_J likewise with their
// strides.  X may be null.  Returns 0 or CC_ERR_CUDA.
struct BatchedF64 {
  int M, N, K, nb;
  const double* A; int64_t a_sm, a_sk;
  const double* B; int64_t b_sj, b_sk, b_sn;
  const double* X; int64_t x_sj, x_sm, x_sn;
  double alpha;
  double* C; int64_t c_sj, c_sm, c_sn;
};
int batched_gemm_f64(const BatchedF64& g, cudaStream_t st);

// Records the text of a failed CUDA call for cc_ladder_strerror.
void note_cuda(cudaError_t e);

// Launch counter shared by every kernel launch of the library.
void count_launch(int n = 1);

// Leading-product window of the mixed contraction, in k-blocks of 32
// (the tuning knob if set, else `dflt`).
int tuned_win_kb(int dflt);
// contraction kernel of the split paths: 0 default, 1 single CTA, 2 CTA pairs
// (tcgen05 cta_group::2), 3 single CTA with one window per k-block
int tuned_contraction();

}  // namespace ccl
