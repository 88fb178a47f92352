// FP64 tensor-core contraction (DMMA, mma.sync m8n8k4 f64) for the plain
// FP64 path.  Same contract as the mixed engine (see gemm.h): K-major A and
// B, M-contiguous FP64 output, K split into chunks added atomically.
//
// CTA tile 64 x 64 x 16, 8 warps as 2 (M) x 4 (N), each warp 32 x 16 =
// 4 x 2 DMMA tiles.  Operand tiles are staged through registers into a
// double-buffered shared-memory ring (row pitch 20 doubles, which keeps
// the fragment reads of each half-warp on distinct banks).
#include <algorithm>

#include "gemm.h"

namespace ccl {
namespace {

constexpr int FBM = 64, FBN = 64, FBK = 16, FP = FBK + 4;

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256) cc_gemm_f64_dmma(const double* __restrict__ A, long long lda,
                                                        long long a_rows, long long a_cols,
                                                        const double* __restrict__ B, long long ldb,
                                                        long long b_rows, long long b_cols, int M, int N, int K,
                                                        int kchunk, double* __restrict__ out, long long ldo,
                                                        int atomic) {
  __shared__ __align__(16) double As[2][FBM][FP];
  __shared__ __align__(16) double Bs[2][FBN][FP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;
  const int m0 = blockIdx.y * FBM, n0 = blockIdx.x * FBN;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(K, k0 + kchunk);
  const int nkt = (k1 - k0 + FBK - 1) / FBK;

  // loader mapping: 64 rows x 16 cols per operand, 4 consecutive cols per thread
  const int lr = tid >> 2, lc = (tid & 3) * 4;
  double ra[4], rb[4];
  auto load = [&](int kt) {
    const long long kk = k0 + (long long)kt * FBK + lc;
    const long long am = m0 + lr, bn = n0 + lr;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long k = kk + e;
      ra[e] = (am < a_rows && k < a_cols && k < k1) ? A[am * lda + k] : 0.0;
      rb[e] = (bn < b_rows && k < b_cols && k < k1) ? B[bn * ldb + k] : 0.0;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      As[buf][lr][lc + e] = ra[e];
      Bs[buf][lr][lc + e] = rb[e];
    }
  };

  double acc[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  if (nkt > 0) {
    load(0);
    stash(0);
  }
  __syncthreads();
  for (int kt = 0; kt < nkt; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nkt) load(kt + 1);
#pragma unroll
    for (int k4 = 0; k4 < FBK; k4 += 4) {
      double af[4], bf[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) af[i] = As[buf][wm * 32 + i * 8 + (lane >> 2)][k4 + (lane & 3)];
#pragma unroll
      for (int j = 0; j < 2; ++j) bf[j] = Bs[buf][wn * 16 + j * 8 + (lane >> 2)][k4 + (lane & 3)];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dmma(acc[i][j], af[i], bf[j]);
    }
    if (kt + 1 < nkt) stash(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + wm * 32 + i * 8 + (lane >> 2);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = n0 + wn * 16 + j * 8 + (lane & 3) * 2 + e;
        if (n < N) {
          double* p = out + (long long)n * ldo + m;
          if (atomic)
            atomicAdd(p, acc[i][j][e]);
          else
            *p = acc[i][j][e];
        }
      }
    }
  }
}

}  // namespace

int gemm_f64(const GemmOp& op, cudaStream_t stream) {
  if (op.M <= 0 || op.N <= 0 || op.K <= 0) return 0;
  if (!op.A || !op.B || !op.out) return -1;  // never launch on a missing operand or output
  if (op.mode != OUT_F64_STORE && op.mode != OUT_F64_ATOMIC) return -1;
  if (op.M > (int64_t)FBM * 65535 || op.K > 2147483647LL) return -1;
  const int64_t kc = op.kchunk ? std::min<int64_t>(op.kchunk, op.K) : op.K;
  const int64_t nsplit = (op.K + kc - 1) / kc;
  if (nsplit > 65535) return -1;
  if (nsplit > 1 && op.mode != OUT_F64_ATOMIC) return -1;  // split chunks must be added atomically
  dim3 grid(static_cast<unsigned>((op.N + FBN - 1) / FBN), static_cast<unsigned>((op.M + FBM - 1) / FBM),
            static_cast<unsigned>(nsplit));
  cc_gemm_f64_dmma<<<grid, 256, 0, stream>>>(
      static_cast<const double*>(op.A), op.lda, op.a_rows, op.a_cols, static_cast<const double*>(op.B), op.ldb,
      op.b_rows, op.b_cols, static_cast<int>(op.M), static_cast<int>(op.N), static_cast<int>(op.K),
      static_cast<int>(kc), static_cast<double*>(op.out), op.ldo, op.mode == OUT_F64_ATOMIC ? 1 : 0);
  count_launch();
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

}  // namespace ccl
