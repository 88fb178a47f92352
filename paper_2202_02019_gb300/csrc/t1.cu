// T1-transformed basis for the ladder (Sec. II.C of arXiv:2202.02019).
//
// With the singles matrix T1 over all orbitals (T1[a][i] = t_i^a, virtual row,
// occupied column), x = I - T1 and y = I + T1^T.  Only two blocks reach the
// vvvv ladder and its density:
//
//   forward, vv block of x L^J y^T:   Lt^J_ac = L^J_ac - sum_i t_i^a L^J_ic
//   back, W^MO = x^T W y for a W that is non-zero in the vv block only:
//        vv block unchanged, ov block (W^J_ic)^MO = - sum_a t_i^a W^J_ac
//
// (y only touches occupied columns, and x only touches virtual rows through
// occupied columns, so no other block contributes.)  Both are batched small
// FP64 matrix products, one per Cholesky vector J, K = o (forward) or v
// (back).  They run once per amplitude iteration, against the ladder's
// O(o^2 v^4) work, so a plain FP64 tiled kernel is enough: its cost is the
// FP64 pipe (2 nj v^2 o flops, about 0.2 s at o=78, v=650, nj=4000).
#include <cstdint>

#include "ccladder.h"
#include "gemm.h"

namespace ccl {
namespace {

constexpr int TM = 32, TN = 64, TK = 32, NT = 256;

// C_J[m][n] = X_J[m][n] + alpha * sum_k A[m][k] B_J[k][n] for J < nb, every
// operand addressed by element strides (see BatchedF64).  X may be null.
__global__ void __launch_bounds__(NT) k_batched_gemm_f64(const BatchedF64 g) {
  const int M = g.M, N = g.N, K = g.K, nb = g.nb;
  const double* __restrict__ A = g.A;
  const double* __restrict__ B = g.B;
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const bool a_k_contig = (g.a_sk == 1);
  const bool b_k_contig = (g.b_sk == 1 && g.b_sn != 1);
  for (int J = blockIdx.z; J < nb; J += gridDim.z) {
    const double* BJ = B + static_cast<int64_t>(J) * g.b_sj;
    double acc[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
    for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
      for (int r = 0; r < (TM * TK) / NT; ++r) {
        const int idx = tid + r * NT;
        const int mm = a_k_contig ? idx / TK : idx % TM;
        const int kk = a_k_contig ? idx % TK : idx / TM;
        const int m = m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < M && k < K) ? A[static_cast<int64_t>(m) * g.a_sm + static_cast<int64_t>(k) * g.a_sk] : 0.0;
      }
#pragma unroll
      for (int r = 0; r < (TK * TN) / NT; ++r) {
        const int idx = tid + r * NT;
        const int nn = b_k_contig ? idx / TK : idx % TN;
        const int kk = b_k_contig ? idx % TK : idx / TN;
        const int n = n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < N && k < K) ? BJ[static_cast<int64_t>(k) * g.b_sk + static_cast<int64_t>(n) * g.b_sn] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < TK; ++kk) {
        const double a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double b = Bs[kk][tx + 16 * j];
          acc[0][j] = fma(a0, b, acc[0][j]);
          acc[1][j] = fma(a1, b, acc[1][j]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int m = m0 + 2 * ty + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n >= N) continue;
        const double x =
            g.X ? g.X[static_cast<int64_t>(J) * g.x_sj + static_cast<int64_t>(m) * g.x_sm + static_cast<int64_t>(n) * g.x_sn]
                : 0.0;
        g.C[static_cast<int64_t>(J) * g.c_sj + static_cast<int64_t>(m) * g.c_sm + static_cast<int64_t>(n) * g.c_sn] =
            fma(g.alpha, acc[i][j], x);
      }
    }
  }
}

int device_ok() {
  int dev = 0, maj = 0, min_ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return CC_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&min_, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return CC_ERR_DEVICE;
  return (maj == 10 && min_ == 3) ? CC_OK : CC_ERR_DEVICE;
}

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

// true if [p, p + n) and [q, q + m) (doubles) overlap
bool overlap(const double* p, int64_t n, const double* q, int64_t m) { return p < q + m && q < p + n; }

}  // namespace

int batched_gemm_f64(const BatchedF64& g, cudaStream_t st) {
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.nb < 65535 ? g.nb : 65535);
  k_batched_gemm_f64<<<grid, NT, 0, st>>>(g);
  count_launch();
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  return CC_OK;
}

}  // namespace ccl

using namespace ccl;

extern "C" {

int cc_ladder_t1_transform(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov, const double* t1,
                           double* L_vv_t1, void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !L_vv || !L_ov || !t1 || !L_vv_t1) return CC_ERR_ARG;
  if (!aligned8(L_vv) || !aligned8(L_ov) || !aligned8(t1) || !aligned8(L_vv_t1)) return CC_ERR_ARG;
  const int64_t nvv = static_cast<int64_t>(nj) * v * v, nov = static_cast<int64_t>(nj) * o * v;
  if (overlap(L_vv_t1, nvv, L_vv, nvv) || overlap(L_vv_t1, nvv, L_ov, nov) ||
      overlap(L_vv_t1, nvv, t1, static_cast<int64_t>(o) * v))
    return CC_ERR_ARG;
  if (const int rc = device_ok()) return rc;
  // M = a (v), N = c (v), K = i (o): A[a][i] = t1[i][a], B_J[i][c] = L_ov[J][i][c]
  const int64_t vv = static_cast<int64_t>(v) * v;
  BatchedF64 g{v, v, o, nj, t1, 1, v, L_ov, static_cast<int64_t>(o) * v, v, 1, L_vv, vv, v, 1, -1.0, L_vv_t1, vv, v, 1};
  return batched_gemm_f64(g, static_cast<cudaStream_t>(stream));
}

int cc_ladder_w_backtransform(int32_t o, int32_t v, int32_t nj, const double* W_vv, const double* t1, double* W_ov,
                              void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !W_vv || !t1 || !W_ov) return CC_ERR_ARG;
  if (!aligned8(W_vv) || !aligned8(t1) || !aligned8(W_ov)) return CC_ERR_ARG;
  const int64_t nvv = static_cast<int64_t>(nj) * v * v, nov = static_cast<int64_t>(nj) * o * v;
  if (overlap(W_ov, nov, W_vv, nvv) || overlap(W_ov, nov, t1, static_cast<int64_t>(o) * v)) return CC_ERR_ARG;
  if (const int rc = device_ok()) return rc;
  // M = i (o), N = c (v), K = a (v): A[i][a] = t1[i][a], B_J[a][c] = W_vv[J][a][c]
  BatchedF64 g{o, v, v, nj, t1, v, 1, W_vv, static_cast<int64_t>(v) * v, v, 1, nullptr, 0, 0, 0, -1.0, W_ov,
               static_cast<int64_t>(o) * v, v, 1};
  return batched_gemm_f64(g, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
