// CD-CCSD vvvv ladder library: workspace planning, preparation / packing
// kernels, reductions and the C ABI declared in include/ccladder.h.
//
// Algorithm (arXiv:2202.02019, closed shell):
//   Virtual rows are cut into blocks of `s`; a pair block (alpha <= beta)
//   holds the pairs a<=b with a in block alpha and b in block beta.  Per pair
//   block, with X^pm_ij = X_ij +- X_ji (Sec. II.B):
//     g-build   G[(a,c),(b,d)] = sum_J L^J_ac L^J_bd           (Sec. II.A)
//     pack      g+[ab,cd] = (G_cd + G_dc)(1/2 if c=d), g-[ab,cd] = G_cd - G_dc
//     ladder    Omega^pm[ab,ij] = sum_{cd} g^pm[ab,cd] tau^pm_ij^cd  (i<=j, c<=d)
//     unpack    Omega_ij^ab = (Omega+ + Omega-)/2, Omega_ij^ba = (Omega+ - Omega-)/2
//     Gamma     Gamma'^pm[ab,cd] = sum_ij w^pm_ij tbar^pm_ij^ab tau^pm_ij^cd
//               (w+ = 1/4 (i=j), 1/2 (i<j); w- = 1/2), Gamma = Gamma'+ + Gamma'-
//               extended by (anti)symmetry in ab and cd (Eq. v4density)
//     density   D^J_xc += sum_{y,d} Gamma_xycd L^J_yd   (Sec. II.C, W-tilde)
//   so that neither g nor Gamma exists beyond one pair block.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "ccladder.h"
#include "gemm.h"

namespace ccl {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

// Process-wide tuning (cc_ladder_set_tuning); 0 = default.
static std::atomic<int> g_tune_block{0}, g_tune_win{0}, g_tune_kernel{0};
int tuned_win_kb(int dflt) {
  const int w = g_tune_win.load();
  if (w > 0) return w;
  const char* e = std::getenv("CC_WIN_KB");
  return (e && *e) ? std::max(1, std::atoi(e)) : dflt;
}
int tuned_contraction() { return g_tune_kernel.load(); }

static std::mutex g_err_mu;
static std::string g_err_text;
void note_cuda(cudaError_t e) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err_text = cudaGetErrorString(e);
}

static inline int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decode_sym(int64_t k, int n, int& p, int& q) {
  int r = 0;
  while (r + 1 < n && pair_sym(r + 1, r + 1, n) <= k) ++r;
  p = r;
  q = static_cast<int>(k - pair_sym(r, r, n)) + r;
}

// local pair index inside a pair block -> (a_l, b_l)
__device__ __forceinline__ void pb_pair(int64_t pr, int nb, int diag, int& al, int& bl) {
  if (!diag) {
    al = static_cast<int>(pr / nb);
    bl = static_cast<int>(pr % nb);
  } else {  // pr = b_l (b_l + 1)/2 + a_l, a_l <= b_l
    int b = static_cast<int>((sqrt(8.0 * static_cast<double>(pr) + 1.0) - 1.0) * 0.5);
    while ((int64_t)(b + 1) * (b + 2) / 2 <= pr) ++b;
    while ((int64_t)b * (b + 1) / 2 > pr) --b;
    bl = b;
    al = static_cast<int>(pr - (int64_t)b * (b + 1) / 2);
  }
}

// ---------------------------------------------------------------------------
// preparation kernels
// ---------------------------------------------------------------------------
// L^J_ac ([nj][v*v]) -> LT[(a,c)][J] (J contiguous, zero for nj <= J < Kj)
// (trans: read L^J_ca instead, for the adjoint ladder)
template <typename T>
__global__ void k_prep_LT(const double* __restrict__ L, int nj, int64_t v2, int v, int trans, T* __restrict__ LT,
                          int64_t Kj, int64_t piece, const float* __restrict__ scl) {
  __shared__ double tile[32][33];
  const float sc = ld_scale(scl);
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int j0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int J = j0 + i;
    const int64_t r = r0 + threadIdx.x;
    const int64_t src = trans ? (r % v) * v + r / v : r;
    tile[i][threadIdx.x] = (J < nj && r < v2) ? L[static_cast<int64_t>(J) * v2 + src] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i;
    const int J = j0 + threadIdx.x;
    if (r < v2 && J < Kj) Store<T>::put(LT, r * Kj + J, piece, tile[threadIdx.x][i], sc);
  }
}

// L^J_yd -> LN[J][y*vp + d] (zero for d >= v)
template <typename T>
__global__ void k_prep_LN(const double* __restrict__ L, int nj, int v, int vp, T* __restrict__ LN, int64_t piece,
                          const float* __restrict__ scl) {
  const float sc = ld_scale(scl);
  const int64_t total = static_cast<int64_t>(nj) * v * vp;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t J = idx / (static_cast<int64_t>(v) * vp);
    const int64_t rem = idx - J * v * vp;
    const int y = static_cast<int>(rem / vp), d = static_cast<int>(rem % vp);
    const double x = d < v ? L[(J * v + y) * v + d] : 0.0;
    Store<T>::put(LN, idx, piece, x, sc);
  }
}

// tau^pm packed, rows = occupied pairs, columns = virtual pairs (K-major for
// the ladder):  tau+[p+(i,j)][k+(c,d)] = tau_ij^cd + tau_ji^cd   (i<=j, c<=d)
//               tau-[p-(i,j)][k-(c,d)] = tau_ij^cd - tau_ji^cd   (i<j,  c<d)
// With r2 non-null the packed doubles are U = r0 t2 + r2 instead (the
// excited-state C2 of App. A; t1 is then not read).
template <typename T>
__global__ void k_pack_tau(const double* __restrict__ t1, const double* __restrict__ t2, int o, int v,
                           T* __restrict__ tp, int64_t ldp, int64_t ppiece, T* __restrict__ tm, int64_t ldm,
                           int64_t mpiece, int minus, const float* __restrict__ scl,
                           const double* __restrict__ r2 = nullptr, double r0 = 1.0) {
  const float sc = ld_scale(scl);
  const int c = blockIdx.x;
  const int64_t pidx = blockIdx.y;
  int i, j;
  decode_sym(pidx, o, i, j);
  const int64_t vv = static_cast<int64_t>(v) * v;
  const double* tij = t2 + (static_cast<int64_t>(i) * o + j) * vv + static_cast<int64_t>(c) * v;
  const double* tji = t2 + (static_cast<int64_t>(j) * o + i) * vv + static_cast<int64_t>(c) * v;
  const double t1ic = t1 ? t1[static_cast<int64_t>(i) * v + c] : 0.0;
  const double t1jc = t1 ? t1[static_cast<int64_t>(j) * v + c] : 0.0;
  const int64_t kp0 = pair_sym(c, c, v) - c;
  const int64_t km0 = (c + 1 < v) ? pair_strict(c, c + 1, v) - (c + 1) : 0;
  const int64_t pm = (i < j) ? pair_strict(i, j, o) : -1;
  const double* rij = r2 ? r2 + (tij - t2) : nullptr;
  const double* rji = r2 ? r2 + (tji - t2) : nullptr;
  for (int d = c + threadIdx.x; d < v; d += blockDim.x) {
    double a, b;
    if (r2) {
      a = fma(r0, tij[d], rij[d]);  // U_ij^cd
      b = fma(r0, tji[d], rji[d]);  // U_ji^cd
    } else {
      a = tij[d] + (t1 ? t1ic * t1[static_cast<int64_t>(j) * v + d] : 0.0);  // tau_ij^cd
      b = tji[d] + (t1 ? t1jc * t1[static_cast<int64_t>(i) * v + d] : 0.0);  // tau_ji^cd
    }
    Store<T>::put(tp, pidx * ldp + kp0 + d, ppiece, a + b, sc);
    if (minus && pm >= 0 && d > c) Store<T>::put(tm, pm * ldm + km0 + d, mpiece, a - b, sc);
  }
}

// out[c][r] = in[r][c] for r < R, c < C (each split piece moved verbatim)
template <typename T, int NPc>
__global__ void k_transpose(const T* __restrict__ in, int64_t R, int64_t C, int64_t ldin, int64_t in_piece,
                            T* __restrict__ out, int64_t ldout, int64_t out_piece) {
  __shared__ T tile[NPc][32][33];
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32, r0 = static_cast<int64_t>(blockIdx.y) * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C)
#pragma unroll
      for (int p = 0; p < NPc; ++p) tile[p][i][threadIdx.x] = in[p * in_piece + r * ldin + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C)
#pragma unroll
      for (int p = 0; p < NPc; ++p) out[p * out_piece + c * ldout + r] = tile[p][threadIdx.x][i];
  }
}

// tbar^pm rows for the pairs of one pair block, weights of the ij sum folded in:
//   tbar+[ab][p+(i,j)] = w (tbar_ij^ab + tbar_ji^ab), w = 1/4 (i=j), 1/2 (i<j)
//   tbar-[ab][p-(i,j)] = 1/2 (tbar_ij^ab - tbar_ji^ab)          (0 for a = b)
template <typename T>
__global__ void k_pack_tbar(const double* __restrict__ tb2, int o, int v, int a0, int b0, int nb, int diag,
                            int64_t pair_off, T* __restrict__ bp, int64_t ldp, int64_t ppiece, T* __restrict__ bm,
                            int64_t ldm, int64_t mpiece, int minus, const float* __restrict__ scl) {
  const float sc = ld_scale(scl);
  int al, bl;
  pb_pair(blockIdx.x, nb, diag, al, bl);
  const int a = a0 + al, b = b0 + bl;
  const int64_t row = pair_off + blockIdx.x;
  const int64_t vv = static_cast<int64_t>(v) * v;
  for (int i = 0; i < o; ++i) {
    for (int j = i + threadIdx.x; j < o; j += blockDim.x) {
      const double x = tb2[(static_cast<int64_t>(i) * o + j) * vv + static_cast<int64_t>(a) * v + b];
      const double y = tb2[(static_cast<int64_t>(j) * o + i) * vv + static_cast<int64_t>(a) * v + b];
      const double w = (i == j) ? 0.25 : 0.5;
      Store<T>::put(bp, row * ldp + pair_sym(i, j, o), ppiece, w * (x + y), sc);
      if (minus && i < j)
        Store<T>::put(bm, row * ldm + pair_strict(i, j, o), mpiece, (a == b) ? 0.0 : 0.5 * (x - y), sc);
    }
  }
}

// ---------------------------------------------------------------------------
// pair-block pack / unpack kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_pair(int idx, int nt, int& ct, int& dt) {
  int r = 0;
  while (r + 1 < nt && pair_sym(r + 1, r + 1, nt) <= idx) ++r;
  ct = r;
  dt = static_cast<int>(idx - pair_sym(r, r, nt)) + r;
}

// G (rows (b_l,d), columns (a_l,c), pitch ldG; FP64 or float-float) ->
// g^pm packed rows:  g+[ab][k+(c,d)] = G_cd + G_dc (G_cc on the diagonal),
//                    g-[ab][k-(c,d)] = G_cd - G_dc (0 for a = b).
template <typename T, typename S>
__global__ void k_pack_g(const S* __restrict__ G, int64_t ldG, int v, int a0, int b0, int nb, int diag, int nt,
                         T* __restrict__ gp, int64_t ldp, int64_t ppiece, T* __restrict__ gm, int64_t ldm,
                         int64_t mpiece, int minus, const float* __restrict__ scl) {
  const float sc = ld_scale(scl);
  using A = Ar<S>;
  using V = typename A::V;
  __shared__ V s1[32][33];  // s1[dd][cc] = G^{ab}_{c,d}
  __shared__ V s2[32][33];  // s2[cc][dd] = G^{ab}_{d,c}
  const int64_t pr = blockIdx.y;
  int al, bl;
  pb_pair(pr, nb, diag, al, bl);
  int ct, dt;
  tile_pair(blockIdx.x, nt, ct, dt);
  const int c0 = ct * 32, d0 = dt * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t colA = static_cast<int64_t>(al) * v;
  const int64_t rowB = static_cast<int64_t>(bl) * v;
  for (int r = ty; r < 32; r += 8) {
    const int d = d0 + r, c = c0 + tx;
    s1[r][tx] = (c < v && d < v) ? A::ld(G, (rowB + d) * ldG + colA + c) : A::zero();
    const int c2 = c0 + r, d2 = d0 + tx;
    s2[r][tx] = (c2 < v && d2 < v) ? A::ld(G, (rowB + c2) * ldG + colA + d2) : A::zero();
  }
  __syncthreads();
  const bool same = (a0 + al) == (b0 + bl);
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, d = d0 + tx;
    if (c >= v || d >= v || d < c) continue;
    const V gcd = s1[tx][r], gdc = s2[r][tx];
    Put<T, V>::put(gp, pr * ldp + pair_sym(c, d, v), ppiece, (c == d) ? gcd : A::add(gcd, gdc), sc);
    if (minus && c < d)
      Put<T, V>::put(gm, pr * ldm + pair_strict(c, d, v), mpiece, same ? A::zero() : A::sub(gcd, gdc), sc);
  }
}

__device__ __forceinline__ double block_sum(double x) {
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = x;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  x = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  }
  return x;  // valid in thread 0
}

// Omega^pm [occupied pair][local pair] -> Omega_ij^ab (and/or the E partial)
template <typename S>
__global__ void k_unpack_omega(const S* __restrict__ Op, const S* __restrict__ Om, int64_t ldO, int o, int v,
                               int a0, int b0, int nb, int diag, int64_t npairs, int minus,
                               double* __restrict__ omega, const double* __restrict__ tbar2,
                               double* __restrict__ epart) {
  using A = Ar<S>;
  using V = typename A::V;
  const int i = blockIdx.x / o, j = blockIdx.x % o;
  const int lo = min(i, j), hi = max(i, j);
  const int64_t pp = pair_sym(lo, hi, o);
  const int64_t pm = (i != j) ? pair_strict(lo, hi, o) : -1;
  const bool neg = i > j;
  const int64_t base = (static_cast<int64_t>(i) * o + j) * v * v;
  double esum = 0.0;
  for (int64_t pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
    int al, bl;
    pb_pair(pr, nb, diag, al, bl);
    const int a = a0 + al, b = b0 + bl;
    const V P = A::ld(Op, pp * ldO + pr);
    V M = (minus && pm >= 0) ? A::ld(Om, pm * ldO + pr) : A::zero();
    if (neg) M = A::sub(A::zero(), M);
    const double wab = 0.5 * A::to_d(A::add(P, M)), wba = 0.5 * A::to_d(A::sub(P, M));
    const int64_t iab = base + static_cast<int64_t>(a) * v + b, iba = base + static_cast<int64_t>(b) * v + a;
    if (omega) {
      omega[iab] = wab;
      if (a != b) omega[iba] = wba;
    }
    if (epart) {
      esum += tbar2[iab] * wab;
      if (a != b) esum += tbar2[iba] * wba;
    }
  }
  if (epart) {
    const double sm = block_sum(esum);
    if (threadIdx.x == 0) epart[blockIdx.x] = sm;
  }
}

// Gamma'^pm [local pair][virtual pair] -> full Gamma^{xy}_{cd} slabs:
//   top[(x_l v + c)][(y_l vp + d)]  x in block alpha, y in block beta
//   bot[(x_l v + c)][(y_l vp + d)]  x in block beta,  y in block alpha
// Gamma_abcd = P(cd) + sgn(c,d) M(cd) for the stored pair (a<=b),
// Gamma_bacd = P(cd) - sgn(c,d) M(cd); P symmetric, M antisymmetric in cd.
template <typename T, typename S>
__global__ void k_unpack_gamma(const S* __restrict__ Gp, const S* __restrict__ Gm, int64_t ldp, int64_t ldm,
                               int v, int vp, int a0, int b0, int nb, int diag, int nt, int minus,
                               T* __restrict__ top, int64_t ldt, int64_t tpiece, T* __restrict__ bot, int64_t ldb,
                               int64_t bpiece, const float* __restrict__ scl) {
  const float sc = ld_scale(scl);
  using A = Ar<S>;
  using V = typename A::V;
  __shared__ V sP[32][33], sM[32][33];  // [c - c0][d - d0], c <= d
  const int64_t pr = blockIdx.y;
  int al, bl;
  pb_pair(pr, nb, diag, al, bl);
  int ct, dt;
  tile_pair(blockIdx.x, nt, ct, dt);
  const int c0 = ct * 32, d0 = dt * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, d = d0 + tx;
    const bool in = c < v && d < v && c <= d;
    sP[r][tx] = in ? A::ld(Gp, pr * ldp + pair_sym(c, d, v)) : A::zero();
    sM[r][tx] = (in && minus && c < d) ? A::ld(Gm, pr * ldm + pair_strict(c, d, v)) : A::zero();
  }
  __syncthreads();
  const bool same = (a0 + al) == (b0 + bl);
  // ordered pairs (x, y): (a, b) adds sgn M, (b, a) subtracts it
  for (int which = 0; which < 2; ++which) {
    if (which == 1 && same) break;
    T* dst;
    int64_t ld, piece, xrow, ycol;
    if (which == 0) {
      dst = top; ld = ldt; piece = tpiece;
      xrow = static_cast<int64_t>(al) * v; ycol = static_cast<int64_t>(bl) * vp;
    } else if (diag) {
      dst = top; ld = ldt; piece = tpiece;
      xrow = static_cast<int64_t>(bl) * v; ycol = static_cast<int64_t>(al) * vp;
    } else {
      dst = bot; ld = ldb; piece = bpiece;
      xrow = static_cast<int64_t>(bl) * v; ycol = static_cast<int64_t>(al) * vp;
    }
    // the tile itself (rows in ct, cols in dt) and, off the diagonal, its mirror; each thread
    // writes two adjacent columns (an even slab offset: ld, ycol and the tile origin are even)
    const int cp = (ty * 32 + tx) & 15, rr = (ty * 32 + tx) >> 4;
    for (int mirror = 0; mirror < (ct == dt ? 1 : 2); ++mirror) {
      const int R0 = mirror ? d0 : c0, W0 = mirror ? c0 : d0;
      for (int r = rr; r < 32; r += 16) {
        const int row = R0 + r, col = W0 + 2 * cp;
        if (row >= v || col >= v) continue;
        V val[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cl = min(col + h, v - 1);
          const int lo = min(row, cl), hi = max(row, cl);
          const V P = sP[lo - c0][hi - d0];
          const V M = sM[lo - c0][hi - d0];
          // sign of M: +1 above the diagonal for (a, b), flipped below it and for (b, a)
          const bool addM = (row < cl) == (which == 0);
          val[h] = (row == cl) ? P : (addM ? A::add(P, M) : A::sub(P, M));
        }
        const int64_t idx = (xrow + row) * ld + ycol + col;
        if (col + 1 < v)
          Put2<T, V>::put2(dst, idx, piece, val[0], val[1], sc);
        else
          Put<T, V>::put(dst, idx, piece, val[0], sc);
      }
    }
  }
}

// float-float -> FP64 (the final three-index density)
__global__ void k_ff_to_f64(const float2* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float2 x = in[k];
    out[k] = static_cast<double>(x.x) + static_cast<double>(x.y);
  }
}

// ---------------------------------------------------------------------------
// reductions, update, debug wait
// ---------------------------------------------------------------------------
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                              double* __restrict__ part) {
  double s = 0.0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    s += x[k] * y[k];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_final(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += part[k];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_update(const double* __restrict__ t2, const double* __restrict__ om, const double* __restrict__ eps,
                         int o, int v, double* __restrict__ out) {
  const int64_t total = static_cast<int64_t>(o) * o * v * v;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(k % v);
    const int a = static_cast<int>((k / v) % v);
    const int j = static_cast<int>((k / (static_cast<int64_t>(v) * v)) % o);
    const int i = static_cast<int>(k / (static_cast<int64_t>(v) * v * o));
    const double den = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    out[k] = t2[k] + om[k] / den;
  }
}

// MP2-like driver from the contraction output G[(j,b)][(i,a)] (ld = o v):
// g[i][j][a][b] = (G[(i,a),(j,b)] + G[(j,b),(i,a)]) / 2, exactly pair symmetric
template <typename S>
__global__ void k_driver_to_t2(const S* __restrict__ G, int o, int v, double* __restrict__ g) {
  const int64_t ov = static_cast<int64_t>(o) * v, total = ov * ov;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(k % v);
    const int a = static_cast<int>((k / v) % v);
    const int j = static_cast<int>((k / (static_cast<int64_t>(v) * v)) % o);
    const int i = static_cast<int>(k / (static_cast<int64_t>(v) * v * o));
    const int64_t ia = static_cast<int64_t>(i) * v + a, jb = static_cast<int64_t>(j) * v + b;
    g[k] = 0.5 * (Ar<S>::to_d(G[jb * ov + ia]) + Ar<S>::to_d(G[ia * ov + jb]));
  }
}

// Jacobi step t' = (g + (Omega_ij^ab + Omega_ji^ba) / 2) / (e_i + e_j - e_a - e_b)
// and per-block partial sums of (t' - t)^2
__global__ void k_jacobi(const double* __restrict__ g, const double* __restrict__ om, const double* __restrict__ t,
                         const double* __restrict__ eps, int o, int v, double* __restrict__ tn,
                         double* __restrict__ part) {
  const int64_t vv = static_cast<int64_t>(v) * v, total = static_cast<int64_t>(o) * o * vv;
  double s = 0.0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(k % v);
    const int a = static_cast<int>((k / v) % v);
    const int j = static_cast<int>((k / vv) % o);
    const int i = static_cast<int>(k / (vv * o));
    const int64_t kt = (static_cast<int64_t>(j) * o + i) * vv + static_cast<int64_t>(b) * v + a;
    const double den = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    const double x = (g[k] + 0.5 * (om[k] + om[kt])) / den;
    const double d = x - t[k];
    s += d * d;
    tn[k] = x;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Doubles as an (o v) x (o v) matrix for the OV^3 contributions:
// P[(i,c)][(m,b)] = alpha x_im^cb + beta x_mi^cb (+ gamma u_im^cb + delta u_mi^cb with a second
// array u) (zero for columns past o v), split into the operand format; (alpha, beta) = (2, -1)
// gives t~ = 2 t - t^T, (1, 0) the amplitudes
template <typename T>
__global__ void k_pack_pairmat(const double* __restrict__ t2, int o, int v, double alpha, double beta,
                               T* __restrict__ P, int64_t ld, int64_t piece, const double* __restrict__ u2 = nullptr,
                               double gamma = 0.0, double delta = 0.0) {
  const int64_t ov = static_cast<int64_t>(o) * v, vv = static_cast<int64_t>(v) * v;
  const int64_t r = blockIdx.x;  // (i, c)
  const int i = static_cast<int>(r / v), c = static_cast<int>(r % v);
  for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) {
    double x = 0.0;
    if (k < ov) {
      const int m = static_cast<int>(k / v), b = static_cast<int>(k % v);
      const int64_t e1 = (static_cast<int64_t>(i) * o + m) * vv + static_cast<int64_t>(c) * v + b;
      const int64_t e2 = (static_cast<int64_t>(m) * o + i) * vv + static_cast<int64_t>(c) * v + b;
      x = alpha * t2[e1] + beta * t2[e2];
      if (u2) x += gamma * u2[e1] + delta * u2[e2];
    }
    Store<T>::put(P, r * ld + k, piece, x, 1.f);
  }
}

// A strided 4-D view of an FP64 array: element (r1, r2, k1, k2) at
// p[r1*sr1 + r2*sr2 + k1*sk1 + k2*sk2], times coef (p null: the view is 0).
struct View {
  const double* p;
  int64_t sr1, sr2, sk1, sk2;
  double coef;
};

// Contraction operand from up to two views: out[r][k] = v1(r, k) + v2(r, k),
// r = r1*R2 + r2 (row), k = k1*K2 + k2 (reduction index, contiguous), zero for
// k >= K1*K2 up to the row pitch ld; written in the operand format.
template <typename T>
__global__ void k_pack_view(View v1, View v2, int64_t R1, int64_t R2, int64_t K1, int64_t K2, T* __restrict__ out,
                            int64_t ld, int64_t piece) {
  const int64_t total = R1 * R2 * ld, K = K1 * K2;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = q / ld, k = q % ld;
    double x = 0.0;
    if (k < K) {
      const int64_t r1 = r / R2, r2 = r % R2, k1 = k / K2, k2 = k % K2;
      x = v1.coef * v1.p[r1 * v1.sr1 + r2 * v1.sr2 + k1 * v1.sk1 + k2 * v1.sk2];
      if (v2.p) x += v2.coef * v2.p[r1 * v2.sr1 + r2 * v2.sr2 + k1 * v2.sk1 + k2 * v2.sk2];
    }
    Store<T>::put(out, q, piece, x, 1.f);
  }
}

// dst[n*sdn + m*sdm] (= | +=) alpha * src[n*ldo + m] for m < M, n < N: a
// contraction output (float-float or FP64) into a strided FP64 array
template <typename S>
__global__ void k_out_view(const S* __restrict__ src, int64_t ldo, int64_t M, int64_t N, double alpha,
                           double* __restrict__ dst, int64_t sdn, int64_t sdm, int accumulate) {
  const int64_t total = M * N;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t n = q / M, m = q % M;
    const double x = alpha * Ar<S>::to_d(src[n * ldo + m]);
    double* d = dst + n * sdn + m * sdm;
    *d = accumulate ? *d + x : x;
  }
}

// out[r][k] = src[r][k] (k < cols), 0 up to ld, in the operand format
template <typename T>
__global__ void k_pack_rows(const double* __restrict__ src, int64_t rows, int64_t cols, T* __restrict__ out,
                            int64_t ld, int64_t piece) {
  const int64_t total = rows * ld;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = q / ld, k = q % ld;
    Store<T>::put(out, q, piece, k < cols ? src[r * cols + k] : 0.0, 1.f);
  }
}

template <typename S>
__global__ void k_to_f64_scaled(const S* __restrict__ in, double* __restrict__ out, int64_t n, double scale) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[k] = scale * Ar<S>::to_d(in[k]);
}

// x[k] *= factor * (*g)  (g: a device scalar, e.g. the incoming gradient of E)
__global__ void k_scale_by(double* __restrict__ x, int64_t n, double factor, const double* __restrict__ g) {
  const double f = factor * (g ? *g : 1.0);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    x[k] *= f;
}

__global__ void k_debug_wait(const int* flag, unsigned long long timeout_ns, Status* st) {
  const volatile int* f = flag;
  const uint64_t t0 = globaltimer();
  while (*f == 0) {
    if (globaltimer() - t0 > timeout_ns) {
      latch_error(st, kErrTimeout, 900);
      return;
    }
    __nanosleep(1000);
  }
}

// ---------------------------------------------------------------------------
// operand scales of the FP16 two-piece path
// ---------------------------------------------------------------------------
// Bounds are accumulated as float bit patterns with atomicMax (non-negative
// floats order like their bits) from power-of-two upper bounds of |x| read
// off the exponent field, so no FP64 arithmetic is needed:
//   bnd[0] max |L|,    bnd[1] max_(a,c) sum_J (L^J_ac)^2
//   bnd[2] max |tau|,  bnd[3] max_(c,d) sum_ij (tau_ij^cd)^2
//   bnd[4] max |tbar|, bnd[5] max_(a,b) sum_ij (tbar_ij^ab)^2
// Loose bounds only cost a few bits of head-room below FP16's range top;
// what matters is that no scaled operand can overflow.
__device__ __forceinline__ float pow2_above(double x) {
  const int e = static_cast<int>((static_cast<unsigned>(__double2hiint(x)) >> 20) & 0x7FF) - 1023;
  const int f = min(max(e + 1, -126), 127);  // |x| < 2^(e+1)
  return __int_as_float((f + 127) << 23);
}

__device__ __forceinline__ void block_max2(float a, float b, unsigned* pa, unsigned* pb) {
  __shared__ float ra[32], rb[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a = fmaxf(a, __shfl_down_sync(0xffffffffu, a, off));
    b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, off));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < static_cast<int>((blockDim.x + 31) >> 5); ++k) {
      a = fmaxf(a, ra[k]);
      b = fmaxf(b, rb[k]);
    }
    atomicMax(pa, __float_as_uint(a));
    atomicMax(pb, __float_as_uint(b));
  }
}

// L [nj][v2]: threads over (a,c), loop over J
__global__ void k_bound_L(const double* __restrict__ L, int nj, int64_t v2, unsigned* __restrict__ bnd) {
  float mx = 0.f, mrow = 0.f;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < v2;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float sq = 0.f;
    for (int J = 0; J < nj; ++J) {
      const float u = pow2_above(L[static_cast<int64_t>(J) * v2 + r]);
      sq += u * u;
      mx = fmaxf(mx, u);
    }
    mrow = fmaxf(mrow, sq);
  }
  block_max2(mx, mrow, bnd + 0, bnd + 1);
}

// x_ij^ab = t2[i][j][a][b] + t1[i][a] t1[j][b] (t1 may be null): threads over (a,b)
// (with r2 non-null: x = r0 t2 + r2, t1 not read)
__global__ void k_bound_amp(const double* __restrict__ t1, const double* __restrict__ t2, int o, int v,
                            unsigned* __restrict__ bnd, const double* __restrict__ r2 = nullptr, double r0 = 1.0) {
  const float r0b = pow2_above(r0);
  const int64_t vv = static_cast<int64_t>(v) * v;
  float mx = 0.f, mrow = 0.f;
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < vv;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int a = static_cast<int>(r / v), b = static_cast<int>(r % v);
    float sq = 0.f;
    for (int i = 0; i < o; ++i)
      for (int j = 0; j < o; ++j) {
        const int64_t e = (static_cast<int64_t>(i) * o + j) * vv + r;
        float u = pow2_above(t2[e]);
        if (r2)
          u = r0b * u + pow2_above(r2[e]);
        else if (t1)
          u += pow2_above(t1[static_cast<int64_t>(i) * v + a]) * pow2_above(t1[static_cast<int64_t>(j) * v + b]);
        sq += u * u;
        mx = fmaxf(mx, u);
      }
    mrow = fmaxf(mrow, sq);
  }
  block_max2(mx, mrow, bnd + 0, bnd + 1);
}

// scale = largest power of two with bound * scale <= 2^14
__device__ __forceinline__ float pow2_scale(float bound) {
  if (!(bound > 0.f)) return 1.f;
  int e;
  frexpf(16384.f / (bound * 1.01f), &e);  // 16384/bound in [2^(e-1), 2^e)
  e = min(max(e - 1, -120), 120);
  return ldexpf(1.f, e);
}

// sc[0] L (LT, LN), sc[1] tau^pm, sc[2] tbar^pm, sc[3] g^pm, sc[4] Gamma slabs
__global__ void k_scales(const unsigned* __restrict__ bnd, float* __restrict__ sc) {
  const float bL = __uint_as_float(bnd[0]), bLrow = __uint_as_float(bnd[1]);
  const float bt = __uint_as_float(bnd[2]), btrow = __uint_as_float(bnd[3]);
  const float bb = __uint_as_float(bnd[4]), bbrow = __uint_as_float(bnd[5]);
  sc[0] = pow2_scale(bL);
  sc[1] = pow2_scale(2.f * bt);                          // tau_ij + tau_ji
  sc[2] = pow2_scale(bb);                                // (1/4, 1/2) weighted sums of two
  sc[3] = pow2_scale(2.f * bLrow);                       // |g+-| <= 2 max |G| <= 2 max_row |L|^2
  sc[4] = pow2_scale(sqrtf(bbrow) * sqrtf(btrow));       // |Gamma| <= |tbar_ab| |tau_cd|
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
struct PBlock {
  int a0, na, b0, nb, diag;
  int64_t npairs, pair_off;
};

struct Plan {
  int o = 0, v = 0, nj = 0, prec = 0;
  int vp = 0, s = 0, nblk = 0, nt = 0;
  int minus = 0;
  int64_t Pvp = 0, Pvm = 0, Pop = 0, Pom = 0;
  int64_t Kj = 0, Kvp = 0, Kvm = 0, Kop = 0, Kom = 0;
  std::vector<PBlock> pbs;
  int64_t maxpairs = 0, maxrows = 0, ldO = 0, ldt = 0;
  int64_t n_epart = 0;
  // Byte offsets inside the system's region (operands prepared once per call,
  // the D accumulator and the E partials) and inside a scratch slot (the
  // intermediates of one pair block in flight).  0 = not present.
  size_t s_scl = 0;  // FP16 path: operand bounds (8 x u32) at +0, scales (5 floats) at +64 (always present)
  size_t s_tp = 0, s_tm = 0, s_LT = 0, s_LN = 0, s_tpT = 0, s_tmT = 0, s_bp = 0, s_bm = 0, s_D = 0, s_E = 0;
  // A scratch slot has four parts: for each of the two chains (residual, density) its operand pieces
  // (g+-; the Gamma slabs) and its float-float (or FP64) scratch (G, Omega+-; Gamma+-).  Slot offsets
  // are relative to the start of their part.
  size_t k_gp = 0, k_gm = 0;              // residual pieces
  size_t k_G = 0, k_Op = 0, k_Om = 0;     // residual scratch
  size_t k_Gt = 0, k_Gb = 0;              // density pieces
  size_t k_Gp = 0, k_Gm = 0;              // density scratch
  size_t sys_bytes = 0, part[4] = {0, 0, 0, 0};  // bytes of: residual pieces, residual scratch, density ...
};

constexpr size_t kStatusBytes = 256;
constexpr int kBatchSlots = 8;  // pair blocks of different systems in flight at once (batched schedule)

static int env_int(const char* name, int dflt) {
  const char* s = std::getenv(name);
  if (!s || !*s) return dflt;
  return std::atoi(s);
}

// bytes of an R x C matrix in the path's element format
static size_t mat_bytes(int prec, int64_t R, int64_t C) {
  return static_cast<size_t>(R) * static_cast<size_t>(C) * (prec == CC_PREC_MIXED ? 6 : prec == CC_PREC_FP16X2 ? 4 : 8);
}

static bool make_plan(const cc_ladder_system& sy, int prec, int which, Plan& P) {
  const int64_t o = sy.o, v = sy.v, nj = sy.nj;
  P.o = sy.o; P.v = sy.v; P.nj = sy.nj; P.prec = prec;
  P.vp = static_cast<int>(rup(v, 16));  // s * vp is then a multiple of 64 (the contraction's K step)
  P.Pvp = v * (v + 1) / 2; P.Pvm = v * (v - 1) / 2;
  P.Pop = o * (o + 1) / 2; P.Pom = o * (o - 1) / 2;
  P.minus = (P.Pvm > 0 && P.Pom > 0) ? 1 : 0;
  // contraction dimensions padded to the mixed engine's K step (64) with zeros
  P.Kj = rup(nj, 64);
  P.Kvp = rup(P.Pvp, 64); P.Kvm = rup(P.Pvm, 64);
  P.Kop = rup(P.Pop, 64); P.Kom = rup(P.Pom, 64);
  int s = g_tune_block.load() > 0 ? g_tune_block.load() : env_int("CC_BLOCK", 48);
  s = std::max(4, (s / 4) * 4);
  s = static_cast<int>(std::min<int64_t>(s, rup(v, 4)));
  P.s = s;
  P.nblk = static_cast<int>((v + s - 1) / s);
  P.nt = static_cast<int>((v + 31) / 32);
  P.pbs.clear();
  int64_t off = 0;
  for (int al = 0; al < P.nblk; ++al)
    for (int be = al; be < P.nblk; ++be) {
      PBlock b;
      b.a0 = al * s; b.na = static_cast<int>(std::min<int64_t>(s, v - b.a0));
      b.b0 = be * s; b.nb = static_cast<int>(std::min<int64_t>(s, v - b.b0));
      b.diag = al == be;
      b.npairs = b.diag ? (int64_t)b.na * (b.na + 1) / 2 : (int64_t)b.na * b.nb;
      b.pair_off = off;
      off += b.npairs;
      P.pbs.push_back(b);
      P.maxpairs = std::max(P.maxpairs, b.npairs);
    }
  if (off != P.Pvp) return false;
  if (P.maxpairs > 65535 || P.Pop > 65535) return false;  // grid.y limits of the pack kernels
  P.maxrows = static_cast<int64_t>(s) * v;
  P.ldO = rup(P.maxpairs, 2);
  P.ldt = static_cast<int64_t>(s) * P.vp;
  P.n_epart = std::max<int64_t>(1024, static_cast<int64_t>(P.pbs.size()) * o * o);

  const bool res = which & (CC_WS_RESIDUAL | CC_WS_LAGRANGIAN);
  const bool den = which & CC_WS_DENSITY;
  // every region starts past a 256-byte gap, so that offset 0 means "not present" in each
  size_t sys = 256, rp = 256, rs = 256, dp = 256, ds = 256;
  auto take = [](size_t& cur, size_t bytes) {
    const size_t at = cur;
    cur += rup(static_cast<int64_t>(bytes), 256);
    return at;
  };
  const int pr = prec;
  P.s_scl = take(sys, 256);  // = 256
  P.s_tp = take(sys, mat_bytes(pr, P.Pop, P.Kvp));
  P.s_tm = take(sys, mat_bytes(pr, P.Pom, P.Kvm));
  if (res) {
    P.s_LT = take(sys, mat_bytes(pr, v * v, P.Kj));
    P.k_G = take(rs, static_cast<size_t>(P.maxrows) * P.maxrows * 8);
    P.k_gp = take(rp, mat_bytes(pr, P.maxpairs, P.Kvp));
    P.k_gm = take(rp, mat_bytes(pr, P.maxpairs, P.Kvm));
    P.k_Op = take(rs, static_cast<size_t>(P.Pop) * P.ldO * 8);
    P.k_Om = take(rs, static_cast<size_t>(P.Pom) * P.ldO * 8);
  }
  if (den) {
    P.s_LN = take(sys, mat_bytes(pr, nj, v * P.vp));
    P.s_tpT = take(sys, mat_bytes(pr, P.Pvp, P.Kop));
    P.s_tmT = take(sys, mat_bytes(pr, P.Pvm, P.Kom));
    P.s_bp = take(sys, mat_bytes(pr, P.Pvp, P.Kop));
    P.s_bm = take(sys, mat_bytes(pr, P.Pvp, P.Kom));
    if (prec != CC_PREC_FP64) P.s_D = take(sys, static_cast<size_t>(nj) * v * v * 8);  // float-float D
    P.k_Gp = take(ds, static_cast<size_t>(P.maxpairs) * P.Kvp * 8);
    P.k_Gm = take(ds, static_cast<size_t>(P.maxpairs) * P.Kvm * 8);
    P.k_Gt = take(dp, mat_bytes(pr, P.maxrows, P.ldt));
    P.k_Gb = take(dp, mat_bytes(pr, P.maxrows, P.ldt));
  }
  P.s_E = take(sys, static_cast<size_t>(P.n_epart) * 8);
  P.sys_bytes = sys;
  P.part[0] = rp;
  P.part[1] = rs;
  P.part[2] = dp;
  P.part[3] = ds;
  return true;
}

// ---------------------------------------------------------------------------
// execution
// ---------------------------------------------------------------------------
// Workspace header (the first kStatusBytes bytes): the latched Status at 0,
// the tile-queue counters of the contraction launches at kQueueOffset (the
// caller's stream) and kQueueOffset + 4 (the density chain's stream).
constexpr size_t kQueueOffset = 224;

struct Ctx {
  cudaStream_t st;
  Status* status;
  int* queue = nullptr;  // tile counter of the mixed contraction launches
  uint64_t timeout_ns;
  bool adjoint = false;  // residual of tbar2 with L^J transposed: sum_ab tbar_ij^ab g_acbd
  int err = 0;
  void check(int rc) {
    if (rc && !err) err = rc;
  }
  void cuda(cudaError_t e) {
    if (e != cudaSuccess && !err) {
      note_cuda(e);
      err = CC_ERR_CUDA;
    }
  }
  void launched(int n = 1) {
    count_launch(n);
    cuda(cudaPeekAtLastError());
  }
};

// Optional instrumentation: CUDA events recorded on the launching stream
// around every contraction launch, summed when read.
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  size_t used = 0;
  double flops = 0.0;
  long long launches = 0;
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};
static Profiler g_prof;

template <typename F>
static int profiled(const GemmOp* ops, int nops, cudaStream_t s, F&& launch) {
  bool on;
  {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    on = g_prof.on;
  }
  if (!on) return launch();
  cudaEvent_t e0, e1;
  {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    e0 = g_prof.get();
    e1 = g_prof.get();
    g_prof.pending.emplace_back(e0, e1);
    for (int i = 0; i < nops; ++i)
      g_prof.flops += 2.0 * static_cast<double>(ops[i].M) * static_cast<double>(ops[i].N) * static_cast<double>(ops[i].K);
    g_prof.launches += 1;
  }
  cudaEventRecord(e0, s);
  const int rc = launch();
  cudaEventRecord(e1, s);
  return rc;
}

template <typename T>
struct Path;
template <>
struct Path<double> {
  using S = double;  // scratch element
  static constexpr int NP = 1;
  static constexpr bool mixed = false;
};
template <>
struct Path<__nv_bfloat16> {
  using S = float2;
  static constexpr int NP = 3;
  static constexpr bool mixed = true;
};
template <>
struct Path<__half> {
  using S = float2;
  static constexpr int NP = 2;
  static constexpr bool mixed = true;
};

template <typename T>
static T* at(char* ws, size_t off) {
  return reinterpret_cast<T*>(ws + off);
}

// One contraction out[n*ldo + m] (= | +=) sum_k A[m][k] B[n][k] as an op
// record; `acc` asks for accumulation into what the output holds.
struct Gm {
  const void* A; int64_t lda, a_rows, a_cols, a_piece;
  const void* B; int64_t ldb, b_rows, b_cols, b_piece;
  int64_t M, N, K;
  void* out; int64_t ldo;
  bool acc;
  const float* sa = nullptr;  // operand scales (FP16 two-piece path)
  const float* sb = nullptr;
  int64_t tri = 0;            // upper block triangle only (see GemmOp::tri)
};

// K chunk for the FP64 path: whole K unless the launch would have fewer
// than ~2 waves of CTAs on 152 SMs; then split K (chunks added atomically).
static int64_t f64_kchunk(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ((M + 63) / 64) * ((N + 63) / 64);
  const int64_t target = 2 * 152;
  if (tiles >= target) return K;
  const int64_t splits = std::min<int64_t>((target + tiles - 1) / tiles, std::max<int64_t>(1, K / 256));
  return std::max<int64_t>(32, rup((K + splits - 1) / splits, 32));
}

// Launch one group of independent contractions (one persistent launch on the
// mixed paths, one launch each on the FP64 path).
template <typename T>
static void run_gemms(const Gm* g, int n, Ctx& c) {
  if (n <= 0) return;
  std::vector<GemmOp> ops(n);
  for (int i = 0; i < n; ++i) {
    GemmOp& o = ops[i];
    o.A = g[i].A; o.lda = g[i].lda; o.a_rows = g[i].a_rows; o.a_cols = g[i].a_cols; o.a_piece = g[i].a_piece;
    o.B = g[i].B; o.ldb = g[i].ldb; o.b_rows = g[i].b_rows; o.b_cols = g[i].b_cols; o.b_piece = g[i].b_piece;
    o.M = g[i].M; o.N = g[i].N; o.K = g[i].K; o.out = g[i].out; o.ldo = g[i].ldo; o.tri = g[i].tri;
    o.status = c.status; o.queue = c.queue; o.timeout_ns = c.timeout_ns;
  }
  if (Path<T>::mixed) {
    for (int i = 0; i < n; ++i) {
      ops[i].mode = g[i].acc ? OUT_FF_ACCUM : OUT_FF_STORE;
      ops[i].pieces = Path<T>::NP;
      ops[i].scale_a = g[i].sa;
      ops[i].scale_b = g[i].sb;
    }
    c.check(profiled(ops.data(), n, c.st, [&] { return gemm_mixed(ops.data(), n, c.st); }));
  } else {
    for (int i = 0; i < n; ++i) {
      GemmOp& o = ops[i];
      o.kchunk = f64_kchunk(o.M, o.N, o.K);
      const bool split = o.kchunk < o.K;
      if (split && !g[i].acc)
        c.cuda(cudaMemsetAsync(o.out, 0, static_cast<size_t>(o.N) * o.ldo * sizeof(double), c.st));
      o.mode = (split || g[i].acc) ? OUT_F64_ATOMIC : OUT_F64_STORE;
      c.check(profiled(&o, 1, c.st, [&] { return gemm_f64(o, c.st); }));
    }
  }
}

// One system of a call: its plan, its workspace region and its outputs.
struct SysRun {
  const cc_ladder_system* sy = nullptr;
  Plan P;
  char* base = nullptr;  // the system's region of the workspace
  double* omega = nullptr;
  double* D = nullptr;
  double* E = nullptr;
  const double* r2 = nullptr;  // excited-state density: the ladder doubles are r0 t2 + r2
  double r0 = 1.0;
  size_t next = 0;             // next pair block to schedule
  double left = 0.0;           // counted flops of the pair blocks not yet scheduled
  std::vector<size_t> subset;  // non-empty: only these pair blocks (a shard of the system)
};

// One pair block in flight: the system, the block, the scratch slot it uses.
// A slot has one part per chain and kind (residual pieces, residual scratch,
// density pieces, density scratch), each as large as the largest system of
// the call needs: the two chains run on different streams, and a slot serves
// different systems (with different layouts) in successive waves, so a
// chain must never touch bytes the other chain may be using.
struct Slot {
  char* part[4];
};
struct Item {
  SysRun* r;
  size_t ib;
  Slot slot;
};

template <typename T>
struct Ptrs {
  using S = typename Path<T>::S;
  T *tp, *tm, *LT, *LN, *tpT, *tmT, *bp, *bm;
  S *Dacc;
  double* epart;
  unsigned* bnd;
  float* scl;
  int64_t tp_piece, tm_piece, LT_piece, LN_piece, tpT_piece, tmT_piece, bp_piece, bm_piece;
  Ptrs(const SysRun& R) {
    const Plan& P = R.P;
    char* w = R.base;
    auto opt = [&](size_t off) { return off ? w + off : nullptr; };
    tp = reinterpret_cast<T*>(opt(P.s_tp));
    tm = reinterpret_cast<T*>(opt(P.s_tm));
    LT = reinterpret_cast<T*>(opt(P.s_LT));
    LN = reinterpret_cast<T*>(opt(P.s_LN));
    tpT = reinterpret_cast<T*>(opt(P.s_tpT));
    tmT = reinterpret_cast<T*>(opt(P.s_tmT));
    bp = reinterpret_cast<T*>(opt(P.s_bp));
    bm = reinterpret_cast<T*>(opt(P.s_bm));
    // D accumulates over pair blocks in float-float scratch (mixed) or directly in the FP64 output
    Dacc = Path<T>::mixed ? reinterpret_cast<S*>(opt(P.s_D)) : reinterpret_cast<S*>(R.D);
    epart = reinterpret_cast<double*>(w + P.s_E);
    bnd = reinterpret_cast<unsigned*>(w + P.s_scl);
    scl = reinterpret_cast<float*>(w + P.s_scl + 64);
    const int64_t vv = static_cast<int64_t>(P.v) * P.v;
    tp_piece = P.Pop * P.Kvp;
    tm_piece = P.Pom * P.Kvm;
    LT_piece = vv * P.Kj;
    LN_piece = static_cast<int64_t>(P.nj) * P.v * P.vp;
    tpT_piece = P.Pvp * P.Kop;
    tmT_piece = P.Pvm * P.Kom;
    bp_piece = P.Pvp * P.Kop;
    bm_piece = P.Pvp * P.Kom;
  }
  // operand scales of the FP16 two-piece path, else null
  const float* SC(int i) const { return std::is_same<T, __half>::value ? scl + i : nullptr; }
};

// Once per system and call: operand scales (FP16 path), tau^pm, L in both
// layouts, the transposed tau^pm and the tbar^pm rows; zeroed D accumulator.
template <typename T>
static void prep_system(const SysRun& R, bool do_res, bool do_den, Ctx& c) {
  const cc_ladder_system& sy = *R.sy;
  const Plan& P = R.P;
  const Ptrs<T> X(R);
  const int o = P.o, v = P.v, nj = P.nj, vp = P.vp;
  const int64_t vv = static_cast<int64_t>(v) * v;
  const int minus = P.minus;
  cudaStream_t st = c.st;
  if (std::is_same<T, __half>::value) {
    // device-side bounds and scales, no host synchronisation
    const double* amp = c.adjoint ? sy.tbar2 : sy.t2;
    c.cuda(cudaMemsetAsync(X.bnd, 0, 8 * sizeof(unsigned), st));
    k_bound_L<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(sy.L_vv, nj, vv, X.bnd);
    k_bound_amp<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(
        c.adjoint ? nullptr : sy.t1, amp, o, v, X.bnd + 2, R.r2, R.r0);
    c.launched(2);
    if (do_den) {
      k_bound_amp<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(
          nullptr, sy.tbar2, o, v, X.bnd + 4);
      c.launched();
    }
    k_scales<<<1, 1, 0, st>>>(X.bnd, X.scl);
    c.launched();
  }
  // tau^pm (both directions need it)
  c.cuda(cudaMemsetAsync(X.tp, 0, mat_bytes(P.prec, P.Pop, P.Kvp), st));
  if (minus) c.cuda(cudaMemsetAsync(X.tm, 0, mat_bytes(P.prec, P.Pom, P.Kvm), st));
  k_pack_tau<T><<<dim3(v, static_cast<unsigned>(P.Pop)), 128, 0, st>>>(
      c.adjoint ? nullptr : sy.t1, c.adjoint ? sy.tbar2 : sy.t2, o, v, X.tp, P.Kvp, X.tp_piece, X.tm, P.Kvm,
      X.tm_piece, minus, X.SC(1), R.r2, R.r0);
  c.launched();
  if (do_res) {
    k_prep_LT<T><<<dim3(static_cast<unsigned>((vv + 31) / 32), static_cast<unsigned>(P.Kj / 32)), dim3(32, 8), 0,
                   st>>>(sy.L_vv, nj, vv, v, c.adjoint ? 1 : 0, X.LT, P.Kj, X.LT_piece, X.SC(0));
    c.launched();
  }
  if (do_den) {
    k_prep_LN<T><<<2048, 256, 0, st>>>(sy.L_vv, nj, v, vp, X.LN, X.LN_piece, X.SC(0));
    c.launched();
    c.cuda(cudaMemsetAsync(X.tpT, 0, mat_bytes(P.prec, P.Pvp, P.Kop), st));
    k_transpose<T, Path<T>::NP><<<dim3(static_cast<unsigned>((P.Pvp + 31) / 32), static_cast<unsigned>((P.Pop + 31) / 32)),
                                  dim3(32, 8), 0, st>>>(X.tp, P.Pop, P.Pvp, P.Kvp, X.tp_piece, X.tpT, P.Kop, X.tpT_piece);
    c.launched();
    c.cuda(cudaMemsetAsync(X.bp, 0, mat_bytes(P.prec, P.Pvp, P.Kop), st));
    if (minus) {
      c.cuda(cudaMemsetAsync(X.tmT, 0, mat_bytes(P.prec, P.Pvm, P.Kom), st));
      k_transpose<T, Path<T>::NP><<<dim3(static_cast<unsigned>((P.Pvm + 31) / 32), static_cast<unsigned>((P.Pom + 31) / 32)),
                                    dim3(32, 8), 0, st>>>(X.tm, P.Pom, P.Pvm, P.Kvm, X.tm_piece, X.tmT, P.Kom, X.tmT_piece);
      c.launched();
      c.cuda(cudaMemsetAsync(X.bm, 0, mat_bytes(P.prec, P.Pvp, P.Kom), st));
    }
    for (const PBlock& b : P.pbs) {
      k_pack_tbar<T><<<static_cast<unsigned>(b.npairs), 128, 0, st>>>(sy.tbar2, o, v, b.a0, b.b0, b.nb, b.diag,
                                                                     b.pair_off, X.bp, P.Kop, X.bp_piece, X.bm, P.Kom,
                                                                     X.bm_piece, minus, X.SC(2));
      c.launched();
    }
    c.cuda(cudaMemsetAsync(X.Dacc, 0, static_cast<size_t>(nj) * vv * 8, st));
  }
  // a shard writes the E partials of its own pair blocks only: the others count as zero
  if (!R.subset.empty()) c.cuda(cudaMemsetAsync(X.epart, 0, static_cast<size_t>(P.n_epart) * 8, st));
}

// The pair blocks of one wave (at most one per system, each with its own
// scratch slot) through the two independent chains of a pair block, each
// enqueued on its own stream so that one chain's memory-bound passes run
// beside the other chain's contractions:
//   residual chain: g-build -> g+- pack -> ladder +- -> Omega unpack (and E partials)
//   density chain:  Gamma+- -> slab unpack -> D slabs
// Each chain has one grouped contraction launch per step for all blocks of the
// wave.  The chains use disjoint scratch (G, g+-, Omega+- vs Gamma+-, slabs).
template <typename T>
static void wave_residual(const std::vector<Item>& items, bool do_E, Ctx& c) {
  using S = typename Path<T>::S;
  cudaStream_t st = c.st;
  auto K = [](const Item& it, size_t off) { return off ? it.slot.part[1] + off : nullptr; };
  auto Q = [](const Item& it, size_t off) { return off ? it.slot.part[0] + off : nullptr; };
  std::vector<Gm> gb, lad;
  for (const Item& it : items) {
    const Plan& P = it.r->P;
    const Ptrs<T> X(*it.r);
    const PBlock& b = P.pbs[it.ib];
    const int v = P.v;
    const int64_t M = static_cast<int64_t>(b.na) * v, N = static_cast<int64_t>(b.nb) * v;
    // g-build: G[(b_l,d)][(a_l,c)] = sum_J L^J_ac L^J_bd  (diagonal block: only a <= b is read)
    gb.push_back({X.LT + static_cast<int64_t>(b.a0) * v * P.Kj, P.Kj, M, P.Kj, X.LT_piece,
                  X.LT + static_cast<int64_t>(b.b0) * v * P.Kj, P.Kj, N, P.Kj, X.LT_piece,
                  M, N, P.Kj, K(it, P.k_G), M, false, X.SC(0), X.SC(0), b.diag ? v : 0});
  }
  run_gemms<T>(gb.data(), static_cast<int>(gb.size()), c);
  if (c.err) return;  // nothing more is launched after a refused or failed launch
  for (const Item& it : items) {
    const Plan& P = it.r->P;
    const Ptrs<T> X(*it.r);
    const PBlock& b = P.pbs[it.ib];
    const unsigned ntp = static_cast<unsigned>(P.nt * (P.nt + 1) / 2);
    k_pack_g<T, S><<<dim3(ntp, static_cast<unsigned>(b.npairs)), dim3(32, 8), 0, st>>>(
        reinterpret_cast<const S*>(K(it, P.k_G)), static_cast<int64_t>(b.na) * P.v, P.v, b.a0, b.b0, b.nb, b.diag,
        P.nt, reinterpret_cast<T*>(Q(it, P.k_gp)), P.Kvp, P.maxpairs * P.Kvp, reinterpret_cast<T*>(Q(it, P.k_gm)),
        P.Kvm, P.maxpairs * P.Kvm, P.minus, X.SC(3));
    c.launched();
    // ladder: Omega^pm[p][pr] = sum_k g^pm[pr][k] tau^pm[p][k]
    // (the g+- maps end at the last virtual pair: columns up to the padded K read as zero)
    lad.push_back({Q(it, P.k_gp), P.Kvp, b.npairs, P.Pvp, P.maxpairs * P.Kvp, X.tp, P.Kvp, P.Pop, P.Kvp, X.tp_piece,
                   b.npairs, P.Pop, P.Kvp, K(it, P.k_Op), P.ldO, false, X.SC(3), X.SC(1)});
    if (P.minus)
      lad.push_back({Q(it, P.k_gm), P.Kvm, b.npairs, P.Pvm, P.maxpairs * P.Kvm, X.tm, P.Kvm, P.Pom, P.Kvm,
                     X.tm_piece, b.npairs, P.Pom, P.Kvm, K(it, P.k_Om), P.ldO, false, X.SC(3), X.SC(1)});
  }
  run_gemms<T>(lad.data(), static_cast<int>(lad.size()), c);
  if (c.err) return;
  for (const Item& it : items) {
    const Plan& P = it.r->P;
    const Ptrs<T> X(*it.r);
    const PBlock& b = P.pbs[it.ib];
    const int64_t o2 = static_cast<int64_t>(P.o) * P.o;
    k_unpack_omega<S><<<static_cast<unsigned>(o2), 256, 0, st>>>(
        reinterpret_cast<const S*>(K(it, P.k_Op)), reinterpret_cast<const S*>(K(it, P.k_Om)), P.ldO, P.o, P.v, b.a0,
        b.b0, b.nb, b.diag, b.npairs, P.minus, it.r->omega, it.r->sy->tbar2,
        do_E ? X.epart + static_cast<int64_t>(it.ib) * o2 : nullptr);
    c.launched();
  }
}

template <typename T>
static void wave_density(const std::vector<Item>& items, Ctx& c) {
  using S = typename Path<T>::S;
  cudaStream_t st = c.st;
  auto K = [](const Item& it, size_t off) { return off ? it.slot.part[3] + off : nullptr; };
  auto Q = [](const Item& it, size_t off) { return off ? it.slot.part[2] + off : nullptr; };
  std::vector<Gm> gam, den;
  for (const Item& it : items) {
    const Plan& P = it.r->P;
    const Ptrs<T> X(*it.r);
    const PBlock& b = P.pbs[it.ib];
    // Gamma'^pm[pr][k] = sum_p tau^pm^T[k][p] tbar^pm[pr][p]
    gam.push_back({X.tpT, P.Kop, P.Pvp, P.Kop, X.tpT_piece, X.bp + b.pair_off * P.Kop, P.Kop, b.npairs, P.Kop,
                   X.bp_piece, P.Pvp, b.npairs, P.Kop, K(it, P.k_Gp), P.Kvp, false, X.SC(1), X.SC(2)});
    if (P.minus)
      gam.push_back({X.tmT, P.Kom, P.Pvm, P.Kom, X.tmT_piece, X.bm + b.pair_off * P.Kom, P.Kom, b.npairs, P.Kom,
                     X.bm_piece, P.Pvm, b.npairs, P.Kom, K(it, P.k_Gm), P.Kvm, false, X.SC(1), X.SC(2)});
  }
  run_gemms<T>(gam.data(), static_cast<int>(gam.size()), c);
  if (c.err) return;
  for (const Item& it : items) {
    const Plan& P = it.r->P;
    const Ptrs<T> X(*it.r);
    const PBlock& b = P.pbs[it.ib];
    const int v = P.v, vp = P.vp, nj = P.nj;
    const int64_t vv = static_cast<int64_t>(v) * v, gt_piece = P.maxrows * P.ldt;
    const unsigned ntp = static_cast<unsigned>(P.nt * (P.nt + 1) / 2);
    k_unpack_gamma<T, S><<<dim3(ntp, static_cast<unsigned>(b.npairs)), dim3(32, 8), 0, st>>>(
        reinterpret_cast<const S*>(K(it, P.k_Gp)), reinterpret_cast<const S*>(K(it, P.k_Gm)), P.Kvp, P.Kvm, v, vp,
        b.a0, b.b0, b.nb, b.diag, P.nt, P.minus, reinterpret_cast<T*>(Q(it, P.k_Gt)), P.ldt, gt_piece,
        reinterpret_cast<T*>(Q(it, P.k_Gb)), P.ldt, gt_piece, X.SC(4));
    c.launched();
    // D^J_(x,c) += sum_(y,d) Gamma[(x,c)][(y,d)] L^J_yd  (top and, off the diagonal, bottom)
    // (the slab maps end at the block's last column: the rest of the padded K reads as zero)
    const int64_t Mt = static_cast<int64_t>(b.na) * v, Kt = rup(static_cast<int64_t>(b.nb) * vp, 64);
    const int64_t Mb = static_cast<int64_t>(b.nb) * v, Kb = rup(static_cast<int64_t>(b.na) * vp, 64);
    den.push_back({Q(it, P.k_Gt), P.ldt, Mt, static_cast<int64_t>(b.nb) * vp, gt_piece,
                   X.LN + static_cast<int64_t>(b.b0) * vp, static_cast<int64_t>(v) * vp, nj,
                   static_cast<int64_t>(v - b.b0) * vp, X.LN_piece, Mt, nj, Kt, X.Dacc + static_cast<int64_t>(b.a0) * v,
                   vv, true, X.SC(4), X.SC(0)});
    if (!b.diag)
      den.push_back({Q(it, P.k_Gb), P.ldt, Mb, static_cast<int64_t>(b.na) * vp, gt_piece,
                     X.LN + static_cast<int64_t>(b.a0) * vp, static_cast<int64_t>(v) * vp, nj,
                     static_cast<int64_t>(v - b.a0) * vp, X.LN_piece, Mb, nj, Kb,
                     X.Dacc + static_cast<int64_t>(b.b0) * v, vv, true, X.SC(4), X.SC(0)});
  }
  run_gemms<T>(den.data(), static_cast<int>(den.size()), c);
}

// Once per system and call, after its last pair block: D to FP64, E summed.
template <typename T>
static void finish_system(const SysRun& R, bool do_res, bool do_den, bool do_E, Ctx& c) {
  const Plan& P = R.P;
  const Ptrs<T> X(R);
  const int64_t vv = static_cast<int64_t>(P.v) * P.v;
  if (do_den && Path<T>::mixed) {
    k_ff_to_f64<<<4096, 256, 0, c.st>>>(reinterpret_cast<const float2*>(X.Dacc), R.D, static_cast<int64_t>(P.nj) * vv);
    c.launched();
  }
  if (do_E && do_res) {
    k_sum_final<<<1, 1024, 0, c.st>>>(X.epart, static_cast<int64_t>(P.pbs.size()) * P.o * P.o, R.E);
    c.launched();
  }
}

// Counted flops of one pair block (g-build, ladder, Gamma, D): the scheduling weight.
static double block_weight(const Plan& P, const PBlock& b) {
  const double p = static_cast<double>(b.npairs), v2 = static_cast<double>(P.v) * P.v;
  const double lad = 2.0 * p * (static_cast<double>(P.Pvp) * P.Pop + static_cast<double>(P.Pvm) * P.Pom);
  const double rows = b.diag ? static_cast<double>(b.na) * b.na : 2.0 * b.na * b.nb;
  return 2.0 * p * v2 * P.nj + 2.0 * lad + 2.0 * P.nj * v2 * rows;
}

// The density chain's stream: one extra stream per device, created on first
// use with that device current and kept until the process exits, forked from
// and joined back to the caller's stream with two events.  A call that uses
// it holds g_side_mu while it enqueues, so that two host threads never
// interleave their forks and joins.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static std::mutex g_side_mu;
static SideStream g_side[64];

static int side_stream(SideStream*& out) {  // caller holds g_side_mu
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CC_ERR_DEVICE;
  SideStream& ss = g_side[dev];
  if (!ss.s) {
    SideStream n;
    cudaError_t e = cudaStreamCreateWithFlags(&n.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&n.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&n.join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      note_cuda(e);
      return CC_ERR_CUDA;
    }
    ss = n;
  }
  out = &ss;
  return CC_OK;
}

// All systems of a call.  Back to back: each system's pair blocks in order
// through one slot.  Batched: every system prepared first, then waves that
// take the next pair block of each of the (up to kBatchSlots) systems with
// the most work left, so each grouped launch carries the tiles of many
// systems.  Either way a system's pair blocks run in their own order, so its
// D accumulates in the same order and the results are the same bits.  With
// both chains to run, the density chain goes to the side stream (context cd)
// between a fork after the preparation and a join before the finish.
template <typename T>
static void run_all(std::vector<SysRun>& R, const std::vector<Slot>& slots, const size_t* part_bytes, bool batched,
                    bool do_res, bool do_den, bool do_E, Ctx& c, Ctx& cd, const SideStream* side) {
  // The D contraction reads the padding columns inside the Gamma slabs (virtual indices v .. vp-1 of
  // each row block) against zeros of L, which is only harmless if those columns hold finite values:
  // the operand-piece part of every slot starts zeroed, and only piece values (finite) are ever
  // written there, whichever system of the call uses the slot.  (The float-float scratch lives in
  // the other part of the slot, so its bytes are never read as pieces.)
  for (const Slot& sl : slots) {
    c.cuda(cudaMemsetAsync(sl.part[0], 0, part_bytes[0], c.st));
    c.cuda(cudaMemsetAsync(sl.part[2], 0, part_bytes[2], c.st));
  }
  Ctx& dc = side ? cd : c;
  auto fork = [&] {
    if (!side) return;
    c.cuda(cudaEventRecord(side->fork, c.st));
    c.cuda(cudaStreamWaitEvent(side->s, side->fork, 0));
  };
  auto join = [&] {
    if (!side) return;
    c.cuda(cudaEventRecord(side->join, side->s));
    c.cuda(cudaStreamWaitEvent(c.st, side->join, 0));
  };
  auto wave = [&](const std::vector<Item>& items) {
    if (do_res && !c.err) wave_residual<T>(items, do_E, c);
    if (do_den && !dc.err) wave_density<T>(items, dc);
  };
  if (!batched) {
    for (SysRun& r : R) {
      if (c.err || dc.err) break;
      prep_system<T>(r, do_res, do_den, c);
      fork();
      if (r.subset.empty()) {
        for (size_t ib = 0; ib < r.P.pbs.size() && !c.err && !dc.err; ++ib) wave({Item{&r, ib, slots[0]}});
      } else {
        for (size_t k = 0; k < r.subset.size() && !c.err && !dc.err; ++k) wave({Item{&r, r.subset[k], slots[0]}});
      }
      join();  // always: the caller's stream must not run ahead of the side stream's work
      if (!c.err && !dc.err) finish_system<T>(r, do_res, do_den, do_E, c);
    }
  } else {
    for (SysRun& r : R) {
      prep_system<T>(r, do_res, do_den, c);
      r.next = 0;
      r.left = 0.0;
      for (const PBlock& b : r.P.pbs) r.left += block_weight(r.P, b);
    }
    fork();
    std::vector<SysRun*> order;
    while (!c.err && !dc.err) {
      order.clear();
      for (SysRun& r : R)
        if (r.next < r.P.pbs.size()) order.push_back(&r);
      if (order.empty()) break;
      std::stable_sort(order.begin(), order.end(), [](const SysRun* a, const SysRun* b) { return a->left > b->left; });
      if (order.size() > slots.size()) order.resize(slots.size());
      std::vector<Item> items;
      for (size_t k = 0; k < order.size(); ++k) {
        SysRun* r = order[k];
        items.push_back(Item{r, r->next, slots[k]});
        r->left -= block_weight(r->P, r->P.pbs[r->next]);
        ++r->next;
      }
      wave(items);
    }
    join();
    if (!c.err && !dc.err)
      for (SysRun& r : R) finish_system<T>(r, do_res, do_den, do_E, c);
  }
  if (!c.err) c.err = dc.err;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static int check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_DEVICE;
  int maj = 0, min_ = 0;
  if (cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return CC_ERR_DEVICE;
  if (cudaDeviceGetAttribute(&min_, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return CC_ERR_DEVICE;
  return (maj == 10 && min_ == 3) ? CC_OK : CC_ERR_DEVICE;
}

static bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

static int validate(const cc_ladder_system* sys, int n_sys, bool need_tbar) {
  if (!sys || n_sys < 1) return CC_ERR_ARG;
  for (int i = 0; i < n_sys; ++i) {
    const cc_ladder_system& s = sys[i];
    if (s.o < 1 || s.v < 1 || s.nj < 1) return CC_ERR_ARG;
    if (!s.L_vv || !s.t2) return CC_ERR_ARG;
    if (need_tbar && !s.tbar2) return CC_ERR_ARG;
    if (!aligned8(s.L_vv) || !aligned8(s.t2) || !aligned8(s.t1) || !aligned8(s.tbar2) || !aligned8(s.eps))
      return CC_ERR_ARG;
  }
  return CC_OK;
}

// Workspace bytes.  Back to back (which without CC_WS_BATCH): the header, one
// system region and one scratch slot, each the largest over the systems.
// Batched (CC_WS_BATCH): the header, every system's own region, and
// min(n_sys, kBatchSlots) slots.  0 on invalid input.
static size_t ws_need(const cc_ladder_system* sys, int n_sys, int prec, int which) {
  size_t sys_max = 0, sys_sum = 0, part_max[4] = {0, 0, 0, 0};
  for (int i = 0; i < n_sys; ++i) {
    Plan P;
    if (!make_plan(sys[i], prec, which, P)) return 0;
    sys_max = std::max(sys_max, P.sys_bytes);
    sys_sum += P.sys_bytes;
    for (int q = 0; q < 4; ++q) part_max[q] = std::max(part_max[q], P.part[q]);
  }
  const size_t slot_max = part_max[0] + part_max[1] + part_max[2] + part_max[3];
  if (which & CC_WS_BATCH)
    return kStatusBytes + sys_sum + static_cast<size_t>(std::min(n_sys, kBatchSlots)) * slot_max;
  return kStatusBytes + sys_max + slot_max;
}

static int run(const cc_ladder_system* sys, int n_sys, double* const* omega, double* const* D, double* E,
               int prec, int which, bool res, bool den, bool want_E, void* ws, size_t ws_bytes, void* stream,
               bool adjoint = false, const double* const* es_r2 = nullptr, const double* es_r0 = nullptr,
               bool clear_status = true, const std::vector<size_t>* subset = nullptr) {
  if (prec != CC_PREC_FP64 && prec != CC_PREC_MIXED && prec != CC_PREC_FP16X2) return CC_ERR_ARG;
  int rc = validate(sys, n_sys, den || want_E || adjoint);
  if (rc) return rc;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  for (int i = 0; i < n_sys; ++i) {
    if (res && omega && !omega[i] && !want_E) return CC_ERR_ARG;
    if (res && omega && omega[i] && !aligned8(omega[i])) return CC_ERR_ARG;
    if (den && (!D || !D[i] || !aligned8(D[i]))) return CC_ERR_ARG;
  }
  if (want_E && (!E || !aligned8(E))) return CC_ERR_ARG;
  if ((rc = check_device())) return rc;
  const size_t need = ws_need(sys, n_sys, prec, which);
  if (!need) return CC_ERR_ARG;
  if (ws_bytes < need) return CC_ERR_WORKSPACE;
  const bool batched = n_sys > 1 && !subset && ws_bytes >= ws_need(sys, n_sys, prec, which | CC_WS_BATCH);
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  c.status = reinterpret_cast<Status*>(ws);
  c.queue = reinterpret_cast<int*>(static_cast<char*>(ws) + kQueueOffset);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.adjoint = adjoint;
  // every call starts from a clear status word; cc_ladder_status() reads it
  if (clear_status) c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), c.st));
  std::vector<SysRun> R(n_sys);
  char* w = static_cast<char*>(ws);
  size_t cur = kStatusBytes, sys_max = 0, part_max[4] = {0, 0, 0, 0};
  for (int i = 0; i < n_sys; ++i) {
    SysRun& r = R[i];
    r.sy = &sys[i];
    make_plan(sys[i], prec, which, r.P);
    r.omega = (res && omega) ? omega[i] : nullptr;
    r.D = den ? D[i] : nullptr;
    r.E = want_E ? E + i : nullptr;
    r.r2 = es_r2 ? es_r2[i] : nullptr;
    r.r0 = es_r0 ? es_r0[i] : 1.0;
    if (subset) {
      for (size_t ib : *subset)
        if (ib >= r.P.pbs.size()) return CC_ERR_ARG;
      r.subset = *subset;
    }
    r.base = w + (batched ? cur : kStatusBytes);
    cur += r.P.sys_bytes;
    sys_max = std::max(sys_max, r.P.sys_bytes);
    for (int q = 0; q < 4; ++q) part_max[q] = std::max(part_max[q], r.P.part[q]);
  }
  const size_t slot_bytes = part_max[0] + part_max[1] + part_max[2] + part_max[3];
  std::vector<Slot> slots;
  char* first = batched ? w + cur : w + kStatusBytes + sys_max;
  for (int k = 0; k < (batched ? std::min(n_sys, kBatchSlots) : 1); ++k) {
    Slot sl;
    char* at_ = first + static_cast<size_t>(k) * slot_bytes;
    for (int q = 0; q < 4; ++q) {
      sl.part[q] = at_;
      at_ += part_max[q];
    }
    slots.push_back(sl);
  }
  // with both chains to run, the density chain gets the side stream and its own tile counter
  std::unique_lock<std::mutex> lk(g_side_mu, std::defer_lock);
  SideStream* side = nullptr;
  Ctx cd = c;
  if (res && den) {
    lk.lock();
    if (const int rc2 = side_stream(side)) return rc2;
    cd.st = side->s;
    cd.queue = reinterpret_cast<int*>(static_cast<char*>(ws) + kQueueOffset + sizeof(int));
  }
  if (prec == CC_PREC_MIXED)
    run_all<__nv_bfloat16>(R, slots, part_max, batched, res, den, want_E, c, cd, side);
  else if (prec == CC_PREC_FP16X2)
    run_all<__half>(R, slots, part_max, batched, res, den, want_E, c, cd, side);
  else
    run_all<double>(R, slots, part_max, batched, res, den, want_E, c, cd, side);
  return c.err;
}

// ---------------------------------------------------------------------------
// doubles amplitude iteration (MP2-like driver + ladder + Jacobi step)
// ---------------------------------------------------------------------------
// driver workspace: status header, L_ov K-major in the operand format, G output
struct DriverPlan {
  int64_t ov, Kj;
  size_t o_LT, o_G, total;
};
static DriverPlan driver_plan(int o, int v, int nj, int prec) {
  DriverPlan d;
  d.ov = static_cast<int64_t>(o) * v;
  d.Kj = rup(nj, 64);
  const int op = prec == CC_PREC_FP64 ? CC_PREC_FP64 : CC_PREC_MIXED;  // split BF16 for every split path
  d.o_LT = kStatusBytes;
  d.o_G = d.o_LT + rup(static_cast<int64_t>(mat_bytes(op, d.ov, d.Kj)), 256);
  d.total = d.o_G + rup(d.ov * d.ov * 8, 256);
  return d;
}

template <typename T>
static int run_driver(int o, int v, int nj, const double* L_ov, double* g, const DriverPlan& d, char* ws,
                      cudaStream_t st) {
  using S = typename Path<T>::S;
  Ctx c;
  c.st = st;
  c.status = reinterpret_cast<Status*>(ws);
  c.queue = reinterpret_cast<int*>(static_cast<char*>(ws) + kQueueOffset);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), st));
  T* LT = at<T>(ws, d.o_LT);
  const int64_t piece = d.ov * d.Kj;
  k_prep_LT<T><<<dim3(static_cast<unsigned>((d.ov + 31) / 32), static_cast<unsigned>(d.Kj / 32)), dim3(32, 8), 0,
                 st>>>(L_ov, nj, d.ov, v, 0, LT, d.Kj, piece, nullptr);
  c.launched();
  S* G = at<S>(ws, d.o_G);
  const Gm gm = {LT, d.Kj, d.ov, d.Kj, piece, LT, d.Kj, d.ov, d.Kj, piece, d.ov, d.ov, d.Kj, G, d.ov, false};
  run_gemms<T>(&gm, 1, c);
  k_driver_to_t2<S><<<4096, 256, 0, st>>>(G, o, v, g);
  c.launched();
  return c.err;
}

static size_t iterate_need(const cc_ladder_system* sys, int prec, size_t* res_bytes) {
  const size_t r = ws_need(sys, 1, prec, CC_WS_RESIDUAL);
  if (!r) return 0;
  const size_t n = static_cast<size_t>(sys->o) * sys->o * sys->v * sys->v * 8;
  *res_bytes = static_cast<size_t>(rup(static_cast<int64_t>(r), 256));
  return *res_bytes + 2 * static_cast<size_t>(rup(static_cast<int64_t>(n), 256)) + 1024 * 8;
}

// ---------------------------------------------------------------------------
// ground-state OV^3 contributions to the three-index intermediates
// ---------------------------------------------------------------------------
struct Ov3Plan {
  int64_t ov, Kov;
  size_t o_P, o_B, o_G, o_Y, total;
};
static Ov3Plan ov3_plan(int o, int v, int nj, int prec) {
  Ov3Plan d;
  d.ov = static_cast<int64_t>(o) * v;
  d.Kov = rup(d.ov, 64);
  const int op = prec == CC_PREC_FP64 ? CC_PREC_FP64 : CC_PREC_MIXED;
  d.o_P = kStatusBytes;
  d.o_B = d.o_P + rup(static_cast<int64_t>(mat_bytes(op, d.ov, d.Kov)), 256);
  d.o_G = d.o_B + rup(static_cast<int64_t>(mat_bytes(op, nj, d.Kov)), 256);
  d.o_Y = d.o_G + rup(static_cast<int64_t>(nj) * d.ov * 8, 256);
  d.total = d.o_Y + rup(static_cast<int64_t>(nj) * d.ov * 8, 256);
  return d;
}

// W_ab^K = R0 sum_m L^a_m Y~^K_bm,  Y~^K_bm = sum_ic t~^cb_im L^K_ic
// W_ic^K = R0 sum_mb t~^cb_im O^K_bm, O^K_bm = sum_a L^a_m L^K_ab
// The t~ matrix P[(i,c)][(m,b)] is symmetric for pair-symmetric t2, so it is
// the A operand of both (o v) x N_J contractions.
template <typename T>
static int run_ov3(int o, int v, int nj, const double* L_vv, const double* L_ov, const double* t2,
                   const double* tbar1, double R0, double* W_vv, double* W_ov, const Ov3Plan& d, char* ws,
                   cudaStream_t st) {
  using S = typename Path<T>::S;
  Ctx c;
  c.st = st;
  c.status = reinterpret_cast<Status*>(ws);
  c.queue = reinterpret_cast<int*>(static_cast<char*>(ws) + kQueueOffset);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), st));
  T* P = at<T>(ws, d.o_P);
  T* B = at<T>(ws, d.o_B);
  S* G = at<S>(ws, d.o_G);
  double* Y = at<double>(ws, d.o_Y);
  const int64_t p_piece = d.ov * d.Kov, b_piece = static_cast<int64_t>(nj) * d.Kov;
  const int64_t nov = static_cast<int64_t>(nj) * d.ov;
  const unsigned grid_e = static_cast<unsigned>(std::min<int64_t>(4096, (nov + 255) / 256));
  k_pack_pairmat<T><<<static_cast<unsigned>(d.ov), 256, 0, st>>>(t2, o, v, 2.0, -1.0, P, d.Kov, p_piece);
  k_pack_rows<T><<<4096, 256, 0, st>>>(L_ov, nj, d.ov, B, d.Kov, b_piece);
  c.launched(2);
  const Gm g1 = {P, d.Kov, d.ov, d.Kov, p_piece, B, d.Kov, nj, d.Kov, b_piece, d.ov, nj, d.Kov, G, d.ov, false};
  run_gemms<T>(&g1, 1, c);  // G[K][(m,b)] = Y~^K_bm
  k_to_f64_scaled<S><<<grid_e, 256, 0, st>>>(G, Y, nov, 1.0);
  c.launched();
  // W_vv[K][a][b] = R0 sum_m tbar1[m][a] Y[K][m][b]
  const int64_t vv = static_cast<int64_t>(v) * v;
  c.check(batched_gemm_f64({v, v, o, nj, tbar1, 1, v, Y, d.ov, v, 1, nullptr, 0, 0, 0, R0, W_vv, vv, v, 1}, st));
  // O[K][m][b] = sum_a tbar1[m][a] L_vv[K][a][b]   (into Y, whose contents are used up)
  c.check(batched_gemm_f64({o, v, v, nj, tbar1, v, 1, L_vv, vv, v, 1, nullptr, 0, 0, 0, 1.0, Y, d.ov, v, 1}, st));
  k_pack_rows<T><<<4096, 256, 0, st>>>(Y, nj, d.ov, B, d.Kov, b_piece);
  c.launched();
  const Gm g2 = {P, d.Kov, d.ov, d.Kov, p_piece, B, d.Kov, nj, d.Kov, b_piece, d.ov, nj, d.Kov, G, d.ov, false};
  run_gemms<T>(&g2, 1, c);  // G[K][(i,c)] = W_ic^K / R0
  k_to_f64_scaled<S><<<grid_e, 256, 0, st>>>(G, W_ov, nov, R0);
  c.launched();
  return c.err;
}

// Excited state, the d_abci block: d_abci = L_ji^ac R_j^b.
//   X^K_aj = sum_ic L_ji^ac L^K_ic,  W_ab^K = sum_j R_j^b X^K_aj
//   P^K_aj = sum_b R_j^b L^K_ab,     W_ci^K = sum_aj L_ji^ac P^K_aj
// The matrix Q[(j,a)][(i,c)] = L_ji^ac is symmetric for pair-symmetric L2 and
// is the A operand of both (o v) x N_J contractions, as t~ is in the ground state.
template <typename T>
static int run_ov3_es_abci(int o, int v, int nj, const double* L_vv, const double* L_ov, const double* L2,
                           const double* R1, double* W_vv, double* W_vo, const Ov3Plan& d, char* ws,
                           cudaStream_t st) {
  using S = typename Path<T>::S;
  Ctx c;
  c.st = st;
  c.status = reinterpret_cast<Status*>(ws);
  c.queue = reinterpret_cast<int*>(static_cast<char*>(ws) + kQueueOffset);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), st));
  T* P = at<T>(ws, d.o_P);
  T* B = at<T>(ws, d.o_B);
  S* G = at<S>(ws, d.o_G);
  double* X = at<double>(ws, d.o_Y);
  const int64_t p_piece = d.ov * d.Kov, b_piece = static_cast<int64_t>(nj) * d.Kov;
  const int64_t nov = static_cast<int64_t>(nj) * d.ov, vv = static_cast<int64_t>(v) * v;
  const unsigned grid_e = static_cast<unsigned>(std::min<int64_t>(4096, (nov + 255) / 256));
  k_pack_pairmat<T><<<static_cast<unsigned>(d.ov), 256, 0, st>>>(L2, o, v, 1.0, 0.0, P, d.Kov, p_piece);
  k_pack_rows<T><<<4096, 256, 0, st>>>(L_ov, nj, d.ov, B, d.Kov, b_piece);
  c.launched(2);
  const Gm g1 = {P, d.Kov, d.ov, d.Kov, p_piece, B, d.Kov, nj, d.Kov, b_piece, d.ov, nj, d.Kov, G, d.ov, false};
  run_gemms<T>(&g1, 1, c);  // G[K][(j,a)] = X^K_aj
  k_to_f64_scaled<S><<<grid_e, 256, 0, st>>>(G, X, nov, 1.0);
  c.launched();
  // W_vv[K][a][b] = sum_j R1[j][b] X[K][j][a]: rows b, columns a, stored transposed
  c.check(batched_gemm_f64({v, v, o, nj, R1, 1, v, X, d.ov, v, 1, nullptr, 0, 0, 0, 1.0, W_vv, vv, 1, v}, st));
  // P[K][j][a] = sum_b R1[j][b] L_vv[K][a][b]   (into X, whose contents are used up)
  c.check(batched_gemm_f64({o, v, v, nj, R1, v, 1, L_vv, vv, 1, v, nullptr, 0, 0, 0, 1.0, X, d.ov, v, 1}, st));
  k_pack_rows<T><<<4096, 256, 0, st>>>(X, nj, d.ov, B, d.Kov, b_piece);
  c.launched();
  const Gm g2 = {P, d.Kov, d.ov, d.Kov, p_piece, B, d.Kov, nj, d.Kov, b_piece, d.ov, nj, d.Kov, G, d.ov, false};
  run_gemms<T>(&g2, 1, c);  // G[K][(i,c)] = W_ci^K
  k_to_f64_scaled<S><<<grid_e, 256, 0, st>>>(G, W_vo, nov, 1.0);
  c.launched();
  return c.err;
}

// ---------------------------------------------------------------------------
// excited-state OV^3: the d_abic block (App. A), eight terms
// ---------------------------------------------------------------------------
// d^es_abic = L^a_m t~^cb_im R0 + L^a_m (2 R~^bc_mi - R~^cb_mi) + 2 X_ab R^c_i
//           - (V_akbi + Y_akbi) R^c_k + L^ad_mk t~^bc_mi R^d_k - L^ad_mn t^bc_mn R^d_i
//           + Y~_akci R^b_k - X_ac R^b_i
// contributes W_ab^K = sum_ic d_abic L^K_ic and W_ic^K = sum_ab d_abic L^K_ab
// (L^K in place of Z^K), built term by term through three-index (and O^2V^2)
// intermediates, never the OV^3 array.  The large contractions run on the
// path's contraction engine (operands packed from strided views of the
// FP64 inputs); the thin ones (one index of length o or 1) as batched FP64
// products.
struct Ov3EsPlan {
  int64_t o, v, nj, ov, vv, oo;
  size_t o_A, o_B, o_out;
  size_t o_YP, o_O1, o_X, o_PK, o_QK, o_PKik, o_VY, o_KK, o_Wam, o_Bt, o_Kt, o_Yt, o_QT, o_P2, o_Op1;
  size_t total;
};

static Ov3EsPlan ov3es_plan(int o_, int v_, int nj_, int prec) {
  Ov3EsPlan d;
  const int64_t o = o_, v = v_, nj = nj_, ov = o * v, vv = v * v, oo = o * o;
  d.o = o; d.v = v; d.nj = nj; d.ov = ov; d.vv = vv; d.oo = oo;
  auto R = [](int64_t x) { return rup(x, 64); };
  // the largest operands (rows x padded K) and outputs (N x M) of the contraction sequence below
  const int64_t a_max = std::max({ov * R(ov), v * R(oo * v), vv * R(oo), oo * R(vv), v * R(oo), vv * R(v), v * R(vv)});
  const int64_t b_max = std::max({nj * R(ov), v * R(oo * v), ov * R(ov), nj * R(oo), nj * R(vv), vv * R(oo), nj * R(v)});
  const int64_t out_max = std::max({nj * ov, vv, ov * ov, nj * vv, nj * oo, vv * v, nj * v});
  const int op = prec == CC_PREC_FP64 ? CC_PREC_FP64 : CC_PREC_MIXED;
  size_t cur = kStatusBytes;
  auto take = [&](size_t bytes) {
    const size_t at = cur;
    cur += rup(static_cast<int64_t>(bytes), 256);
    return at;
  };
  d.o_A = take(mat_bytes(op, a_max, 1));
  d.o_B = take(mat_bytes(op, b_max, 1));
  d.o_out = take(static_cast<size_t>(out_max) * 8);
  d.o_YP = take(nj * ov * 8);
  d.o_O1 = take(nj * ov * 8);
  d.o_X = take(vv * 8);
  d.o_PK = take(nj * 8);
  d.o_QK = take(nj * 8);
  d.o_PKik = take(nj * oo * 8);
  d.o_VY = take(ov * ov * 8);
  d.o_KK = take(nj * oo * 8);
  d.o_Wam = take(ov * 8);
  d.o_Bt = take(oo * ov * 8);
  d.o_Kt = take(v * vv * 8);
  d.o_Yt = take(ov * ov * 8);
  d.o_QT = take(nj * ov * 8);
  d.o_P2 = take(nj * ov * 8);
  d.o_Op1 = take(nj * ov * 8);
  d.total = cur;
  return d;
}

template <typename T>
struct EsContract {
  using S = typename Path<T>::S;
  Ctx& c;
  char* ws;
  const Ov3EsPlan& d;
  static unsigned grid(int64_t n) { return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256))); }
  // out[n][m] = sum_k A[m][k] B[n][k], A rows m = (r1, r2) of the views a1 + a2, B rows n likewise,
  // k = (k1, k2); returns the contraction output (row pitch M)
  const S* run(View a1, View a2, int64_t MR1, int64_t MR2, View b1, View b2, int64_t NR1, int64_t NR2, int64_t K1,
               int64_t K2) {
    const int64_t M = MR1 * MR2, N = NR1 * NR2, ld = rup(K1 * K2, 64);
    T* A = at<T>(ws, d.o_A);
    T* B = at<T>(ws, d.o_B);
    S* out = at<S>(ws, d.o_out);
    k_pack_view<T><<<grid(M * ld), 256, 0, c.st>>>(a1, a2, MR1, MR2, K1, K2, A, ld, M * ld);
    k_pack_view<T><<<grid(N * ld), 256, 0, c.st>>>(b1, b2, NR1, NR2, K1, K2, B, ld, N * ld);
    c.launched(2);
    const Gm g = {A, ld, M, ld, M * ld, B, ld, N, ld, N * ld, M, N, ld, out, M, false};
    run_gemms<T>(&g, 1, c);
    return out;
  }
  // dst[n*sdn + m*sdm] (= | +=) alpha * out[n][m]
  void put(const S* src, int64_t M, int64_t N, double alpha, double* dst, int64_t sdn, int64_t sdm, bool acc) {
    k_out_view<S><<<grid(M * N), 256, 0, c.st>>>(src, M, M, N, alpha, dst, sdn, sdm, acc ? 1 : 0);
    c.launched();
  }
  void bat(const BatchedF64& g) { c.check(batched_gemm_f64(g, c.st)); }
};

template <typename T>
static int run_ov3_es_abic(int o_, int v_, int nj_, const double* L_vv, const double* L_ov, const double* tbar1,
                           const double* L2, const double* t2, double R0, const double* R1, const double* R2,
                           double* W_vv, double* W_ov, const Ov3EsPlan& d, char* ws, cudaStream_t st) {
  Ctx c;
  c.st = st;
  c.status = reinterpret_cast<Status*>(ws);
  c.queue = reinterpret_cast<int*>(ws + kQueueOffset);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), st));
  EsContract<T> E{c, ws, d};
  using S = typename Path<T>::S;
  const int o = o_, v = v_, nj = nj_;
  const int64_t ov = d.ov, vv = d.vv, oo = d.oo, ovv = static_cast<int64_t>(o) * vv;
  double* YP = at<double>(ws, d.o_YP);
  double* O1 = at<double>(ws, d.o_O1);
  double* X = at<double>(ws, d.o_X);
  double* PK = at<double>(ws, d.o_PK);
  double* QK = at<double>(ws, d.o_QK);
  double* PKik = at<double>(ws, d.o_PKik);
  double* VY = at<double>(ws, d.o_VY);
  double* KK = at<double>(ws, d.o_KK);
  double* Wam = at<double>(ws, d.o_Wam);
  double* Bt = at<double>(ws, d.o_Bt);
  double* Kt = at<double>(ws, d.o_Kt);
  double* Yt = at<double>(ws, d.o_Yt);
  double* QT = at<double>(ws, d.o_QT);
  double* P2 = at<double>(ws, d.o_P2);
  double* Op1 = at<double>(ws, d.o_Op1);
  const View none{nullptr, 0, 0, 0, 0, 0.0};
  c.cuda(cudaMemsetAsync(W_vv, 0, static_cast<size_t>(nj) * vv * 8, st));
  c.cuda(cudaMemsetAsync(W_ov, 0, static_cast<size_t>(nj) * ov * 8, st));

  // W_am = L^ad_mk R^d_k  ([m][a], one batched product per k)
  for (int k = 0; k < o && !c.err; ++k)
    E.bat({1, v, v, o, R1 + static_cast<int64_t>(k) * v, 0, 1, L2 + static_cast<int64_t>(k) * vv, ovv, 1, v,
           k ? Wam : nullptr, v, 0, 1, 1.0, Wam, v, 0, 1});
  // X_ab = L^ad_kl t^bd_kl  (M = a, N = b, K = (kl, d)), then P^K = R^c_i L^K_ic and Q^K = X_ab L^K_ab
  E.put(E.run({L2, v, 0, vv, 1, 1.0}, none, v, 1, {t2, v, 0, vv, 1, 1.0}, none, v, 1, oo, v), v, v, 1.0, X, 1, v,
        false);
  E.bat({1, 1, static_cast<int>(ov), nj, R1, 0, 1, L_ov, ov, 1, 0, nullptr, 0, 0, 0, 1.0, PK, 1, 0, 0});
  E.bat({1, 1, static_cast<int>(vv), nj, X, 0, 1, L_vv, vv, 1, 0, nullptr, 0, 0, 0, 1.0, QK, 1, 0, 0});

  // terms 1, 2 and 5: left factor (L^a_m, then W_am) times a pair matrix P[(i,c)][(m,b)] (symmetric):
  // W_ab += left[m][a] sum_ic P^cb_im L^K_ic, W_ic += sum_mb P^cb_im (sum_a left[m][a] L^K_ab)
  const int64_t Kov = rup(ov, 64);
  for (int pass = 0; pass < 2 && !c.err; ++pass) {
    T* A = at<T>(ws, d.o_A);
    T* B = at<T>(ws, d.o_B);
    const S* out = at<S>(ws, d.o_out);
    if (pass == 0)  // R0 t~ + 2 R~^bc_mi - R~^cb_mi = R0 (2 t_im - t_mi)^cb + (5 R_im - 4 R_mi)^cb
      k_pack_pairmat<T><<<static_cast<unsigned>(ov), 256, 0, st>>>(t2, o, v, 2.0 * R0, -R0, A, Kov, ov * Kov, R2,
                                                                    5.0, -4.0);
    else
      k_pack_pairmat<T><<<static_cast<unsigned>(ov), 256, 0, st>>>(t2, o, v, 2.0, -1.0, A, Kov, ov * Kov);
    c.launched();
    const double* left = pass == 0 ? tbar1 : Wam;
    k_pack_view<T><<<EsContract<T>::grid(nj * Kov), 256, 0, st>>>(View{L_ov, ov, 0, 1, 0, 1.0}, none, nj, 1, ov, 1, B,
                                                                  Kov, nj * Kov);
    c.launched();
    const Gm g1 = {A, Kov, ov, Kov, ov * Kov, B, Kov, nj, Kov, nj * Kov, ov, nj, Kov, const_cast<S*>(out), ov, false};
    run_gemms<T>(&g1, 1, c);
    E.put(out, ov, nj, 1.0, YP, ov, 1, false);                                        // YP[K][(m,b)]
    E.bat({v, v, o, nj, left, 1, v, YP, ov, v, 1, W_vv, vv, v, 1, 1.0, W_vv, vv, v, 1});
    E.bat({o, v, v, nj, left, v, 1, L_vv, vv, v, 1, nullptr, 0, 0, 0, 1.0, O1, ov, v, 1});
    k_pack_view<T><<<EsContract<T>::grid(nj * Kov), 256, 0, st>>>(View{O1, ov, 0, 1, 0, 1.0}, none, nj, 1, ov, 1, B,
                                                                  Kov, nj * Kov);
    c.launched();
    const Gm g2 = {A, Kov, ov, Kov, ov * Kov, B, Kov, nj, Kov, nj * Kov, ov, nj, Kov, const_cast<S*>(out), ov, false};
    run_gemms<T>(&g2, 1, c);
    E.put(out, ov, nj, 1.0, W_ov, ov, 1, true);
  }

  // term 3: 2 X_ab R^c_i
  E.bat({static_cast<int>(vv), 1, 1, nj, X, 1, 0, PK, 1, 0, 0, W_vv, vv, 1, 0, 2.0, W_vv, vv, 1, 0});
  E.bat({static_cast<int>(ov), 1, 1, nj, R1, 1, 0, QK, 1, 0, 0, W_ov, ov, 1, 0, 2.0, W_ov, ov, 1, 0});

  // term 4: -(V_akbi + Y_akbi) R^c_k, VY[(b,i)][(a,k)] = V + Y (two contractions over (j,c) and (l,d))
  E.put(E.run({L2, v, vv, ovv, 1, 1.0}, none, v, o, {t2, v, vv, ovv, 1, 1.0}, none, v, o, o, v), ov, ov, 1.0, VY, ov,
        1, false);
  E.put(E.run({L2, v, ovv, vv, 1, 1.0}, none, v, o, {t2, v, ovv, vv, 1, 1.0}, none, v, o, o, v), ov, ov, 1.0, VY, ov,
        1, true);
  E.bat({o, o, v, nj, R1, v, 1, L_ov, ov, 1, v, nullptr, 0, 0, 0, 1.0, PKik, oo, o, 1});        // PKik[K][k][i]
  E.put(E.run({VY, o, o * ov, ov, 1, 1.0}, none, v, v, {PKik, oo, 0, 1, o, 1.0}, none, nj, 1, o, o), vv, nj, -1.0,
        W_vv, vv, 1, true);
  E.put(E.run({VY, ov, 1, o, o * ov, 1.0}, none, o, o, {L_vv, vv, 0, v, 1, 1.0}, none, nj, 1, v, v), oo, nj, 1.0, KK,
        oo, 1, false);                                                                   // KK[K][i][k]
  E.bat({v, o, o, nj, R1, 1, v, KK, oo, 1, o, W_ov, ov, 1, v, -1.0, W_ov, ov, 1, v});

  // term 6: -B_iamn t^bc_mn with B_iamn = L^ad_mn R^d_i, one i at a time (K_i[(b,c)][a] = sum_mn B t)
  E.bat({o, v, v, static_cast<int>(oo), R1, v, 1, L2, vv, 1, v, nullptr, 0, 0, 0, 1.0, Bt, ov, v, 1});  // Bt[mn][i][a]
  for (int i = 0; i < o && !c.err; ++i) {
    E.put(E.run({Bt + static_cast<int64_t>(i) * v, 1, 0, ov, 0, 1.0}, none, v, 1, {t2, v, 1, vv, 0, 1.0}, none, v, v,
                oo, 1),
          v, vv, 1.0, Kt, v, 1, false);
    E.put(E.run({Kt, 1, vv, v, 0, 1.0}, none, v, v, {L_ov + static_cast<int64_t>(i) * v, ov, 0, 1, 0, 1.0}, none, nj,
                1, v, 1),
          vv, nj, -1.0, W_vv, vv, 1, true);
    E.put(E.run({Kt, v, 0, 1, vv, 1.0}, none, v, 1, {L_vv, vv, 0, v, 1, 1.0}, none, nj, 1, v, v), v, nj, -1.0,
          W_ov + static_cast<int64_t>(i) * v, ov, 1, true);
  }

  // term 7: Y~_akci R^b_k, Yt[(c,i)][(a,k)] = L^ea_mk t~^ec_mi (t~ = 2 t_mi - t_im)
  E.put(E.run({L2, 1, vv, ovv, v, 1.0}, none, v, o, {t2, 1, vv, ovv, v, 2.0}, {t2, 1, ovv, vv, v, -1.0}, v, o, o, v),
        ov, ov, 1.0, Yt, ov, 1, false);
  E.put(E.run({Yt, o, 1, ov, o * ov, 1.0}, none, v, o, {L_ov, ov, 0, v, 1, 1.0}, none, nj, 1, o, v), ov, nj, 1.0, QT,
        ov, 1, false);                                                                   // QT[K][a][k]
  E.bat({v, v, o, nj, R1, 1, v, QT, ov, 1, o, W_vv, vv, 1, v, 1.0, W_vv, vv, 1, v});
  E.bat({o, v, v, nj, R1, v, 1, L_vv, vv, 1, v, nullptr, 0, 0, 0, 1.0, P2, ov, v, 1});         // P2[K][k][a]
  E.put(E.run({Yt, ov, o * ov, o, 1, 1.0}, none, o, v, {P2, ov, 0, 1, v, 1.0}, none, nj, 1, v, o), ov, nj, 1.0, W_ov,
        ov, 1, true);

  // term 8: -X_ac R^b_i
  E.bat({v, o, v, nj, X, v, 1, L_ov, ov, 1, v, nullptr, 0, 0, 0, 1.0, Op1, ov, o, 1});        // Op1[K][a][i]
  E.bat({v, v, o, nj, R1, 1, v, Op1, ov, 1, o, W_vv, vv, 1, v, -1.0, W_vv, vv, 1, v});
  E.bat({v, o, v, nj, X, 1, v, P2, ov, 1, v, W_ov, ov, 1, v, -1.0, W_ov, ov, 1, v});
  return c.err;
}

}  // namespace ccl

using namespace ccl;

extern "C" {

int cc_ladder_ov3_es_abci(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov,
                          const double* L2, const double* R1, double* W_vv, double* W_vo, cc_precision p, void* ws,
                          size_t ws_bytes, void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !L_vv || !L_ov || !L2 || !R1 || !W_vv || !W_vo) return CC_ERR_ARG;
  if (!aligned8(L_vv) || !aligned8(L_ov) || !aligned8(L2) || !aligned8(R1) || !aligned8(W_vv) || !aligned8(W_vo))
    return CC_ERR_ARG;
  if (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) return CC_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  const Ov3Plan d = ov3_plan(o, v, nj, p);
  if (ws_bytes < d.total) return CC_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p == CC_PREC_FP64)
    return run_ov3_es_abci<double>(o, v, nj, L_vv, L_ov, L2, R1, W_vv, W_vo, d, static_cast<char*>(ws), st);
  return run_ov3_es_abci<__nv_bfloat16>(o, v, nj, L_vv, L_ov, L2, R1, W_vv, W_vo, d, static_cast<char*>(ws), st);
}

size_t cc_ladder_ov3_es_abic_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p) {
  if (o < 1 || v < 1 || nj < 1 || (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2)) return 0;
  return ov3es_plan(o, v, nj, p).total;
}

int cc_ladder_ov3_es_abic(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov,
                          const double* tbar1, const double* L2, const double* t2, double R0, const double* R1,
                          const double* R2, double* W_vv, double* W_ov, cc_precision p, void* ws, size_t ws_bytes,
                          void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !L_vv || !L_ov || !tbar1 || !L2 || !t2 || !R1 || !R2 || !W_vv || !W_ov)
    return CC_ERR_ARG;
  for (const void* q : {static_cast<const void*>(L_vv), static_cast<const void*>(L_ov),
                        static_cast<const void*>(tbar1), static_cast<const void*>(L2), static_cast<const void*>(t2),
                        static_cast<const void*>(R1), static_cast<const void*>(R2), static_cast<const void*>(W_vv),
                        static_cast<const void*>(W_ov)})
    if (!aligned8(q)) return CC_ERR_ARG;
  if (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) return CC_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  const Ov3EsPlan d = ov3es_plan(o, v, nj, p);
  if (ws_bytes < d.total) return CC_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p == CC_PREC_FP64)
    return run_ov3_es_abic<double>(o, v, nj, L_vv, L_ov, tbar1, L2, t2, R0, R1, R2, W_vv, W_ov, d,
                                   static_cast<char*>(ws), st);
  return run_ov3_es_abic<__nv_bfloat16>(o, v, nj, L_vv, L_ov, tbar1, L2, t2, R0, R1, R2, W_vv, W_ov, d,
                                        static_cast<char*>(ws), st);
}

size_t cc_ladder_ov3_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p) {
  if (o < 1 || v < 1 || nj < 1 || (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2)) return 0;
  return ov3_plan(o, v, nj, p).total;
}

int cc_ladder_ov3_gs(int32_t o, int32_t v, int32_t nj, const double* L_vv, const double* L_ov, const double* t2,
                     const double* tbar1, double R0, double* W_vv, double* W_ov, cc_precision p, void* ws,
                     size_t ws_bytes, void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !L_vv || !L_ov || !t2 || !tbar1 || !W_vv || !W_ov) return CC_ERR_ARG;
  if (!aligned8(L_vv) || !aligned8(L_ov) || !aligned8(t2) || !aligned8(tbar1) || !aligned8(W_vv) || !aligned8(W_ov))
    return CC_ERR_ARG;
  if (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) return CC_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  const Ov3Plan d = ov3_plan(o, v, nj, p);
  if (ws_bytes < d.total) return CC_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p == CC_PREC_FP64)
    return run_ov3<double>(o, v, nj, L_vv, L_ov, t2, tbar1, R0, W_vv, W_ov, d, static_cast<char*>(ws), st);
  return run_ov3<__nv_bfloat16>(o, v, nj, L_vv, L_ov, t2, tbar1, R0, W_vv, W_ov, d, static_cast<char*>(ws), st);
}

size_t cc_ladder_mp2_driver_workspace_size(int32_t o, int32_t v, int32_t nj, cc_precision p) {
  if (o < 1 || v < 1 || nj < 1 || (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2)) return 0;
  return driver_plan(o, v, nj, p).total;
}

int cc_ladder_mp2_driver(int32_t o, int32_t v, int32_t nj, const double* L_ov, double* g, cc_precision p, void* ws,
                         size_t ws_bytes, void* stream) {
  if (o < 1 || v < 1 || nj < 1 || !L_ov || !g || !aligned8(L_ov) || !aligned8(g)) return CC_ERR_ARG;
  if (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) return CC_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  const DriverPlan d = driver_plan(o, v, nj, p);
  if (ws_bytes < d.total) return CC_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p == CC_PREC_FP64) return run_driver<double>(o, v, nj, L_ov, g, d, static_cast<char*>(ws), st);
  return run_driver<__nv_bfloat16>(o, v, nj, L_ov, g, d, static_cast<char*>(ws), st);
}

size_t cc_ladder_iterate_workspace_size(const cc_ladder_system* sys, cc_precision p) {
  if (validate(sys, 1, false) || (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2)) return 0;
  size_t r = 0;
  return iterate_need(sys, p, &r);
}

int cc_ladder_iterate(const cc_ladder_system* sys, const double* g_drv, int n_iter, double* t2_out, double* dnorm2,
                      cc_precision p, void* ws, size_t ws_bytes, void* stream) {
  if (validate(sys, 1, false) || !sys->eps || !g_drv || !t2_out || !dnorm2 || n_iter < 1) return CC_ERR_ARG;
  if (!aligned8(g_drv) || !aligned8(t2_out) || !aligned8(dnorm2)) return CC_ERR_ARG;
  if (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) return CC_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  size_t rb = 0;
  const size_t need = iterate_need(sys, p, &rb);
  if (!need) return CC_ERR_ARG;
  if (ws_bytes < need) return CC_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  const size_t n = static_cast<size_t>(sys->o) * sys->o * sys->v * sys->v;
  const size_t nb = static_cast<size_t>(rup(static_cast<int64_t>(n * 8), 256));
  double* om = reinterpret_cast<double*>(w + rb);
  double* tmp = reinterpret_cast<double*>(w + rb + nb);
  double* part = reinterpret_cast<double*>(w + rb + 2 * nb);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double* cur = sys->t2;
  for (int k = 0; k < n_iter; ++k) {
    double* target = ((n_iter - 1 - k) % 2 == 0) ? t2_out : tmp;
    cc_ladder_system sk = *sys;
    sk.t2 = cur;
    double* omp[1] = {om};
    const int rc = run(&sk, 1, omp, nullptr, nullptr, p, CC_WS_RESIDUAL, true, false, false, ws, rb, stream, false,
                       nullptr, nullptr, k == 0);
    if (rc) return rc;
    k_jacobi<<<1024, 256, 0, st>>>(g_drv, om, cur, sys->eps, sys->o, sys->v, target, part);
    k_sum_final<<<1, 1024, 0, st>>>(part, 1024, dnorm2 + k);
    count_launch(2);
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      note_cuda(e);
      return CC_ERR_CUDA;
    }
    cur = target;
  }
  return CC_OK;
}


size_t cc_ladder_workspace_size(const cc_ladder_system* sys, int n_sys, cc_precision p, int which) {
  if (validate(sys, n_sys, false) || (p != CC_PREC_FP64 && p != CC_PREC_MIXED && p != CC_PREC_FP16X2) ||
      !(which & CC_WS_STEP) || (which & ~(CC_WS_STEP | CC_WS_BATCH)))
    return 0;
  return ws_need(sys, n_sys, p, which);
}

int cc_ladder_residual(const cc_ladder_system* sys, int n_sys, double* const* omega, cc_precision p, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!omega) return CC_ERR_ARG;
  for (int i = 0; sys && i < n_sys; ++i)
    if (!omega[i]) return CC_ERR_ARG;
  return run(sys, n_sys, omega, nullptr, nullptr, p, CC_WS_RESIDUAL, true, false, false, ws, ws_bytes, stream);
}

int cc_ladder_residual_adjoint(const cc_ladder_system* sys, int n_sys, double* const* out, cc_precision p,
                               void* ws, size_t ws_bytes, void* stream) {
  if (!out) return CC_ERR_ARG;
  for (int i = 0; sys && i < n_sys; ++i)
    if (!out[i]) return CC_ERR_ARG;
  return run(sys, n_sys, out, nullptr, nullptr, p, CC_WS_RESIDUAL, true, false, false, ws, ws_bytes, stream, true);
}

int cc_ladder_density(const cc_ladder_system* sys, int n_sys, double* const* D, cc_precision p, void* ws,
                      size_t ws_bytes, void* stream) {
  if (!D) return CC_ERR_ARG;
  return run(sys, n_sys, nullptr, D, nullptr, p, CC_WS_DENSITY, false, true, false, ws, ws_bytes, stream);
}

int cc_ladder_density_es(const cc_ladder_system* sys, int n_sys, const double* const* R2, const double* R0,
                         double* const* D, cc_precision p, void* ws, size_t ws_bytes, void* stream) {
  if (!D || !R2 || !R0 || !sys || n_sys < 1) return CC_ERR_ARG;
  for (int i = 0; i < n_sys; ++i)
    if (!R2[i] || !aligned8(R2[i])) return CC_ERR_ARG;
  return run(sys, n_sys, nullptr, D, nullptr, p, CC_WS_DENSITY, false, true, false, ws, ws_bytes, stream, false, R2,
             R0);
}

int cc_ladder_lagrangian(const cc_ladder_system* sys, int n_sys, double* E, double* const* omega_opt, cc_precision p,
                         void* ws, size_t ws_bytes, void* stream) {
  if (omega_opt == nullptr)
    return run(sys, n_sys, nullptr, nullptr, E, p, CC_WS_LAGRANGIAN, true, false, true, ws, ws_bytes, stream);
  // Omega given: plain FP64 reduction sum tbar * Omega
  int rc = validate(sys, n_sys, true);
  if (rc) return rc;
  if (!E || !aligned8(E) || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return CC_ERR_ARG;
  if ((rc = check_device())) return rc;
  if (ws_bytes < kStatusBytes + 1024 * 8) return CC_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + kStatusBytes);
  if (cudaMemsetAsync(ws, 0, sizeof(Status), st) != cudaSuccess) return CC_ERR_CUDA;
  for (int i = 0; i < n_sys; ++i) {
    if (!omega_opt[i] || !aligned8(omega_opt[i])) return CC_ERR_ARG;
    const int64_t n = static_cast<int64_t>(sys[i].o) * sys[i].o * sys[i].v * sys[i].v;
    k_dot_partial<<<1024, 256, 0, st>>>(sys[i].tbar2, omega_opt[i], n, part);
    k_sum_final<<<1, 1024, 0, st>>>(part, 1024, E + i);
    count_launch(2);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      note_cuda(e);
      return CC_ERR_CUDA;
    }
  }
  return CC_OK;
}

int cc_ladder_step(const cc_ladder_system* sys, int n_sys, double* const* omega, double* const* D, double* E,
                   cc_precision p, void* ws, size_t ws_bytes, void* stream) {
  if (!omega || !D || !E) return CC_ERR_ARG;
  for (int i = 0; sys && i < n_sys; ++i)
    if (!omega[i]) return CC_ERR_ARG;
  return run(sys, n_sys, omega, D, E, p, CC_WS_STEP, true, true, true, ws, ws_bytes, stream);
}

int cc_ladder_pair_blocks(const cc_ladder_system* sys, int32_t* count, int32_t* edge) {
  if (validate(sys, 1, false) || !count) return CC_ERR_ARG;
  Plan P;
  if (!make_plan(*sys, CC_PREC_FP64, CC_WS_STEP, P)) return CC_ERR_ARG;
  *count = static_cast<int32_t>(P.pbs.size());
  if (edge) *edge = P.s;
  return CC_OK;
}

int cc_ladder_step_blocks(const cc_ladder_system* sys, const int32_t* blocks, int n_blocks, double* omega,
                          double* D_part, double* E_part, cc_precision p, void* ws, size_t ws_bytes, void* stream) {
  if (!sys || !blocks || n_blocks < 1 || !omega || !D_part || !E_part) return CC_ERR_ARG;
  if (validate(sys, 1, true)) return CC_ERR_ARG;
  Plan P;
  if (!make_plan(*sys, CC_PREC_FP64, CC_WS_STEP, P)) return CC_ERR_ARG;
  std::vector<size_t> subset;
  std::vector<char> seen(P.pbs.size(), 0);
  for (int k = 0; k < n_blocks; ++k) {
    const int32_t b = blocks[k];
    if (b < 0 || static_cast<size_t>(b) >= P.pbs.size() || seen[b]) return CC_ERR_ARG;  // out of range or repeated
    seen[b] = 1;
    subset.push_back(static_cast<size_t>(b));
  }
  double* om[1] = {omega};
  double* Dp[1] = {D_part};
  return run(sys, 1, om, Dp, E_part, p, CC_WS_STEP, true, true, true, ws, ws_bytes, stream, false, nullptr, nullptr,
             true, &subset);
}

int cc_ladder_update(const cc_ladder_system* sys, int n_sys, double* const* omega, double* const* t2_out,
                     void* stream) {
  int rc = validate(sys, n_sys, false);
  if (rc) return rc;
  if (!omega || !t2_out) return CC_ERR_ARG;
  if ((rc = check_device())) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_sys; ++i) {
    if (!sys[i].eps || !omega[i] || !t2_out[i] || !aligned8(omega[i]) || !aligned8(t2_out[i])) return CC_ERR_ARG;
    k_update<<<1024, 256, 0, st>>>(sys[i].t2, omega[i], sys[i].eps, sys[i].o, sys[i].v, t2_out[i]);
    count_launch();
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      note_cuda(e);
      return CC_ERR_CUDA;
    }
  }
  return CC_OK;
}

int cc_ladder_scale_by(double* x, int64_t n, double factor, const double* g, void* stream) {
  if (!x || n < 1 || !aligned8(x) || !aligned8(g)) return CC_ERR_ARG;
  if (const int rc = check_device()) return rc;
  const int64_t blocks = std::min<int64_t>(4096, (n + 255) / 256);
  k_scale_by<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, factor, g);
  count_launch();
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  return CC_OK;
}

int cc_ladder_status(void* ws, void* stream) {
  if (!ws) return CC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  Status h{0, 0};
  e = cudaMemcpy(&h, ws, sizeof(Status), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  if (h.code) {
    Status z{0, 0};
    cudaMemcpy(ws, &z, sizeof(Status), cudaMemcpyHostToDevice);
  }
  return h.code;
}

int cc_ladder_debug_wait(const int* flag, long long timeout_ns, void* ws, void* stream) {
  if (!flag || !ws || timeout_ns <= 0) return CC_ERR_ARG;
  int rc = check_device();
  if (rc) return rc;
  k_debug_wait<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(flag, static_cast<unsigned long long>(timeout_ns),
                                                                reinterpret_cast<Status*>(ws));
  count_launch();
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  return CC_OK;
}

const char* cc_ladder_strerror(int code) {
  static thread_local std::string buf;
  switch (code) {
    case CC_OK: return "ok";
    case CC_ERR_ARG: return "invalid argument (NULL pointer, dimension < 1, misalignment or size limit)";
    case CC_ERR_DEVICE: return "current CUDA device is not sm_103 (GB300)";
    case CC_ERR_WORKSPACE: return "workspace smaller than cc_ladder_workspace_size()";
    case CC_ERR_TIMEOUT: return "a bounded device wait gave up (CC_ERR_TIMEOUT)";
    case CC_ERR_SIZE: return "request exceeds the fixed device scratch (at most 64 systems per no-allocation call)";
    case CC_ERR_CUDA: {
      std::lock_guard<std::mutex> lk(g_err_mu);
      buf = "CUDA error: " + g_err_text;
      return buf.c_str();
    }
    default: return "unknown error code";
  }
}

long long cc_ladder_launch_count(void) { return g_launches.load(); }

int cc_ladder_set_contraction(int kind) {
  if (kind != 0 && kind != CC_KERNEL_SINGLE && kind != CC_KERNEL_PAIR && kind != CC_KERNEL_KBLOCK_WINDOWS &&
      kind != CC_KERNEL_PAIR_KBLOCK_WINDOWS)
    return CC_ERR_ARG;
  ccl::g_tune_kernel.store(kind);
  return CC_OK;
}

int cc_ladder_set_tuning(int block_edge, int win_kblocks) {
  if (block_edge < 0 || (block_edge > 0 && (block_edge % 4 || block_edge > 256))) return CC_ERR_ARG;
  if (win_kblocks < 0 || (win_kblocks > 0 && (win_kblocks > 8 || (win_kblocks & (win_kblocks - 1)))))
    return CC_ERR_ARG;
  g_tune_block.store(block_edge);
  g_tune_win.store(win_kblocks);
  return CC_OK;
}

void cc_ladder_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = enable != 0;
  g_prof.pending.clear();
  g_prof.used = 0;
  g_prof.flops = 0.0;
  g_prof.launches = 0;
}

int cc_ladder_profile_read(double* gemm_ms, long long* gemm_launches, double* gemm_flops) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  // contraction launches of the two chains may overlap in time: the time reported is the length
  // of the union of their [start, end] intervals on a common timeline
  std::vector<std::pair<double, double>> iv;
  if (!g_prof.pending.empty()) {
    cudaEvent_t ref = g_prof.pending.front().first;
    for (auto& pr : g_prof.pending)
      if (cudaEventSynchronize(pr.second) != cudaSuccess) return CC_ERR_CUDA;
    for (auto& pr : g_prof.pending) {
      float t0 = 0.f, t1 = 0.f;
      if (cudaEventElapsedTime(&t0, ref, pr.first) != cudaSuccess) return CC_ERR_CUDA;
      if (cudaEventElapsedTime(&t1, ref, pr.second) != cudaSuccess) return CC_ERR_CUDA;
      iv.emplace_back(t0, t1);
    }
  }
  std::sort(iv.begin(), iv.end());
  double ms = 0.0, lo = 0.0, hi = 0.0;
  bool open = false;
  for (const auto& x : iv) {
    if (!open || x.first > hi) {
      if (open) ms += hi - lo;
      lo = x.first;
      hi = x.second;
      open = true;
    } else {
      hi = std::max(hi, x.second);
    }
  }
  if (open) ms += hi - lo;
  if (gemm_ms) *gemm_ms = ms;
  if (gemm_launches) *gemm_launches = g_prof.launches;
  if (gemm_flops) *gemm_flops = g_prof.flops;
  g_prof.pending.clear();
  g_prof.used = 0;
  g_prof.flops = 0.0;
  g_prof.launches = 0;
  return CC_OK;
}

}  // extern "C"
