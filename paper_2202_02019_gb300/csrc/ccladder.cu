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
static std::atomic<int> g_tune_block{0}, g_tune_win{0};
int tuned_win_kb(int dflt) {
  const int w = g_tune_win.load();
  if (w > 0) return w;
  const char* e = std::getenv("CC_WIN_KB");
  return (e && *e) ? std::max(1, std::atoi(e)) : dflt;
}

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
// P[(i,c)][(m,b)] = alpha x_im^cb + beta x_mi^cb (zero for columns past o v), split into
// the operand format; (alpha, beta) = (2, -1) gives t~ = 2 t - t^T, (1, 0) the amplitudes
template <typename T>
__global__ void k_pack_pairmat(const double* __restrict__ t2, int o, int v, double alpha, double beta,
                               T* __restrict__ P, int64_t ld, int64_t piece) {
  const int64_t ov = static_cast<int64_t>(o) * v, vv = static_cast<int64_t>(v) * v;
  const int64_t r = blockIdx.x;  // (i, c)
  const int i = static_cast<int>(r / v), c = static_cast<int>(r % v);
  for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) {
    double x = 0.0;
    if (k < ov) {
      const int m = static_cast<int>(k / v), b = static_cast<int>(k % v);
      x = alpha * t2[(static_cast<int64_t>(i) * o + m) * vv + static_cast<int64_t>(c) * v + b] +
          beta * t2[(static_cast<int64_t>(m) * o + i) * vv + static_cast<int64_t>(c) * v + b];
    }
    Store<T>::put(P, r * ld + k, piece, x, 1.f);
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
  // byte offsets into the workspace; 0 = not present (offset 0 is the status header)
  size_t o_LT = 0, o_LN = 0, o_tp = 0, o_tm = 0, o_tpT = 0, o_tmT = 0, o_bp = 0, o_bm = 0;
  size_t o_G = 0, o_gp = 0, o_gm = 0, o_Op = 0, o_Om = 0, o_Gp = 0, o_Gm = 0, o_Gt = 0, o_Gb = 0, o_E = 0;
  size_t o_D = 0;
  size_t total = 0;
};

constexpr size_t kStatusBytes = 256;

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
  size_t cur = kStatusBytes;
  auto take = [&](size_t bytes) {
    const size_t at = cur;
    cur += rup(static_cast<int64_t>(bytes), 256);
    return at;
  };
  const int pr = prec;
  P.o_tp = take(mat_bytes(pr, P.Pop, P.Kvp));
  P.o_tm = take(mat_bytes(pr, P.Pom, P.Kvm));
  if (res) {
    P.o_LT = take(mat_bytes(pr, v * v, P.Kj));
    P.o_G = take(static_cast<size_t>(P.maxrows) * P.maxrows * 8);
    P.o_gp = take(mat_bytes(pr, P.maxpairs, P.Kvp));
    P.o_gm = take(mat_bytes(pr, P.maxpairs, P.Kvm));
    P.o_Op = take(static_cast<size_t>(P.Pop) * P.ldO * 8);
    P.o_Om = take(static_cast<size_t>(P.Pom) * P.ldO * 8);
  }
  if (den) {
    P.o_LN = take(mat_bytes(pr, nj, v * P.vp));
    P.o_tpT = take(mat_bytes(pr, P.Pvp, P.Kop));
    P.o_tmT = take(mat_bytes(pr, P.Pvm, P.Kom));
    P.o_bp = take(mat_bytes(pr, P.Pvp, P.Kop));
    P.o_bm = take(mat_bytes(pr, P.Pvp, P.Kom));
    P.o_Gp = take(static_cast<size_t>(P.maxpairs) * P.Kvp * 8);
    P.o_Gm = take(static_cast<size_t>(P.maxpairs) * P.Kvm * 8);
    P.o_Gt = take(mat_bytes(pr, P.maxrows, P.ldt));
    P.o_Gb = take(mat_bytes(pr, P.maxrows, P.ldt));
    if (prec != CC_PREC_FP64) P.o_D = take(static_cast<size_t>(nj) * v * v * 8);  // float-float D
  }
  P.o_E = take(static_cast<size_t>(P.n_epart) * 8);
  P.total = cur;
  return true;
}

// ---------------------------------------------------------------------------
// execution
// ---------------------------------------------------------------------------
struct Ctx {
  cudaStream_t st;
  Status* status;
  uint64_t timeout_ns;
  bool adjoint = false;  // residual of tbar2 with L^J transposed: sum_ab tbar_ij^ab g_acbd
  const double* r2 = nullptr;  // excited-state density: the ladder doubles are r0 t2 + r2
  double r0 = 1.0;
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
static int profiled(const GemmOp& g, cudaStream_t s, F&& launch, const GemmOp* g2) {
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
    g_prof.flops += 2.0 * static_cast<double>(g.M) * static_cast<double>(g.N) * static_cast<double>(g.K);
    if (g2) g_prof.flops += 2.0 * static_cast<double>(g2->M) * static_cast<double>(g2->N) * static_cast<double>(g2->K);
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

// Launch one group of up to two contractions of the same shape class.
template <typename T>
static void run_gemms(const Gm* g, int n, Ctx& c) {
  std::vector<GemmOp> ops(n);
  for (int i = 0; i < n; ++i) {
    GemmOp& o = ops[i];
    o.A = g[i].A; o.lda = g[i].lda; o.a_rows = g[i].a_rows; o.a_cols = g[i].a_cols; o.a_piece = g[i].a_piece;
    o.B = g[i].B; o.ldb = g[i].ldb; o.b_rows = g[i].b_rows; o.b_cols = g[i].b_cols; o.b_piece = g[i].b_piece;
    o.M = g[i].M; o.N = g[i].N; o.K = g[i].K; o.out = g[i].out; o.ldo = g[i].ldo; o.tri = g[i].tri;
    o.status = c.status; o.timeout_ns = c.timeout_ns;
  }
  if (Path<T>::mixed) {
    for (int i = 0; i < n; ++i) {
      ops[i].mode = g[i].acc ? OUT_FF_ACCUM : OUT_FF_STORE;
      ops[i].pieces = Path<T>::NP;
      ops[i].scale_a = g[i].sa;
      ops[i].scale_b = g[i].sb;
    }
    c.check(profiled(ops[0], c.st, [&] { return gemm_mixed(ops.data(), n, c.st); }, n > 1 ? &ops[1] : nullptr));
  } else {
    for (int i = 0; i < n; ++i) {
      GemmOp& o = ops[i];
      o.kchunk = f64_kchunk(o.M, o.N, o.K);
      const bool split = o.kchunk < o.K;
      if (split && !g[i].acc)
        c.cuda(cudaMemsetAsync(o.out, 0, static_cast<size_t>(o.N) * o.ldo * sizeof(double), c.st));
      o.mode = (split || g[i].acc) ? OUT_F64_ATOMIC : OUT_F64_STORE;
      c.check(profiled(o, c.st, [&] { return gemm_f64(o, c.st); }, nullptr));
    }
  }
}

template <typename T>
static void run_system(const cc_ladder_system& sy, const Plan& P, char* ws, double* omega, double* D, double* E,
                       bool do_res, bool do_den, bool do_E, Ctx& c) {
  using S = typename Path<T>::S;
  const int o = P.o, v = P.v, nj = P.nj, vp = P.vp;
  const int64_t vv = static_cast<int64_t>(v) * v;
  const int minus = P.minus;
  cudaStream_t st = c.st;
  T* tp = at<T>(ws, P.o_tp);
  T* tm = at<T>(ws, P.o_tm);
  const int64_t tp_piece = P.Pop * P.Kvp, tm_piece = P.Pom * P.Kvm;

  // --- operand scales of the FP16 two-piece path (device-side, no host sync)
  constexpr bool scaled = std::is_same<T, __half>::value;
  unsigned* bnd = reinterpret_cast<unsigned*>(ws + 64);
  float* scl = reinterpret_cast<float*>(ws + 128);
  auto SC = [&](int i) -> const float* { return scaled ? scl + i : nullptr; };
  if (scaled) {
    const double* amp = c.adjoint ? sy.tbar2 : sy.t2;
    c.cuda(cudaMemsetAsync(bnd, 0, 8 * sizeof(unsigned), st));
    k_bound_L<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(sy.L_vv, nj, vv, bnd);
    k_bound_amp<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(
        c.adjoint ? nullptr : sy.t1, amp, o, v, bnd + 2, c.r2, c.r0);
    c.launched(2);
    if (do_den) {
      k_bound_amp<<<static_cast<unsigned>(std::min<int64_t>(4096, (vv + 255) / 256)), 256, 0, st>>>(
          nullptr, sy.tbar2, o, v, bnd + 4);
      c.launched();
    }
    k_scales<<<1, 1, 0, st>>>(bnd, scl);
    c.launched();
  }

  // --- tau^pm (both directions need it)
  c.cuda(cudaMemsetAsync(tp, 0, mat_bytes(P.prec, P.Pop, P.Kvp), st));
  if (minus) c.cuda(cudaMemsetAsync(tm, 0, mat_bytes(P.prec, P.Pom, P.Kvm), st));
  k_pack_tau<T><<<dim3(v, static_cast<unsigned>(P.Pop)), 128, 0, st>>>(
      c.adjoint ? nullptr : sy.t1, c.adjoint ? sy.tbar2 : sy.t2, o, v, tp, P.Kvp, tp_piece, tm, P.Kvm, tm_piece,
      minus, SC(1), c.r2, c.r0);
  c.launched();

  double* epart = at<double>(ws, P.o_E);
  const int64_t o2 = static_cast<int64_t>(o) * o;

  // --- residual-side preparation
  T *LT = nullptr, *gp = nullptr, *gm = nullptr;
  S *G = nullptr, *Op = nullptr, *Om = nullptr;
  const int64_t LT_piece = vv * P.Kj, g_piece_p = P.maxpairs * P.Kvp, g_piece_m = P.maxpairs * P.Kvm;
  if (do_res) {
    LT = at<T>(ws, P.o_LT);
    G = at<S>(ws, P.o_G);
    gp = at<T>(ws, P.o_gp);
    gm = at<T>(ws, P.o_gm);
    Op = at<S>(ws, P.o_Op);
    Om = at<S>(ws, P.o_Om);
    k_prep_LT<T><<<dim3(static_cast<unsigned>((vv + 31) / 32), static_cast<unsigned>(P.Kj / 32)), dim3(32, 8), 0,
                   st>>>(sy.L_vv, nj, vv, v, c.adjoint ? 1 : 0, LT, P.Kj, LT_piece, SC(0));
    c.launched();
    c.cuda(cudaMemsetAsync(gp, 0, mat_bytes(P.prec, P.maxpairs, P.Kvp), st));
    if (minus) c.cuda(cudaMemsetAsync(gm, 0, mat_bytes(P.prec, P.maxpairs, P.Kvm), st));
  }

  // --- density-side preparation
  T *LN = nullptr, *tpT = nullptr, *tmT = nullptr, *bp = nullptr, *bm = nullptr, *Gt = nullptr, *Gb = nullptr;
  S *Gp = nullptr, *Gm_ = nullptr, *Dacc = nullptr;
  const int64_t LN_piece = static_cast<int64_t>(nj) * v * vp;
  const int64_t tpT_piece = P.Pvp * P.Kop, tmT_piece = P.Pvm * P.Kom;
  const int64_t bp_piece = P.Pvp * P.Kop, bm_piece = P.Pvp * P.Kom;
  const int64_t gt_piece = P.maxrows * P.ldt;
  if (do_den) {
    LN = at<T>(ws, P.o_LN);
    tpT = at<T>(ws, P.o_tpT);
    tmT = at<T>(ws, P.o_tmT);
    bp = at<T>(ws, P.o_bp);
    bm = at<T>(ws, P.o_bm);
    Gp = at<S>(ws, P.o_Gp);
    Gm_ = at<S>(ws, P.o_Gm);
    Gt = at<T>(ws, P.o_Gt);
    Gb = at<T>(ws, P.o_Gb);
    // D accumulates over pair blocks: in float-float scratch (mixed) or
    // directly in the FP64 output (FP64 path)
    Dacc = Path<T>::mixed ? at<S>(ws, P.o_D) : reinterpret_cast<S*>(D);
    k_prep_LN<T><<<2048, 256, 0, st>>>(sy.L_vv, nj, v, vp, LN, LN_piece, SC(0));
    c.launched();
    c.cuda(cudaMemsetAsync(tpT, 0, mat_bytes(P.prec, P.Pvp, P.Kop), st));
    k_transpose<T, Path<T>::NP><<<dim3(static_cast<unsigned>((P.Pvp + 31) / 32), static_cast<unsigned>((P.Pop + 31) / 32)),
                                  dim3(32, 8), 0, st>>>(tp, P.Pop, P.Pvp, P.Kvp, tp_piece, tpT, P.Kop, tpT_piece);
    c.launched();
    c.cuda(cudaMemsetAsync(bp, 0, mat_bytes(P.prec, P.Pvp, P.Kop), st));
    if (minus) {
      c.cuda(cudaMemsetAsync(tmT, 0, mat_bytes(P.prec, P.Pvm, P.Kom), st));
      k_transpose<T, Path<T>::NP><<<dim3(static_cast<unsigned>((P.Pvm + 31) / 32), static_cast<unsigned>((P.Pom + 31) / 32)),
                                    dim3(32, 8), 0, st>>>(tm, P.Pom, P.Pvm, P.Kvm, tm_piece, tmT, P.Kom, tmT_piece);
      c.launched();
      c.cuda(cudaMemsetAsync(bm, 0, mat_bytes(P.prec, P.Pvp, P.Kom), st));
    }
    for (const PBlock& b : P.pbs) {
      k_pack_tbar<T><<<static_cast<unsigned>(b.npairs), 128, 0, st>>>(sy.tbar2, o, v, b.a0, b.b0, b.nb, b.diag,
                                                                     b.pair_off, bp, P.Kop, bp_piece, bm, P.Kom,
                                                                     bm_piece, minus, SC(2));
      c.launched();
    }
    c.cuda(cudaMemsetAsync(Gt, 0, mat_bytes(P.prec, P.maxrows, P.ldt), st));
    c.cuda(cudaMemsetAsync(Gb, 0, mat_bytes(P.prec, P.maxrows, P.ldt), st));
    c.cuda(cudaMemsetAsync(Dacc, 0, static_cast<size_t>(nj) * vv * 8, st));
  }

  const unsigned ntp = static_cast<unsigned>(P.nt * (P.nt + 1) / 2);
  for (size_t ib = 0; ib < P.pbs.size() && !c.err; ++ib) {
    const PBlock& b = P.pbs[ib];
    if (do_res) {
      // g-build: G[(b_l,d)][(a_l,c)] = sum_J L^J_ac L^J_bd
      const int64_t M = static_cast<int64_t>(b.na) * v, N = static_cast<int64_t>(b.nb) * v;
      const Gm g = {LT + static_cast<int64_t>(b.a0) * v * P.Kj, P.Kj, M, P.Kj, LT_piece,
                    LT + static_cast<int64_t>(b.b0) * v * P.Kj, P.Kj, N, P.Kj, LT_piece,
                    M, N, P.Kj, G, M, false, SC(0), SC(0), b.diag ? v : 0};  // diagonal block: pairs a <= b only
      run_gemms<T>(&g, 1, c);
      k_pack_g<T, S><<<dim3(ntp, static_cast<unsigned>(b.npairs)), dim3(32, 8), 0, st>>>(
          G, M, v, b.a0, b.b0, b.nb, b.diag, P.nt, gp, P.Kvp, g_piece_p, gm, P.Kvm, g_piece_m, minus, SC(3));
      c.launched();
      // ladder: Omega^pm[p][pr] = sum_k g^pm[pr][k] tau^pm[p][k]  (both signs in one launch)
      const Gm lg[2] = {
          {gp, P.Kvp, b.npairs, P.Kvp, g_piece_p, tp, P.Kvp, P.Pop, P.Kvp, tp_piece, b.npairs, P.Pop, P.Kvp, Op,
           P.ldO, false, SC(3), SC(1)},
          {gm, P.Kvm, b.npairs, P.Kvm, g_piece_m, tm, P.Kvm, P.Pom, P.Kvm, tm_piece, b.npairs, P.Pom, P.Kvm, Om,
           P.ldO, false, SC(3), SC(1)}};
      run_gemms<T>(lg, minus ? 2 : 1, c);
      k_unpack_omega<S><<<static_cast<unsigned>(o2), 256, 0, st>>>(
          Op, Om, P.ldO, o, v, b.a0, b.b0, b.nb, b.diag, b.npairs, minus, omega, sy.tbar2,
          do_E ? epart + static_cast<int64_t>(ib) * o2 : nullptr);
      c.launched();
    }
    if (do_den) {
      // Gamma'^pm[pr][k] = sum_p tau^pm^T[k][p] tbar^pm[pr][p]  (both signs in one launch)
      const Gm gg[2] = {
          {tpT, P.Kop, P.Pvp, P.Kop, tpT_piece, bp + b.pair_off * P.Kop, P.Kop, b.npairs, P.Kop, bp_piece, P.Pvp,
           b.npairs, P.Kop, Gp, P.Kvp, false, SC(1), SC(2)},
          {tmT, P.Kom, P.Pvm, P.Kom, tmT_piece, bm + b.pair_off * P.Kom, P.Kom, b.npairs, P.Kom, bm_piece, P.Pvm,
           b.npairs, P.Kom, Gm_, P.Kvm, false, SC(1), SC(2)}};
      run_gemms<T>(gg, minus ? 2 : 1, c);
      k_unpack_gamma<T, S><<<dim3(ntp, static_cast<unsigned>(b.npairs)), dim3(32, 8), 0, st>>>(
          Gp, Gm_, P.Kvp, P.Kvm, v, vp, b.a0, b.b0, b.nb, b.diag, P.nt, minus, Gt, P.ldt, gt_piece, Gb, P.ldt,
          gt_piece, SC(4));
      c.launched();
      // D^J_(x,c) += sum_(y,d) Gamma[(x,c)][(y,d)] L^J_yd  (top and, off the diagonal, bottom)
      const int64_t Mt = static_cast<int64_t>(b.na) * v, Kt = rup(static_cast<int64_t>(b.nb) * vp, 64);
      const int64_t Mb = static_cast<int64_t>(b.nb) * v, Kb = rup(static_cast<int64_t>(b.na) * vp, 64);
      const Gm dg[2] = {
          {Gt, P.ldt, Mt, P.ldt, gt_piece, LN + static_cast<int64_t>(b.b0) * vp, static_cast<int64_t>(v) * vp, nj,
           static_cast<int64_t>(v - b.b0) * vp, LN_piece, Mt, nj, Kt, Dacc + static_cast<int64_t>(b.a0) * v, vv,
           true, SC(4), SC(0)},
          {Gb, P.ldt, Mb, P.ldt, gt_piece, LN + static_cast<int64_t>(b.a0) * vp, static_cast<int64_t>(v) * vp, nj,
           static_cast<int64_t>(v - b.a0) * vp, LN_piece, Mb, nj, Kb, Dacc + static_cast<int64_t>(b.b0) * v, vv,
           true, SC(4), SC(0)}};
      run_gemms<T>(dg, b.diag ? 1 : 2, c);
    }
  }
  if (do_den && Path<T>::mixed) {
    k_ff_to_f64<<<4096, 256, 0, st>>>(reinterpret_cast<const float2*>(Dacc), D, static_cast<int64_t>(nj) * vv);
    c.launched();
  }
  if (do_E && do_res) {
    k_sum_final<<<1, 1024, 0, st>>>(epart, static_cast<int64_t>(P.pbs.size()) * o2, E);
    c.launched();
  }
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

static size_t ws_need(const cc_ladder_system* sys, int n_sys, int prec, int which) {
  size_t need = 0;
  for (int i = 0; i < n_sys; ++i) {
    Plan P;
    if (!make_plan(sys[i], prec, which, P)) return 0;
    need = std::max(need, P.total);
  }
  return need;
}

static int run(const cc_ladder_system* sys, int n_sys, double* const* omega, double* const* D, double* E,
               int prec, int which, bool res, bool den, bool want_E, void* ws, size_t ws_bytes, void* stream,
               bool adjoint = false, const double* const* es_r2 = nullptr, const double* es_r0 = nullptr,
               bool clear_status = true) {
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
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  c.status = reinterpret_cast<Status*>(ws);
  c.timeout_ns = static_cast<uint64_t>(env_int("CC_TIMEOUT_MS", 4000)) * 1000000ull;
  c.adjoint = adjoint;
  // every call starts from a clear status word; cc_ladder_status() reads it
  if (clear_status) c.cuda(cudaMemsetAsync(ws, 0, sizeof(Status), c.st));
  for (int i = 0; i < n_sys && !c.err; ++i) {
    Plan P;
    make_plan(sys[i], prec, which, P);
    double* om = (res && omega) ? omega[i] : nullptr;
    double* Dd = den ? D[i] : nullptr;
    double* Ei = want_E ? E + i : nullptr;
    c.r2 = es_r2 ? es_r2[i] : nullptr;
    c.r0 = es_r0 ? es_r0[i] : 1.0;
    if (prec == CC_PREC_MIXED)
      run_system<__nv_bfloat16>(sys[i], P, static_cast<char*>(ws), om, Dd, Ei, res, den, want_E, c);
    else if (prec == CC_PREC_FP16X2)
      run_system<__half>(sys[i], P, static_cast<char*>(ws), om, Dd, Ei, res, den, want_E, c);
    else
      run_system<double>(sys[i], P, static_cast<char*>(ws), om, Dd, Ei, res, den, want_E, c);
  }
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
      !(which & CC_WS_STEP))
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
  double ms = 0.0;
  for (auto& pr : g_prof.pending) {
    if (cudaEventSynchronize(pr.second) != cudaSuccess) return CC_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess) return CC_ERR_CUDA;
    ms += t;
  }
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
