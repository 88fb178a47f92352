// Split-operand tensor-core contraction for sm_103a (tcgen05 + TMA + TMEM).
// Three kernels share the scheme below: cc_gemm_split3_tc (one CTA per 128 x
// 128 tile, windows of a tunable length, the split-BF16 default),
// cc_gemm_split3_w1 (one window per 64-term k-block, three window buffers,
// the split-FP16 default) and cc_gemm_split3_pair (CTA pairs on 256 x 128
// tiles); each is described where it is defined.
//
// Two piece schemes share the kernel.
//  * NP = 3 (split BF16): every operand element is x = x0 + x1 + x2, three
//    BF16 pieces (24 significant bits, each the round-to-nearest BF16 of what
//    the previous ones left).  A useful product a*b is formed from the six
//    piece products of weight at least 2^-16 of the leading one,
//    a0b0 + (a0b1 + a1b0 + a0b2 + a1b1 + a2b0); the dropped terms are
//    O(2^-24) relative.
//  * NP = 2 (scaled split FP16): the operand matrix is first multiplied by a
//    power of two that brings its largest element to at most 2^14, then
//    x = x0 + x1 with two FP16 pieces (22 significant bits); a*b is
//    a0b0 + (a0b1 + a1b0), the dropped a1b1 is O(2^-22) relative.  The
//    epilogue divides by the two scales (exact).
//
// Accumulation.  The tensor core adds each K=16 step into its FP32
// accumulator with a truncating (round-toward-zero) alignment, which biases
// every output toward zero, growing linearly with the number of steps.  So:
//   * the leading product a0b0 goes to its own TMEM accumulator H, which is
//     restarted every window of K terms (default 128 for BF16 pieces, 64 for
//     FP16 pieces, whose 22-bit products lose more bits per step; tunable),
//     so the bias never spans more than a few tensor-core steps;
//   * the small products (weight <= 2^-8 of the leading one) go to a second
//     accumulator L, restarted every 4096 terms; its truncation bias is
//     scaled down by that weight.
// The drain warps add the window sums (and the L segment sums) in FP32
// (round to nearest, unbiased) and every FOLD windows fold that partial sum
// error-free into a two-sum (HI in registers, LO in TMEM), so the long K sum
// carries no rounding drift.  H is double-buffered (H0, H1) so the drain of
// one window overlaps the MMAs of the next; the MMA warp waits for the
// (rare) L drain.  Measured on GB300, the drain is what bounds short windows:
// a two-sum per window (instead of one FP32 add) or a third H buffer with
// both halves of the two-sum in registers (96 registers a thread, spilling)
// ran 10-25% slower.  One CTA owns a 128 x 128 output tile over the whole K
// and writes the float-float result hi + lo (or adds it to the value there).
//
// Persistent, grouped launch.  One launch takes a list of up to MAXP
// independent problems (the +- pair of one contraction, both D slabs, or the
// same contraction of many systems of a batch); their 128 x 128 output tiles
// form one flattened list, problems ordered by K (longest first).  The grid
// holds at most one CTA per SM, and each CTA pulls tiles from a device work
// queue (an atomic counter in the workspace header) until the list is empty.
// Barriers, TMEM and the smem ring live across tiles, so the TMA warp loads
// the next tile while the MMA warp finishes the current one, and the MMA warp
// starts the next tile's windows while the drain warps write the previous
// tile's result.  Every tile is computed by one CTA over its whole K in the
// same arithmetic order whatever CTA takes it: results are bit-for-bit
// independent of the scheduling and of the grouping.
//
// CTA = 18 warps: warp 0 pulls tiles and issues TMA loads (one elected lane),
// warp 1 owns TMEM and issues tcgen05.mma (one elected lane), warps 2-17 drain
// (warp w reads TMEM lane quarter w%4 and the 32-column slice (w-2)/4).  The
// TMA warp hands each tile's (problem, m0, n0) to the others through a
// two-entry shared-memory ring.  Tile 128 x 128 x 64 with a 192 KB smem ring
// (BF16: 2 stages of 3 A + 3 B pieces; FP16: 3 stages of 2 + 2), 128-byte
// swizzle (128-byte TMA rows move operands ~1.2x faster than 64-byte ones).
// Every CTA loads its own A and B tiles (one 3-D box of all pieces each).
// TMEM columns: H0 [0,128), H1 [128,256), L [256,384), LO [384,512).
// Every wait is bounded (globaltimer) and latches CC_ERR_TIMEOUT; on the way
// out the TMA warp waits (bounded) for its own copies in flight and the MMA
// warp for its own MMAs before TMEM is released.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "gemm.h"

namespace ccl {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int RASTER_GROUP = 8;           // m-tiles per raster group (L2 reuse of B panels)
constexpr int A_PIECE = BM * BK * 2;      // 16384 B (one 16-bit piece of a 128 x 64 tile)
constexpr int B_PIECE = BN * BK * 2;      // 16384 B
constexpr int SMEM_BYTES = 196608 + 1024 + 512;  // stages * stage bytes is 192 KB for both schemes
constexpr uint32_t TMEM_COLS = 512;
constexpr int FOLD = 32;                  // H windows summed in FP32 before the error-free fold
constexpr uint32_t COL_H0 = 0, COL_H1 = 128, COL_L = 256, COL_LO = 384;
constexpr int NDRAIN = 16;                // draining warps (4 per TMEM lane quarter)
constexpr int NTHREADS = (2 + NDRAIN) * 32;
constexpr int DCOLS = BN / (NDRAIN / 4);  // accumulator columns per drain thread
constexpr int TRING = 2;                  // tile hand-off ring entries
constexpr int MAXP = GEMM_MAX_PROBLEMS;

// Piece schemes.  NP = 3: BF16 pieces, six products, the leading one last.
// NP = 2: FP16 pieces of power-of-two scaled operands, three products.
template <int NP>
struct Scheme;
template <>
struct Scheme<3> {
  static constexpr int STAGES = 2;
  static constexpr int NPROD = 6;
  static constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN);
  static __device__ __forceinline__ void pieces(int q, int& pa, int& pb) {
    switch (q) {
      case 0: pa = 2; pb = 0; break;
      case 1: pa = 1; pb = 1; break;
      case 2: pa = 0; pb = 2; break;
      case 3: pa = 1; pb = 0; break;
      case 4: pa = 0; pb = 1; break;
      default: pa = 0; pb = 0; break;
    }
  }
};
template <>
struct Scheme<2> {
  static constexpr int STAGES = 3;
  static constexpr int NPROD = 3;
  static constexpr uint32_t IDESC = idesc_f16_f32(BM, BN);
  static __device__ __forceinline__ void pieces(int q, int& pa, int& pb) {
    switch (q) {
      case 0: pa = 1; pb = 0; break;
      case 1: pa = 0; pb = 1; break;
      default: pa = 0; pb = 0; break;
    }
  }
};

struct Prob {
  CUtensorMap ta, tb;  // boxes {64, 128, NP}: all pieces of a 128-row, 64-term tile
  float2* out;
  const float* sa;     // operand scales (mixed FP16 scheme) or null
  const float* sb;
  long long ldo;
  int M, N, K, mode;
  int tri;             // > 0: skip output tiles with every row block above every column block
  int mt, nt;          // m-tiles, n-tiles
  int tile0;           // first entry of this problem in the flattened tile list
};
struct Probs {
  Prob p[MAXP];
  int nprob;
  int total;   // tiles in the flattened list
  int win_kb;  // k-blocks per H window
  int lwin;    // H windows per L segment
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that ignores the abort flag (used on the way out, for work this
// thread itself put in flight).
__device__ __forceinline__ bool mbar_wait_own(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > timeout_ns) return false;
  return true;
}

// Flattened tile t -> (problem, m0, n0) for output tiles TBM rows high; false
// for a tile the problem skips.
template <int TBM>
__device__ __forceinline__ bool decode_tile(const Probs& P, int t, int& pi, int& m0, int& n0) {
  int p = 0;
  while (p + 1 < P.nprob && P.p[p + 1].tile0 <= t) ++p;
  const Prob& pr = P.p[p];
  // grouped raster: consecutive tiles sweep the n-tiles of RASTER_GROUP m-tiles
  const int lin = t - pr.tile0;
  const int grp = lin / (RASTER_GROUP * pr.nt);
  const int gm0 = grp * RASTER_GROUP;
  const int gsz = min(RASTER_GROUP, pr.mt - gm0);
  const int in_grp = lin - grp * RASTER_GROUP * pr.nt;
  pi = p;
  m0 = (gm0 + in_grp % gsz) * TBM;
  n0 = (in_grp / gsz) * BN;
  if (pr.tri > 0) {
    // rows and columns come in blocks of pr.tri (a symmetric product's pair index): a tile whose
    // smallest row block lies past its largest column block computes nothing anybody reads
    const int n_end = min(pr.N, n0 + BN);
    if (m0 / pr.tri > (n_end - 1) / pr.tri) return false;
  }
  return true;
}

// error-free FP32 accumulation: hi + lo += x
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float t = s - hi;
  const float e = (hi - (s - t)) + (x - t);
  hi = s;
  lo += e;
}

// acc += DCOLS TMEM columns of this thread's row (round-to-nearest adds, two
// lanes per packed FP32x2 instruction: the drain's instructions share issue
// slots with the MMA and TMA warps, so fewer of them is measurably faster)
__device__ __forceinline__ void add_cols(uint32_t src, float (&acc)[DCOLS]) {
#pragma unroll
  for (int c = 0; c < DCOLS; c += 16) {
    uint32_t r[16];
    tmem_ld16(src + c, r);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
      unsigned long long a2, r2, s2;
      asm("mov.b64 %0, {%1, %2};" : "=l"(a2) : "f"(acc[c + j]), "f"(acc[c + j + 1]));
      asm("mov.b64 %0, {%1, %2};" : "=l"(r2) : "r"(r[j]), "r"(r[j + 1]));
      asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s2) : "l"(a2), "l"(r2));
      asm("mov.b64 {%0, %1}, %2;" : "=f"(acc[c + j]), "=f"(acc[c + j + 1]) : "l"(s2));
    }
  }
}

// (HI, LO[TMEM]) += acc error-free, then acc = 0
__device__ __forceinline__ void fold_cols(uint32_t lo_addr, float (&acc)[DCOLS], float (&HI)[DCOLS]) {
#pragma unroll
  for (int c = 0; c < DCOLS; c += 8) {
    uint32_t l[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7])
                 : "r"(lo_addr + c));
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float lo = __uint_as_float(l[j]);
      two_sum_acc(HI[c + j], lo, acc[c + j]);
      acc[c + j] = 0.f;
      l[j] = __float_as_uint(lo);
    }
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(lo_addr + c),
                 "r"(l[0]), "r"(l[1]), "r"(l[2]), "r"(l[3]), "r"(l[4]), "r"(l[5]), "r"(l[6]), "r"(l[7])
                 : "memory");
  }
  tmem_st_wait();
}

template <int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    cc_gemm_split3_tc(const __grid_constant__ Probs P, int* __restrict__ queue, Status* st,
                      unsigned long long timeout_ns) {
  using SC = Scheme<NP>;
  constexpr int STAGES = SC::STAGES;
  constexpr int A_STAGE = NP * A_PIECE, B_STAGE = NP * B_PIECE, STAGE = A_STAGE + B_STAGE;
  const int WIN_KB = P.win_kb, LWIN = P.lwin;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* hfull = empty + STAGES;   // [2]
  uint64_t* hempty = hfull + 2;       // [2]
  uint64_t* lfull = hempty + 2;       // [1]
  uint64_t* lempty = lfull + 1;       // [1]
  uint64_t* tfull = lempty + 1;       // [TRING]
  uint64_t* tempty = tfull + TRING;   // [TRING]
  uint64_t* mdone = tempty + TRING;   // [1]
  int4* ring = reinterpret_cast<int4*>(mdone + 2);  // [TRING] (16-byte aligned)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ring + TRING);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);  // one MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&hfull[b], 1);
      mbar_init(&hempty[b], NDRAIN);
    }
    mbar_init(lfull, 1);
    mbar_init(lempty, NDRAIN);
    for (int r = 0; r < TRING; ++r) {
      mbar_init(&tfull[r], 1);
      mbar_init(&tempty[r], 1 + NDRAIN);  // the MMA lane and every drain warp
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: pull tiles from the queue, hand them on, load their operands
      long long g = 0;  // k-blocks issued so far (stage ring position)
      int tc = 0;       // tiles handed on so far (tile ring position)
      bool ok = true;
      while (ok) {
        int pi = -1, m0 = 0, n0 = 0;
        for (;;) {
          const int t = atomicAdd(queue, 1);
          if (t >= P.total) break;
          if (decode_tile<BM>(P, t, pi, m0, n0)) break;
          pi = -1;
        }
        const int slot = tc % TRING;
        if (!mbar_wait_bounded(&tempty[slot], ((tc / TRING) & 1) ^ 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 106);
          break;
        }
        ring[slot] = make_int4(pi, m0, n0, 0);
        mbar_arrive(&tfull[slot]);
        ++tc;
        if (pi < 0) break;
        const Prob& pr = P.p[pi];
        const int nkb = pr.K / BK;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          const uint32_t ph = static_cast<uint32_t>((g / STAGES) & 1);
          if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort_flag, timeout_ns)) {
            latch_error(st, kErrTimeout, 101);
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * STAGE;
          mbar_expect_tx(&full[s], STAGE);  // every piece of the A and B tiles
          tma_load_3d(&pr.ta, &full[s], sa, kb * BK, m0, 0);
          tma_load_3d(&pr.tb, &full[s], sa + A_STAGE, kb * BK, n0, 0);
        }
      }
      // our own copies still in flight (only after an abort) land before the CTA leaves
      for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
        mbar_wait_own(&full[q % STAGES], static_cast<uint32_t>((q / STAGES) & 1), timeout_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;  // k-blocks consumed
      int gw = 0;       // H windows issued (H buffer = gw & 1)
      int gl = 0;       // L segments issued
      int tc = 0;
      bool ok = true;
      while (ok) {
        const int slot = tc % TRING;
        if (!mbar_wait_bounded(&tfull[slot], (tc / TRING) & 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 107);
          break;
        }
        const int4 e = ring[slot];
        mbar_arrive(&tempty[slot]);
        ++tc;
        if (e.x < 0) break;
        const int nkb = P.p[e.x].K / BK;
        const int nwin = (nkb + WIN_KB - 1) / WIN_KB;
        for (int w = 0; w < nwin && ok; ++w, ++gw) {
          const int hb = gw & 1;
          const uint32_t hcol = hb ? COL_H1 : COL_H0;
          const bool lseg_start = (w % LWIN) == 0;
          if (gw >= 2 && !mbar_wait_bounded(&hempty[hb], ((gw >> 1) - 1) & 1, abort_flag, timeout_ns)) {
            latch_error(st, kErrTimeout, 104);
            ok = false;
            break;
          }
          if (lseg_start && gl > 0 && !mbar_wait_bounded(lempty, (gl - 1) & 1, abort_flag, timeout_ns)) {
            latch_error(st, kErrTimeout, 105);
            ok = false;
            break;
          }
          tc_fence_after();
          const int kb_beg = w * WIN_KB, kb_end = min(nkb, (w + 1) * WIN_KB);
          for (int kb = kb_beg; kb < kb_end; ++kb, ++g) {
            const int s = static_cast<int>(g % STAGES);
            const uint32_t ph = static_cast<uint32_t>((g / STAGES) & 1);
            if (!mbar_wait_bounded(&full[s], ph, abort_flag, timeout_ns)) {
              latch_error(st, kErrTimeout, 102);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_base = smem_u32(smem + s * STAGE);
            const uint32_t b_base = a_base + A_STAGE;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const bool first = (kb == kb_beg) && ks == 0;
#pragma unroll
              for (int q = 0; q < SC::NPROD; ++q) {
                int pa, pb;
                SC::pieces(q, pa, pb);
                const uint64_t ad = sdesc_k_sw128(a_base + pa * A_PIECE + ks * 32);
                const uint64_t bd = sdesc_k_sw128(b_base + pb * B_PIECE + ks * 32);
                if (q == SC::NPROD - 1)
                  umma_f16(tmem + hcol, ad, bd, SC::IDESC, first ? 0u : 1u);
                else
                  umma_f16(tmem + COL_L, ad, bd, SC::IDESC, (first && lseg_start && q == 0) ? 0u : 1u);
              }
            }
            umma_commit(&empty[s]);  // releases the stage once its MMAs have read it
          }
          if (!ok) break;
          umma_commit(&hfull[hb]);
          if ((w + 1) % LWIN == 0 || w == nwin - 1) {
            umma_commit(lfull);
            ++gl;
          }
        }
      }
      // every MMA this thread issued completes before TMEM is released
      umma_commit(mdone);
      mbar_wait_own(mdone, 0, timeout_ns);
    }
    __syncwarp();
  } else {
    // drain warps: window sums go into acc (FP32, round to nearest); every
    // FOLD windows acc is added error-free into (HI registers, LO in TMEM
    // columns [384, 512)).
    const int q = warp & 3;                  // TMEM lane quarter
    const int cb = ((warp - 2) >> 2) * DCOLS;  // first accumulator column of this warp
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    const uint32_t lo_addr = tmem + lane_off + COL_LO + cb;
    int gw = 0, gl = 0, tc = 0;
    bool ok = true;
    while (ok) {
      const int slot = tc % TRING;
      bool got = mbar_wait_bounded(&tfull[slot], (tc / TRING) & 1, abort_flag, timeout_ns);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const int4 e = ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[slot]);
      ++tc;
      if (e.x < 0) break;
      const Prob& pr = P.p[e.x];
      const int nkb = pr.K / BK;
      const int nwin = (nkb + WIN_KB - 1) / WIN_KB;
      float acc[DCOLS], HI[DCOLS];
#pragma unroll
      for (int j = 0; j < DCOLS; ++j) acc[j] = HI[j] = 0.f;
      {
        uint32_t z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
        for (int c = 0; c < DCOLS; c += 16) tmem_st16(lo_addr + c, z);
        tmem_st_wait();
      }
      for (int w = 0; w < nwin; ++w, ++gw) {
        const int hb = gw & 1;
        got = mbar_wait_bounded(&hfull[hb], (gw >> 1) & 1, abort_flag, timeout_ns);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        add_cols(tmem + lane_off + (hb ? COL_H1 : COL_H0) + cb, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&hempty[hb]);
        if ((w + 1) % LWIN == 0 || w == nwin - 1) {
          got = mbar_wait_bounded(lfull, gl & 1, abort_flag, timeout_ns);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          tc_fence_after();
          add_cols(tmem + lane_off + COL_L + cb, acc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(lempty);
          ++gl;
        }
        if ((w + 1) % FOLD == 0 || w == nwin - 1) fold_cols(lo_addr, acc, HI);
      }
      ok = ok && !*abort_flag;
      if (!ok) break;
      const int m0 = e.y, n0 = e.z;
      const int row = m0 + q * 32 + lane;
      const float inv = (1.f / ld_scale(pr.sa)) * (1.f / ld_scale(pr.sb));  // powers of two: exact
#pragma unroll
      for (int c = 0; c < DCOLS; c += 8) {
        uint32_t l[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]),
                       "=r"(l[7])
                     : "r"(lo_addr + c));
        tmem_ld_wait();
        if (row < pr.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = n0 + cb + c + j;
            if (n < pr.N) {
              float2 v = ff_scale(ff_fast_two_sum(HI[c + j], __uint_as_float(l[j])), inv);
              float2* p = pr.out + static_cast<long long>(n) * pr.ldo + row;
              if (pr.mode == OUT_FF_ACCUM) v = ff_add(*p, v);
              *p = v;
            }
          }
        }
      }
    }
    if (!ok && lane == 0) latch_error(st, kErrTimeout, 103);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// One-k-block-window variant.  Every 64-term k-block is its own window, and
// all products of a k-block go into the window's accumulator: the small
// products first (while it is still small, so their truncation is scaled by
// their weight), the leading product last.  With no separate L accumulator
// the TMEM holds three H buffers (H0 [0,128), H1 [128,256), H2 [256,384), LO
// [384,512)), so the drain of a window has two windows of MMA time before its
// buffer is needed again, and one commit per k-block (to the window's hfull)
// both releases the stage and hands the window to the drain warps.  The
// drain, fold and epilogue are the single-CTA kernel's (FOLD1 windows per
// fold, the same 4096 terms).
constexpr int NHBUF = 3;
constexpr int FOLD1 = 64;

template <int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    cc_gemm_split3_w1(const __grid_constant__ Probs P, int* __restrict__ queue, Status* st,
                      unsigned long long timeout_ns) {
  using SC = Scheme<NP>;
  constexpr int STAGES = SC::STAGES;
  static_assert(STAGES <= NHBUF, "a stage's release is read from the hfull of its k-block: the next phase of "
                                 "that barrier needs the k-block being loaded only if STAGES <= NHBUF");
  constexpr int A_STAGE = NP * A_PIECE, B_STAGE = NP * B_PIECE, STAGE = A_STAGE + B_STAGE;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* hfull = full + STAGES;       // [NHBUF]
  uint64_t* hempty = hfull + NHBUF;      // [NHBUF]
  uint64_t* tfull = hempty + NHBUF;      // [TRING]
  uint64_t* tempty = tfull + TRING;      // [TRING]
  uint64_t* mdone = tempty + TRING;      // [1]
  int4* ring = reinterpret_cast<int4*>(smem + STAGES * STAGE + 256);  // [TRING] (16-byte aligned)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ring + TRING);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
    for (int b = 0; b < NHBUF; ++b) {
      mbar_init(&hfull[b], 1);        // one MMA commit per window (= k-block)
      mbar_init(&hempty[b], NDRAIN);  // every drain warp
    }
    for (int r = 0; r < TRING; ++r) {
      mbar_init(&tfull[r], 1);
      mbar_init(&tempty[r], 1 + NDRAIN);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tslot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // k-blocks (= windows) issued so far
      int tc = 0;
      bool ok = true;
      while (ok) {
        int pi = -1, m0 = 0, n0 = 0;
        for (;;) {
          const int t = atomicAdd(queue, 1);
          if (t >= P.total) break;
          if (decode_tile<BM>(P, t, pi, m0, n0)) break;
          pi = -1;
        }
        const int slot = tc % TRING;
        if (!mbar_wait_bounded(&tempty[slot], ((tc / TRING) & 1) ^ 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 306);
          break;
        }
        ring[slot] = make_int4(pi, m0, n0, 0);
        mbar_arrive(&tfull[slot]);
        ++tc;
        if (pi < 0) break;
        const Prob& pr = P.p[pi];
        const int nkb = pr.K / BK;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          if (g >= STAGES) {
            // the stage's previous k-block g - STAGES is done once its window's hfull phase completes
            const long long q = g - STAGES;
            if (!mbar_wait_bounded(&hfull[q % NHBUF], static_cast<uint32_t>((q / NHBUF) & 1), abort_flag,
                                   timeout_ns)) {
              latch_error(st, kErrTimeout, 301);
              ok = false;
              break;
            }
          }
          uint8_t* sa = smem + s * STAGE;
          mbar_expect_tx(&full[s], STAGE);
          tma_load_3d(&pr.ta, &full[s], sa, kb * BK, m0, 0);
          tma_load_3d(&pr.tb, &full[s], sa + A_STAGE, kb * BK, n0, 0);
        }
      }
      for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
        mbar_wait_own(&full[q % STAGES], static_cast<uint32_t>((q / STAGES) & 1), timeout_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int tc = 0;
      bool ok = true;
      while (ok) {
        const int slot = tc % TRING;
        if (!mbar_wait_bounded(&tfull[slot], (tc / TRING) & 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 307);
          break;
        }
        const int4 e = ring[slot];
        mbar_arrive(&tempty[slot]);
        ++tc;
        if (e.x < 0) break;
        const int nkb = P.p[e.x].K / BK;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = static_cast<int>(g % STAGES);
          const int hb = static_cast<int>(g % NHBUF);
          if (g >= NHBUF && !mbar_wait_bounded(&hempty[hb], static_cast<uint32_t>(((g / NHBUF) - 1) & 1),
                                               abort_flag, timeout_ns)) {
            latch_error(st, kErrTimeout, 304);
            ok = false;
            break;
          }
          if (!mbar_wait_bounded(&full[s], static_cast<uint32_t>((g / STAGES) & 1), abort_flag, timeout_ns)) {
            latch_error(st, kErrTimeout, 302);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(smem + s * STAGE);
          const uint32_t b_base = a_base + A_STAGE;
          const uint32_t hcol = tmem + static_cast<uint32_t>(hb) * 128u;
          // small products first (the window's accumulator starts with them), the leading one last
#pragma unroll
          for (int q = 0; q < SC::NPROD; ++q) {
            int pa, pb;
            SC::pieces(q, pa, pb);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const uint64_t ad = sdesc_k_sw128(a_base + pa * A_PIECE + ks * 32);
              const uint64_t bd = sdesc_k_sw128(b_base + pb * B_PIECE + ks * 32);
              umma_f16(hcol, ad, bd, SC::IDESC, (q == 0 && ks == 0) ? 0u : 1u);
            }
          }
          umma_commit(&hfull[hb]);  // the window is done, and so is its k-block's stage
        }
      }
      umma_commit(mdone);
      mbar_wait_own(mdone, 0, timeout_ns);
    }
    __syncwarp();
  } else {
    const int q = warp & 3;
    const int cb = ((warp - 2) >> 2) * DCOLS;
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    const uint32_t lo_addr = tmem + lane_off + COL_LO + cb;
    long long g = 0;
    int tc = 0;
    bool ok = true;
    while (ok) {
      const int slot = tc % TRING;
      bool got = mbar_wait_bounded(&tfull[slot], (tc / TRING) & 1, abort_flag, timeout_ns);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const int4 e = ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[slot]);
      ++tc;
      if (e.x < 0) break;
      const Prob& pr = P.p[e.x];
      const int nkb = pr.K / BK;
      float acc[DCOLS], HI[DCOLS];
#pragma unroll
      for (int j = 0; j < DCOLS; ++j) acc[j] = HI[j] = 0.f;
      {
        uint32_t z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
        for (int c = 0; c < DCOLS; c += 16) tmem_st16(lo_addr + c, z);
        tmem_st_wait();
      }
      for (int w = 0; w < nkb; ++w, ++g) {
        const int hb = static_cast<int>(g % NHBUF);
        got = mbar_wait_bounded(&hfull[hb], static_cast<uint32_t>((g / NHBUF) & 1), abort_flag, timeout_ns);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        add_cols(tmem + lane_off + static_cast<uint32_t>(hb) * 128u + cb, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&hempty[hb]);
        if ((w + 1) % FOLD1 == 0 || w == nkb - 1) fold_cols(lo_addr, acc, HI);
      }
      ok = ok && !*abort_flag;
      if (!ok) break;
      const int m0 = e.y, n0 = e.z;
      const int row = m0 + q * 32 + lane;
      const float inv = (1.f / ld_scale(pr.sa)) * (1.f / ld_scale(pr.sb));  // powers of two: exact
#pragma unroll
      for (int c = 0; c < DCOLS; c += 8) {
        uint32_t l[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]),
                       "=r"(l[7])
                     : "r"(lo_addr + c));
        tmem_ld_wait();
        if (row < pr.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = n0 + cb + c + j;
            if (n < pr.N) {
              float2 v = ff_scale(ff_fast_two_sum(HI[c + j], __uint_as_float(l[j])), inv);
              float2* p = pr.out + static_cast<long long>(n) * pr.ldo + row;
              if (pr.mode == OUT_FF_ACCUM) v = ff_add(*p, v);
              *p = v;
            }
          }
        }
      }
    }
    if (!ok && lane == 0) latch_error(st, kErrTimeout, 303);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// CTA-pair variant.  A cluster of two CTAs on two SMs owns a 256 x 128 output
// tile: the even CTA issues tcgen05.mma.cta_group::2 (M = 256), which reads
// A from both CTAs' shared memory (128 rows each) and B from both (64 of the
// 128 columns each), and leaves rows 0-127 of D in the even CTA's TMEM and
// rows 128-255 in the odd one's.  Per SM this loads 72 KB per BF16 k-block
// instead of 96 KB and the tensor core reads 6 KB of operands per K=16 step
// instead of 8 KB, so the smem ring holds three BF16 stages (four FP16 ones)
// instead of two: more of the load latency is hidden.  The arithmetic of
// every output element (products, windows, drains, folds) is the single-CTA
// kernel's.
//
// Signalling across the pair uses plain remote arrives and stores, each
// addressed to one CTA:
//   * the even CTA's producer pulls tiles from the queue and writes each into
//     both CTAs' tile rings; before each k-block it arrives on the odd CTA's
//     go[s] so that the odd producer may load its halves into stage s; the
//     loads of both CTAs complete on the even CTA's full[s];
//   * the MMA commits empty[s], hfull and lfull in the even CTA; its drain
//     warp 2 relays each hfull / lfull phase to the odd CTA;
//   * hempty, lempty and tempty live in the even CTA and count the arrivals
//     of both CTAs' consumers;
//   * a wait that gives up also raises the other CTA's abort flag.
constexpr int PAIR_BM = 2 * BM;                 // output rows per pair tile
constexpr int B_HALF = (BN / 2) * BK * 2;       // 8192 B: one 16-bit piece of a 64 x 64 B half-tile
constexpr int PAIR_SMEM_BYTES = 221184 + 1024 + 512;  // ring, barriers (< 512 B), 1024-byte alignment
constexpr int PAIR_TEMPTY = 2 * (1 + NDRAIN);   // tile-ring consumers of both CTAs

template <int NP>
struct PairStages;
template <>
struct PairStages<3> {
  static constexpr int N = 3;  // 3 x 72 KB
};
template <>
struct PairStages<2> {
  static constexpr int N = 4;  // 4 x 48 KB
};

__device__ __forceinline__ bool pair_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t peer_abort,
                                          uint64_t timeout_ns) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait_cluster(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > timeout_ns) {
      *abort = 1;
      st_cluster_u32(peer_abort, 1u);
      return false;
    }
  }
}

// W1: the pair form of cc_gemm_split3_w1 (one window per k-block, three
// window buffers, one commit per k-block that also releases the stage; three
// stages so that the stage release can be read from the window's hfull).
template <int NP, bool W1>
__global__ void __launch_bounds__(NTHREADS, 1)
    cc_gemm_split3_pair(const __grid_constant__ Probs P, int* __restrict__ queue, Status* st,
                        unsigned long long timeout_ns) {
  using SC = Scheme<NP>;
  constexpr int STAGES = W1 ? 3 : PairStages<NP>::N;
  constexpr int NH = W1 ? NHBUF : 2;  // window buffers
  constexpr int A_STAGE = NP * A_PIECE, B_STAGE = NP * B_HALF, STAGE = A_STAGE + B_STAGE;
  static_assert(STAGES * STAGE <= 221184, "pair stages exceed the shared-memory ring");
  constexpr uint32_t IDESC = NP == 3 ? idesc_bf16_f32(PAIR_BM, BN) : idesc_f16_f32(PAIR_BM, BN);
  const int WIN_KB = P.win_kb, LWIN = P.lwin;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 221184);
  uint64_t* go = full + STAGES;
  uint64_t* empty = go + STAGES;
  uint64_t* hfull = empty + STAGES;   // [NH]
  uint64_t* hempty = hfull + NH;      // [NH]
  uint64_t* lfull = hempty + NH;      // [1]
  uint64_t* lempty = lfull + 1;       // [1]
  uint64_t* tfull = lempty + 1;       // [TRING]
  uint64_t* tempty = tfull + TRING;   // [TRING]
  uint64_t* mdone = tempty + TRING;   // [1]  (at most 25 barriers: 200 B)
  int4* ring = reinterpret_cast<int4*>(smem + 221184 + 256);  // [TRING] (16-byte aligned)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ring + TRING);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool lead = rank == 0;
  const uint32_t peer = rank ^ 1u;
  const uint32_t peer_abort = mapa_rank(const_cast<int*>(abort_flag), peer);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);   // the even producer's expect_tx; bytes of both CTAs
      mbar_init(&go[s], 1);     // one arrive from the even producer per k-block
      mbar_init(&empty[s], 1);  // one MMA commit
    }
    for (int b = 0; b < NH; ++b) {
      mbar_init(&hfull[b], 1);
      mbar_init(&hempty[b], 2 * NDRAIN);
    }
    mbar_init(lfull, 1);
    mbar_init(lempty, 2 * NDRAIN);
    for (int r = 0; r < TRING; ++r) {
      mbar_init(&tfull[r], 1);
      mbar_init(&tempty[r], PAIR_TEMPTY);
    }
    mbar_init(mdone, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc_pair(tslot, TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync_all();  // both CTAs' barriers are initialised before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;
      int tc = 0;
      bool ok = true;
      if (lead) {
        while (ok) {
          int pi = -1, m0 = 0, n0 = 0;
          for (;;) {
            const int t = atomicAdd(queue, 1);
            if (t >= P.total) break;
            if (decode_tile<PAIR_BM>(P, t, pi, m0, n0)) break;
            pi = -1;
          }
          const int slot = tc % TRING;
          if (!pair_wait(&tempty[slot], ((tc / TRING) & 1) ^ 1, abort_flag, peer_abort, timeout_ns)) {
            latch_error(st, kErrTimeout, 206);
            break;
          }
          const int4 e = make_int4(pi, m0, n0, 0);
          ring[slot] = e;
          st_cluster_v4(mapa_rank(&ring[slot], peer), e);
          mbar_arrive(&tfull[slot]);
          mbar_arrive_cluster(mapa_rank(&tfull[slot], peer));
          ++tc;
          if (pi < 0) break;
          const Prob& pr = P.p[pi];
          const int nkb = pr.K / BK;
          for (int kb = 0; kb < nkb; ++kb, ++g) {
            const int s = static_cast<int>(g % STAGES);
            const uint32_t ph = static_cast<uint32_t>((g / STAGES) & 1);
            bool freed;
            if constexpr (W1) {
              const long long q = g - STAGES;  // the stage's previous k-block: done when its window is
              freed = q < 0 || pair_wait(&hfull[q % NH], static_cast<uint32_t>((q / NH) & 1), abort_flag,
                                         peer_abort, timeout_ns);
            } else {
              freed = pair_wait(&empty[s], ph ^ 1, abort_flag, peer_abort, timeout_ns);
            }
            if (!freed) {
              latch_error(st, kErrTimeout, 201);
              ok = false;
              break;
            }
            // the odd CTA may now load its halves of k-block g into its stage s
            mbar_arrive_cluster(mapa_rank(&go[s], peer));
            uint8_t* sa = smem + s * STAGE;
            mbar_expect_tx(&full[s], 2 * STAGE);
            tma_load_3d_pair(&pr.ta, smem_u32(&full[s]), sa, kb * BK, m0, 0);
            tma_load_3d_pair(&pr.tb, smem_u32(&full[s]), sa + A_STAGE, kb * BK, n0, 0);
          }
        }
        // copies of both CTAs still in flight (only after an abort) land before either CTA leaves
        for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
          mbar_wait_own(&full[q % STAGES], static_cast<uint32_t>((q / STAGES) & 1), timeout_ns);
      } else {
        while (ok) {
          const int slot = tc % TRING;
          if (!pair_wait(&tfull[slot], (tc / TRING) & 1, abort_flag, peer_abort, timeout_ns)) {
            latch_error(st, kErrTimeout, 207);
            break;
          }
          const int4 e = ring[slot];
          mbar_arrive_cluster(mapa_rank(&tempty[slot], 0));
          ++tc;
          if (e.x < 0) break;
          const Prob& pr = P.p[e.x];
          const int nkb = pr.K / BK;
          for (int kb = 0; kb < nkb; ++kb, ++g) {
            const int s = static_cast<int>(g % STAGES);
            if (!pair_wait(&go[s], static_cast<uint32_t>((g / STAGES) & 1), abort_flag, peer_abort, timeout_ns)) {
              latch_error(st, kErrTimeout, 208);
              ok = false;
              break;
            }
            uint8_t* sa = smem + s * STAGE;
            const uint32_t bar = mapa_rank(&full[s], 0);
            tma_load_3d_pair(&pr.ta, bar, sa, kb * BK, e.y + BM, 0);
            tma_load_3d_pair(&pr.tb, bar, sa + A_STAGE, kb * BK, e.z + BN / 2, 0);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lead && lane == 0) {
      long long g = 0;  // k-blocks consumed
      int gw = 0;       // H windows issued (H buffer = gw & 1)
      int gl = 0;       // L segments issued
      int tc = 0;
      bool ok = true;
      while (ok) {
        const int slot = tc % TRING;
        if (!pair_wait(&tfull[slot], (tc / TRING) & 1, abort_flag, peer_abort, timeout_ns)) {
          latch_error(st, kErrTimeout, 207);
          break;
        }
        const int4 e = ring[slot];
        mbar_arrive(&tempty[slot]);
        ++tc;
        if (e.x < 0) break;
        const int nkb = P.p[e.x].K / BK;
        if constexpr (W1) {
          for (int kb = 0; kb < nkb; ++kb, ++g) {
            const int s = static_cast<int>(g % STAGES);
            const int hb = static_cast<int>(g % NH);
            if (g >= NH && !pair_wait(&hempty[hb], static_cast<uint32_t>(((g / NH) - 1) & 1), abort_flag, peer_abort,
                                      timeout_ns)) {
              latch_error(st, kErrTimeout, 204);
              ok = false;
              break;
            }
            if (!pair_wait(&full[s], static_cast<uint32_t>((g / STAGES) & 1), abort_flag, peer_abort, timeout_ns)) {
              latch_error(st, kErrTimeout, 202);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_base = smem_u32(smem + s * STAGE);
            const uint32_t b_base = a_base + A_STAGE;
            const uint32_t hcol = tmem + static_cast<uint32_t>(hb) * 128u;
#pragma unroll
            for (int q = 0; q < SC::NPROD; ++q) {  // small products first, the leading one last
              int pa, pb;
              SC::pieces(q, pa, pb);
#pragma unroll
              for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t ad = sdesc_k_sw128(a_base + pa * A_PIECE + ks * 32);
                const uint64_t bd = sdesc_k_sw128(b_base + pb * B_HALF + ks * 32);
                umma_f16_pair(hcol, ad, bd, IDESC, (q == 0 && ks == 0) ? 0u : 1u);
              }
            }
            umma_commit_pair(&hfull[hb]);  // the window is done, and so is its stage (of both CTAs)
          }
          continue;
        }
        const int nwin = (nkb + WIN_KB - 1) / WIN_KB;
        for (int w = 0; w < nwin && ok; ++w, ++gw) {
          const int hb = gw & 1;
          const uint32_t hcol = hb ? COL_H1 : COL_H0;
          const bool lseg_start = (w % LWIN) == 0;
          if (gw >= 2 && !pair_wait(&hempty[hb], ((gw >> 1) - 1) & 1, abort_flag, peer_abort, timeout_ns)) {
            latch_error(st, kErrTimeout, 204);
            ok = false;
            break;
          }
          if (lseg_start && gl > 0 && !pair_wait(lempty, (gl - 1) & 1, abort_flag, peer_abort, timeout_ns)) {
            latch_error(st, kErrTimeout, 205);
            ok = false;
            break;
          }
          tc_fence_after();
          const int kb_beg = w * WIN_KB, kb_end = min(nkb, (w + 1) * WIN_KB);
          for (int kb = kb_beg; kb < kb_end; ++kb, ++g) {
            const int s = static_cast<int>(g % STAGES);
            const uint32_t ph = static_cast<uint32_t>((g / STAGES) & 1);
            if (!pair_wait(&full[s], ph, abort_flag, peer_abort, timeout_ns)) {
              latch_error(st, kErrTimeout, 202);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_base = smem_u32(smem + s * STAGE);
            const uint32_t b_base = a_base + A_STAGE;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
              const bool first = (kb == kb_beg) && ks == 0;
#pragma unroll
              for (int q = 0; q < SC::NPROD; ++q) {
                int pa, pb;
                SC::pieces(q, pa, pb);
                const uint64_t ad = sdesc_k_sw128(a_base + pa * A_PIECE + ks * 32);
                const uint64_t bd = sdesc_k_sw128(b_base + pb * B_HALF + ks * 32);
                if (q == SC::NPROD - 1)
                  umma_f16_pair(tmem + hcol, ad, bd, IDESC, first ? 0u : 1u);
                else
                  umma_f16_pair(tmem + COL_L, ad, bd, IDESC, (first && lseg_start && q == 0) ? 0u : 1u);
              }
            }
            umma_commit_pair(&empty[s]);  // releases the stage (of both CTAs) once its MMAs have read it
          }
          if (!ok) break;
          umma_commit_pair(&hfull[hb]);
          if ((w + 1) % LWIN == 0 || w == nwin - 1) {
            umma_commit_pair(lfull);
            ++gl;
          }
        }
      }
      // every MMA this thread issued completes before TMEM is released
      umma_commit_pair(mdone);
      mbar_wait_own(mdone, 0, timeout_ns);
    }
    __syncwarp();
  } else {
    // drain warps of both CTAs: as in the single-CTA kernel, on this CTA's 128
    // rows of the pair tile; the even CTA's warp 2 relays every hfull / lfull
    // phase to the odd CTA, whose drain warps arrive on the even CTA's
    // hempty / lempty / tempty
    const int q = warp & 3;
    const int cb = ((warp - 2) >> 2) * DCOLS;
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    const uint32_t lo_addr = tmem + lane_off + COL_LO + cb;
    const bool relay = lead && warp == 2 && lane == 0;
    int gw = 0, gl = 0, tc = 0;
    bool ok = true;
    while (ok) {
      const int slot = tc % TRING;
      bool got = pair_wait(&tfull[slot], (tc / TRING) & 1, abort_flag, peer_abort, timeout_ns);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const int4 e = ring[slot];
      __syncwarp();
      if (lane == 0) {
        if (lead)
          mbar_arrive(&tempty[slot]);
        else
          mbar_arrive_cluster(mapa_rank(&tempty[slot], 0));
      }
      ++tc;
      if (e.x < 0) break;
      const Prob& pr = P.p[e.x];
      const int nkb = pr.K / BK;
      const int nwin = (nkb + WIN_KB - 1) / WIN_KB;
      float acc[DCOLS], HI[DCOLS];
#pragma unroll
      for (int j = 0; j < DCOLS; ++j) acc[j] = HI[j] = 0.f;
      {
        uint32_t z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
        for (int c = 0; c < DCOLS; c += 16) tmem_st16(lo_addr + c, z);
        tmem_st_wait();
      }
      if constexpr (W1) {
        for (int w = 0; w < nkb; ++w, ++gw) {
          const int hb = gw % NH;
          got = pair_wait(&hfull[hb], static_cast<uint32_t>((gw / NH) & 1), abort_flag, peer_abort, timeout_ns);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          if (relay) mbar_arrive_cluster(mapa_rank(&hfull[hb], 1));
          tc_fence_after();
          add_cols(tmem + lane_off + static_cast<uint32_t>(hb) * 128u + cb, acc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (lead)
              mbar_arrive(&hempty[hb]);
            else
              mbar_arrive_cluster(mapa_rank(&hempty[hb], 0));
          }
          if ((w + 1) % FOLD1 == 0 || w == nkb - 1) fold_cols(lo_addr, acc, HI);
        }
      } else
      for (int w = 0; w < nwin; ++w, ++gw) {
        const int hb = gw & 1;
        got = pair_wait(&hfull[hb], (gw >> 1) & 1, abort_flag, peer_abort, timeout_ns);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        if (relay) mbar_arrive_cluster(mapa_rank(&hfull[hb], 1));
        tc_fence_after();
        add_cols(tmem + lane_off + (hb ? COL_H1 : COL_H0) + cb, acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (lead)
            mbar_arrive(&hempty[hb]);
          else
            mbar_arrive_cluster(mapa_rank(&hempty[hb], 0));
        }
        if ((w + 1) % LWIN == 0 || w == nwin - 1) {
          got = pair_wait(lfull, gl & 1, abort_flag, peer_abort, timeout_ns);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          if (relay) mbar_arrive_cluster(mapa_rank(lfull, 1));
          tc_fence_after();
          add_cols(tmem + lane_off + COL_L + cb, acc);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (lead)
              mbar_arrive(lempty);
            else
              mbar_arrive_cluster(mapa_rank(lempty, 0));
          }
          ++gl;
        }
        if ((w + 1) % FOLD == 0 || w == nwin - 1) fold_cols(lo_addr, acc, HI);
      }
      ok = ok && !*abort_flag;
      if (!ok) break;
      const int m0 = e.y + static_cast<int>(rank) * BM, n0 = e.z;
      const int row = m0 + q * 32 + lane;
      const float inv = (1.f / ld_scale(pr.sa)) * (1.f / ld_scale(pr.sb));  // powers of two: exact
#pragma unroll
      for (int c = 0; c < DCOLS; c += 8) {
        uint32_t l[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]),
                       "=r"(l[7])
                     : "r"(lo_addr + c));
        tmem_ld_wait();
        if (row < pr.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = n0 + cb + c + j;
            if (n < pr.N) {
              float2 v = ff_scale(ff_fast_two_sum(HI[c + j], __uint_as_float(l[j])), inv);
              float2* p = pr.out + static_cast<long long>(n) * pr.ldo + row;
              if (pr.mode == OUT_FF_ACCUM) v = ff_add(*p, v);
              *p = v;
            }
          }
        }
      }
    }
    if (!ok && lane == 0) latch_error(st, kErrTimeout, 203);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // the pair's MMAs are done and every copy has landed before TMEM and smem go
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;


EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// 3-D map over the piece-stacked 16-bit matrix: dims {cols, rows, pieces}.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int64_t piece,
              int box_rows, int box_pieces, int npieces, CUtensorMapDataType dtype) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(npieces)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(piece) * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows),
                       static_cast<cuuint32_t>(box_pieces)};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, dtype, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// SM count of the current device (cached per device).
int sm_count(int dev) {
  static std::atomic<int> cache[64];
  int n = cache[dev].load();
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  cache[dev].store(n);
  return n;
}

// Clusters of two CTAs that fit on the device at once (cached per device).
template <int NP, bool W1>
int pair_clusters(int dev) {
  static std::atomic<int> cache[64];
  int n = cache[dev].load();
  if (n > 0) return n;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * 256, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = PAIR_SMEM_BYTES;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaOccupancyMaxActiveClusters(&n, cc_gemm_split3_pair<NP, W1>, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = sm_count(dev) / 2;
  }
  cache[dev].store(n);
  return n;
}

template <int NP, bool PAIR, bool W1 = false>
int launch(const GemmOp* ops, int nops, cudaStream_t stream) {
  static_assert(sizeof(Probs) <= 32000, "launch parameters exceed the kernel parameter limit");
  constexpr int TBM = PAIR ? PAIR_BM : BM;
  Probs P;
  memset(&P, 0, sizeof(P));
  const CUtensorMapDataType dt = NP == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  // window given in 32-term units; FP16 leading products (22 significant
  // bits) lose more to the truncating accumulation than BF16 ones (16 bits),
  // so their default window is half as long
  P.win_kb = std::max(1, tuned_win_kb(NP == 2 ? 2 : 4) * 32 / BK);
  P.lwin = std::max(1, (4096 / BK) / P.win_kb);      // L segment of 4096 K terms
  // longest K first: the queue hands out the longest tiles before the short ones
  std::vector<int> order(nops);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ops[a].K > ops[b].K; });
  int64_t total = 0;
  for (int k = 0; k < nops; ++k) {
    const GemmOp& op = ops[order[k]];
    Prob& pr = P.p[k];
    if (op.mode != OUT_FF_STORE && op.mode != OUT_FF_ACCUM) return -1;
    if (!op.A || !op.B || !op.out) return -1;  // never launch on a missing operand or output
    if (op.M <= 0 || op.N <= 0 || op.K <= 0) return -1;
    if (op.K % BK || op.K > 2147483647LL || op.M > 2147483647LL || op.N > 2147483647LL) return -1;
    if ((reinterpret_cast<uintptr_t>(op.A) | reinterpret_cast<uintptr_t>(op.B)) & 15) return -1;
    if ((op.lda | op.ldb | op.a_piece | op.b_piece) & 7) return -1;
    if (!make_map(&pr.ta, op.A, op.a_rows, op.a_cols, op.lda, op.a_piece, BM, NP, NP, dt)) return -4;
    if (!make_map(&pr.tb, op.B, op.b_rows, op.b_cols, op.ldb, op.b_piece, PAIR ? BN / 2 : BN, NP, NP, dt)) return -4;
    pr.out = static_cast<float2*>(op.out);
    pr.sa = op.scale_a;
    pr.sb = op.scale_b;
    pr.ldo = op.ldo;
    pr.M = static_cast<int>(op.M);
    pr.N = static_cast<int>(op.N);
    pr.K = static_cast<int>(op.K);
    pr.mode = op.mode;
    pr.tri = static_cast<int>(op.tri);
    pr.mt = static_cast<int>((op.M + TBM - 1) / TBM);
    pr.nt = static_cast<int>((op.N + BN - 1) / BN);
    pr.tile0 = static_cast<int>(total);
    total += static_cast<int64_t>(pr.mt) * pr.nt;
    if (total > 2000000000LL) return -1;
  }
  P.nprob = nops;
  P.total = static_cast<int>(total);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -4;
  // the shared-memory opt-in is a per-device function attribute: set it once for every device used
  static std::atomic<uint64_t> attr_set{0};
  if (!(attr_set.load() & (1ull << dev))) {
    const cudaError_t attr_err =
        PAIR ? cudaFuncSetAttribute(cc_gemm_split3_pair<NP, W1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    PAIR_SMEM_BYTES)
        : W1 ? cudaFuncSetAttribute(cc_gemm_split3_w1<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)
             : cudaFuncSetAttribute(cc_gemm_split3_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (attr_err != cudaSuccess) {
      note_cuda(attr_err);
      return -4;
    }
    attr_set.fetch_or(1ull << dev);
  }
  int* queue = ops[0].queue;
  if (!queue) return -1;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), stream);
  if (e == cudaSuccess && PAIR) {
    const int64_t clusters = std::min<int64_t>(total, pair_clusters<NP, W1>(dev));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(2 * clusters), 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = PAIR_SMEM_BYTES;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, cc_gemm_split3_pair<NP, W1>, P, queue, ops[0].status, ops[0].timeout_ns);
    if (e == cudaSuccess) e = cudaPeekAtLastError();
  } else if (e == cudaSuccess) {
    const int64_t ctas = std::min<int64_t>(total, sm_count(dev));
    if (W1)
      cc_gemm_split3_w1<NP><<<static_cast<unsigned>(ctas), NTHREADS, SMEM_BYTES, stream>>>(
          P, queue, ops[0].status, ops[0].timeout_ns);
    else
      cc_gemm_split3_tc<NP><<<static_cast<unsigned>(ctas), NTHREADS, SMEM_BYTES, stream>>>(
          P, queue, ops[0].status, ops[0].timeout_ns);
    e = cudaPeekAtLastError();
  }
  if (e != cudaSuccess) {
    note_cuda(e);
    return -4;
  }
  count_launch();
  return 0;
}

}  // namespace

int gemm_mixed(const GemmOp* ops, int nops, cudaStream_t stream) {
  if (nops < 1 || nops > MAXP) return -1;
  for (int i = 1; i < nops; ++i)
    if (ops[i].pieces != ops[0].pieces) return -1;
  // default: the single-CTA kernel for split BF16, one window per k-block for split FP16 (whose
  // 64-term windows already made the L drain and the double-buffered window handshake its bound)
  int kind = tuned_contraction();
  if (kind == 0) kind = ops[0].pieces == 2 ? 3 : 1;
  if (ops[0].pieces == 3)
    return kind == 2 ? launch<3, true>(ops, nops, stream)
         : kind == 3 ? launch<3, false, true>(ops, nops, stream)
         : kind == 4 ? launch<3, true, true>(ops, nops, stream)
                     : launch<3, false>(ops, nops, stream);
  if (ops[0].pieces == 2)
    return kind == 2 ? launch<2, true>(ops, nops, stream)
         : kind == 3 ? launch<2, false, true>(ops, nops, stream)
         : kind == 4 ? launch<2, true, true>(ops, nops, stream)
                     : launch<2, false>(ops, nops, stream);
  return -1;
}

}  // namespace ccl
