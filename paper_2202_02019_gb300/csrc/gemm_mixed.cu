// Split-BF16 tensor-core contraction for sm_103a (tcgen05 + TMA + TMEM).
//
// Every operand element is stored as three BF16 pieces x = x0 + x1 + x2
// (24 significant bits, each piece the round-to-nearest BF16 of what the
// previous ones left).  One useful product a*b is formed from the six piece
// products whose weight is at least 2^-16 of the leading one:
//   a0b0 + (a0b1 + a1b0 + a0b2 + a1b1 + a2b0),
// the dropped terms are O(2^-24) relative.
//
// Accumulation.  The tensor core adds each K=16 step into its FP32
// accumulator with a truncating (round-toward-zero) alignment, which biases
// every output by about -1.7e-8 per step, growing linearly with K.  So:
//   * the leading product a0b0 goes to its own TMEM accumulator H, which is
//     restarted every WIN_KB k-blocks (128 terms); the drain warps add each
//     window into an error-free FP32 two-sum (hi in registers, lo in TMEM),
//     so the bias never spans more than 8 tensor-core steps;
//   * the five small products (weight <= 2^-8 of the leading one) go to a
//     second accumulator L, drained the same way every LWIN windows (4096
//     terms); its truncation bias is scaled down by that weight.
// H is double-buffered (H0, H1) so the drain of one window overlaps the
// MMAs of the next; the MMA warp waits for the (rare) L drain.  One CTA
// owns a 128 x 128 output tile over the whole K and writes the float-float
// result hi + lo (or adds it to the float-float value already there).
//
// CTA = 10 warps: warp 0 issues TMA loads (one elected lane), warp 1 owns
// TMEM and issues tcgen05.mma (one elected lane), warps 2-9 drain (warp w
// reads TMEM lane quarter w%4, column half (w-2)/4).  Tile 128 x 128 x 32,
// 4-stage smem ring (48 KB per stage: 3 A pieces + 3 B pieces, 64-byte
// swizzle).  TMEM columns: H0 [0,128), H1 [128,256), L [256,384), lo [384,512).
// Every wait is bounded (globaltimer) and latches CC_ERR_TIMEOUT.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gemm.h"

namespace ccl {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 4, NP = 3;
constexpr int WIN_KB = 4;                 // k-blocks per H window (128 K terms)
constexpr int LWIN = 32;                  // H windows per L segment (4096 K terms)
constexpr int A_PIECE = BM * BK * 2;      // 8192 B
constexpr int B_PIECE = BN * BK * 2;      // 8192 B
constexpr int A_STAGE = NP * A_PIECE;     // 24576 B
constexpr int B_STAGE = NP * B_PIECE;     // 24576 B
constexpr int STAGE = A_STAGE + B_STAGE;  // 49152 B
constexpr int SMEM_BYTES = STAGES * STAGE + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_H0 = 0, COL_H1 = 128, COL_L = 256, COL_LO = 384;
constexpr int NTHREADS = 320;
constexpr int NDRAIN = 8;                 // draining warps
constexpr uint32_t IDESC = idesc_bf16_f32(BM, BN);

struct Prob {
  CUtensorMap ta, tb;
  float2* out;
  long long ldo;
  int M, N, K, mode;
};
struct Probs {
  Prob p[2];
};

// piece indices of the six kept products; q = 5 is the leading a0b0
__device__ __forceinline__ void product_pieces(int q, int& pa, int& pb) {
  switch (q) {
    case 0: pa = 2; pb = 0; break;
    case 1: pa = 1; pb = 1; break;
    case 2: pa = 0; pb = 2; break;
    case 3: pa = 1; pb = 0; break;
    case 4: pa = 0; pb = 1; break;
    default: pa = 0; pb = 0; break;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// error-free FP32 accumulation: hi + lo += x
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float t = s - hi;
  const float e = (hi - (s - t)) + (x - t);
  hi = s;
  lo += e;
}

// Drain 64 TMEM columns of this thread's row into (hi, lo[TMEM]), 16 at a time.
__device__ __forceinline__ void drain64(uint32_t src, uint32_t lo_addr, float (&hi)[64]) {
#pragma unroll
  for (int c = 0; c < 64; c += 16) {
    uint32_t r[16], l[16];
    tmem_ld16(src + c, r);
    tmem_ld16(lo_addr + c, l);
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float lo = __uint_as_float(l[j]);
      two_sum_acc(hi[c + j], lo, __uint_as_float(r[j]));
      l[j] = __float_as_uint(lo);
    }
    tmem_st16(lo_addr + c, l);
  }
  tmem_st_wait();
}

__global__ void __launch_bounds__(NTHREADS, 1)
    cc_gemm_split3_tc(const __grid_constant__ Probs P, Status* st, unsigned long long timeout_ns) {
  const Prob& pr = P.p[blockIdx.z];
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  if (n0 >= pr.N || m0 >= pr.M) return;  // whole CTA outside this problem

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* hfull = empty + STAGES;   // [2]
  uint64_t* hempty = hfull + 2;       // [2]
  uint64_t* lfull = hempty + 2;       // [1]
  uint64_t* lempty = lfull + 1;       // [1]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(lempty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = pr.K / BK;
  const int nwin = (nkb + WIN_KB - 1) / WIN_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&hfull[b], 1);
      mbar_init(&hempty[b], NDRAIN);
    }
    mbar_init(lfull, 1);
    mbar_init(lempty, NDRAIN);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch(&pr.ta);
    tma_prefetch(&pr.tb);
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
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait_bounded(&empty[s], ph ^ 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 101);
          break;
        }
        uint8_t* sa = smem + s * STAGE;
        mbar_expect_tx(&full[s], STAGE);
        tma_load_3d(&pr.ta, &full[s], sa, kb * BK, m0, 0);
        tma_load_3d(&pr.tb, &full[s], sa + A_STAGE, kb * BK, n0, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int w = 0; w < nwin && ok; ++w) {
        const int hb = w & 1;
        const uint32_t hcol = hb ? COL_H1 : COL_H0;
        const bool lseg_start = (w % LWIN) == 0;
        if (w >= 2 && !mbar_wait_bounded(&hempty[hb], ((w >> 1) - 1) & 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 104);
          break;
        }
        if (w > 0 && lseg_start &&
            !mbar_wait_bounded(lempty, ((w / LWIN) - 1) & 1, abort_flag, timeout_ns)) {
          latch_error(st, kErrTimeout, 105);
          break;
        }
        tc_fence_after();
        const int kb_beg = w * WIN_KB, kb_end = min(nkb, (w + 1) * WIN_KB);
        for (int kb = kb_beg; kb < kb_end; ++kb) {
          const int s = kb % STAGES;
          const uint32_t ph = (kb / STAGES) & 1;
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
            for (int q = 0; q < 6; ++q) {
              int pa, pb;
              product_pieces(q, pa, pb);
              const uint64_t ad = sdesc_k_sw64(a_base + pa * A_PIECE + ks * 32);
              const uint64_t bd = sdesc_k_sw64(b_base + pb * B_PIECE + ks * 32);
              if (q == 5)
                umma_f16(tmem + hcol, ad, bd, IDESC, first ? 0u : 1u);
              else
                umma_f16(tmem + COL_L, ad, bd, IDESC, (first && lseg_start && q == 0) ? 0u : 1u);
            }
          }
          umma_commit(&empty[s]);
        }
        umma_commit(&hfull[hb]);
        if ((w + 1) % LWIN == 0 || w == nwin - 1) umma_commit(lfull);
      }
    }
    __syncwarp();
  } else {
    // drain warps: hi in registers, lo in TMEM columns [384, 512)
    const int q = warp & 3;               // TMEM lane quarter
    const int half = (warp - 2) >> 2;     // column half
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    const uint32_t lo_addr = tmem + lane_off + COL_LO + half * 64;
    float hi[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) hi[j] = 0.f;
    {
      uint32_t z[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) z[j] = 0u;
      tmem_st32(lo_addr, z);
      tmem_st32(lo_addr + 32, z);
      tmem_st_wait();
    }
    bool ok = true;
    for (int w = 0; w < nwin && ok; ++w) {
      const int hb = w & 1;
      bool got = mbar_wait_bounded(&hfull[hb], (w >> 1) & 1, abort_flag, timeout_ns);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const bool lseg_end = (w + 1) % LWIN == 0 || w == nwin - 1;
#pragma unroll 1
      for (int pass = 0; pass < (lseg_end ? 2 : 1); ++pass) {
        if (pass == 1) {
          got = mbar_wait_bounded(lfull, (w / LWIN) & 1, abort_flag, timeout_ns);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
        }
        tc_fence_after();
        const uint32_t src = pass == 0 ? (hb ? COL_H1 : COL_H0) : COL_L;
        drain64(tmem + lane_off + src + half * 64, lo_addr, hi);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (pass == 0)
            mbar_arrive(&hempty[hb]);
          else if (w != nwin - 1)
            mbar_arrive(lempty);
        }
      }
    }
    ok = ok && !*abort_flag;
    if (!ok) {
      if (lane == 0) latch_error(st, kErrTimeout, 103);
    } else {
      const int row = m0 + q * 32 + lane;
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        uint32_t l[16];
        tmem_ld16(lo_addr + c, l);
        tmem_ld_wait();
        if (row < pr.M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + half * 64 + c + j;
            if (n < pr.N) {
              float2 v = ff_fast_two_sum(hi[c + j], __uint_as_float(l[j]));
              float2* p = pr.out + static_cast<long long>(n) * pr.ldo + row;
              if (pr.mode == OUT_FF_ACCUM) v = ff_add(*p, v);
              *p = v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
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

// 3-D map over the piece-stacked BF16 matrix: dims {cols, rows, 3 pieces}.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int64_t piece,
              int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows), 3};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(piece) * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows), 3};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int gemm_mixed(const GemmOp* ops, int nops, cudaStream_t stream) {
  if (nops < 1 || nops > 2) return -1;
  Probs P;
  memset(&P, 0, sizeof(P));
  int64_t mt = 0, nt = 0;
  for (int i = 0; i < nops; ++i) {
    const GemmOp& op = ops[i];
    if (op.mode != OUT_FF_STORE && op.mode != OUT_FF_ACCUM) return -1;
    if (op.M <= 0 || op.N <= 0 || op.K <= 0) return -1;
    if (op.K % BK || op.K > 2147483647LL || op.M > (int64_t)BM * 65535 || op.N > (int64_t)BN * 2147483647LL)
      return -1;
    if ((reinterpret_cast<uintptr_t>(op.A) | reinterpret_cast<uintptr_t>(op.B)) & 15) return -1;
    if ((op.lda | op.ldb | op.a_piece | op.b_piece) & 7) return -1;
    if (!make_map(&P.p[i].ta, op.A, op.a_rows, op.a_cols, op.lda, op.a_piece, BM)) return -4;
    if (!make_map(&P.p[i].tb, op.B, op.b_rows, op.b_cols, op.ldb, op.b_piece, BN)) return -4;
    P.p[i].out = static_cast<float2*>(op.out);
    P.p[i].ldo = op.ldo;
    P.p[i].M = static_cast<int>(op.M);
    P.p[i].N = static_cast<int>(op.N);
    P.p[i].K = static_cast<int>(op.K);
    P.p[i].mode = op.mode;
    mt = std::max<int64_t>(mt, (op.M + BM - 1) / BM);
    nt = std::max<int64_t>(nt, (op.N + BN - 1) / BN);
  }
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(cc_gemm_split3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) return -4;
  dim3 grid(static_cast<unsigned>(nt), static_cast<unsigned>(mt), static_cast<unsigned>(nops));
  cc_gemm_split3_tc<<<grid, NTHREADS, SMEM_BYTES, stream>>>(P, ops[0].status, ops[0].timeout_ns);
  count_launch();
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

}  // namespace ccl
