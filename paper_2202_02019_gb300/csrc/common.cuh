// Device helpers shared by the ladder kernels: split-BF16 storage, pair
// indexing, PTX wrappers for mbarrier / TMA / tcgen05, bounded waits.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccl {

// ---------------------------------------------------------------- status word
// The first bytes of every workspace hold a device status word; kernels that
// give up a bounded wait latch CC_ERR_TIMEOUT (-5) there.
struct Status {
  int code;
  int where;
};

constexpr int kErrTimeout = -5;

// ---------------------------------------------------------------- split BF16
// x ~= p0 + p1 + p2 with each piece the round-to-nearest BF16 of what the
// previous pieces left over (24 significant bits in total).
struct Split3 {
  __nv_bfloat16 p[3];
};

__device__ __forceinline__ Split3 split3(double x) {
  Split3 s;
  s.p[0] = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(s.p[0]);
  s.p[1] = __double2bfloat16(r);
  r -= (double)__bfloat162float(s.p[1]);
  s.p[2] = __double2bfloat16(r);
  return s;
}

// Element store of an FP64 value for the operand formats: FP64 (one piece),
// split-BF16 (three pieces `piece` elements apart) or scaled split-FP16 (two
// pieces of x * scl; scl is a power of two chosen so that |x| * scl <= 2^14).
template <typename T>
struct Store;

template <>
struct Store<double> {
  static __device__ __forceinline__ void put(double* base, int64_t idx, int64_t /*piece*/, double x, float) {
    base[idx] = x;
  }
};

template <>
struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ void put(__nv_bfloat16* base, int64_t idx, int64_t piece, double x, float) {
    Split3 s = split3(x);
    base[idx] = s.p[0];
    base[idx + piece] = s.p[1];
    base[idx + 2 * piece] = s.p[2];
  }
};

template <>
struct Store<__half> {
  static __device__ __forceinline__ void put(__half* base, int64_t idx, int64_t piece, double x, float scl) {
    const double y = x * static_cast<double>(scl);
    const __half h0 = __double2half(y);
    base[idx] = h0;
    base[idx + piece] = __double2half(y - static_cast<double>(__half2float(h0)));
  }
};

__device__ __forceinline__ float ld_scale(const float* s) { return s ? *s : 1.f; }

// ---------------------------------------------------------------- float-float
// Intermediates of the mixed path are unevaluated sums hi + lo of two FP32
// numbers (48 significant bits).  All arithmetic on them uses FP32 only:
// GB300 runs FP64 arithmetic at about 1/1800 of its BF16 tensor rate, so
// no FP64 instruction may sit in a per-element hot loop.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a = 0
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = ff_two_sum(a.x, b.x);
  return ff_fast_two_sum(s.x, s.y + (a.y + b.y));
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_scale(float2 a, float c) { return make_float2(a.x * c, a.y * c); }

// x = hi + lo  ~=  p0 + p1 + p2, every step in FP32 (hi - p0 and r - p1 are exact)
__device__ __forceinline__ Split3 split3_ff(float2 x) {
  Split3 s;
  s.p[0] = __float2bfloat16_rn(x.x);
  const float r = (x.x - __bfloat162float(s.p[0])) + x.y;
  s.p[1] = __float2bfloat16_rn(r);
  s.p[2] = __float2bfloat16_rn(r - __bfloat162float(s.p[1]));
  return s;
}

// Scratch arithmetic of the two paths: FP64 values (FP64 path) or
// float-float values (mixed path).
template <typename S>
struct Ar;
template <>
struct Ar<double> {
  using V = double;
  static __device__ __forceinline__ V ld(const double* p, int64_t i) { return p[i]; }
  static __device__ __forceinline__ V zero() { return 0.0; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
  static __device__ __forceinline__ V scale(V a, float c) { return a * static_cast<double>(c); }
  static __device__ __forceinline__ double to_d(V a) { return a; }
};
template <>
struct Ar<float2> {
  using V = float2;
  static __device__ __forceinline__ V ld(const float2* p, int64_t i) { return p[i]; }
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ V add(V a, V b) { return ff_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return ff_add(a, ff_neg(b)); }
  static __device__ __forceinline__ V scale(V a, float c) { return ff_scale(a, c); }
  static __device__ __forceinline__ double to_d(V a) {
    return static_cast<double>(a.x) + static_cast<double>(a.y);
  }
};

// Operand store: FP64 path keeps the value, mixed paths split float-float
// values into three BF16 pieces or two scaled FP16 pieces.
template <typename T, typename V>
struct Put;
template <>
struct Put<double, double> {
  static __device__ __forceinline__ void put(double* base, int64_t idx, int64_t, double x, float) { base[idx] = x; }
};
template <>
struct Put<__nv_bfloat16, float2> {
  static __device__ __forceinline__ void put(__nv_bfloat16* base, int64_t idx, int64_t piece, float2 x, float) {
    const Split3 s = split3_ff(x);
    base[idx] = s.p[0];
    base[idx + piece] = s.p[1];
    base[idx + 2 * piece] = s.p[2];
  }
};
// x * scl = h0 + h1 in FP32 arithmetic (scl a power of two: the products are exact)
template <>
struct Put<__half, float2> {
  static __device__ __forceinline__ void put(__half* base, int64_t idx, int64_t piece, float2 x, float scl) {
    const float hi = x.x * scl;
    const __half h0 = __float2half_rn(hi);
    base[idx] = h0;
    base[idx + piece] = __float2half_rn((hi - __half2float(h0)) + x.y * scl);
  }
};

// Two adjacent elements at once (idx even, so the 16-bit pieces of the pair
// form one aligned 32-bit word): the same values as two Put::put calls with
// half the conversions and stores.
template <typename T, typename V>
struct Put2;
template <>
struct Put2<double, double> {
  static __device__ __forceinline__ void put2(double* base, int64_t idx, int64_t, double x0, double x1, float) {
    base[idx] = x0;
    base[idx + 1] = x1;
  }
};
template <>
struct Put2<__nv_bfloat16, float2> {
  static __device__ __forceinline__ void put2(__nv_bfloat16* base, int64_t idx, int64_t piece, float2 x0, float2 x1,
                                              float) {
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(x0.x, x1.x);
    const float2 b0 = __bfloat1622float2(p0);
    const float r0 = (x0.x - b0.x) + x0.y, r1 = (x1.x - b0.y) + x1.y;
    const __nv_bfloat162 p1 = __floats2bfloat162_rn(r0, r1);
    const float2 b1 = __bfloat1622float2(p1);
    const __nv_bfloat162 p2 = __floats2bfloat162_rn(r0 - b1.x, r1 - b1.y);
    *reinterpret_cast<__nv_bfloat162*>(base + idx) = p0;
    *reinterpret_cast<__nv_bfloat162*>(base + idx + piece) = p1;
    *reinterpret_cast<__nv_bfloat162*>(base + idx + 2 * piece) = p2;
  }
};
template <>
struct Put2<__half, float2> {
  static __device__ __forceinline__ void put2(__half* base, int64_t idx, int64_t piece, float2 x0, float2 x1,
                                              float scl) {
    const float hi0 = x0.x * scl, hi1 = x1.x * scl;
    const __half2 h0 = __floats2half2_rn(hi0, hi1);
    const float2 b0 = __half22float2(h0);
    *reinterpret_cast<__half2*>(base + idx) = h0;
    *reinterpret_cast<__half2*>(base + idx + piece) =
        __floats2half2_rn((hi0 - b0.x) + x0.y * scl, (hi1 - b0.y) + x1.y * scl);
  }
};

// ---------------------------------------------------------------- pair index
// Row-major upper triangle of an n x n index square.
//   symmetric pairs  p <= q : k = p*(2n - p + 1)/2 + (q - p)
//   strict pairs     p <  q : k = p*(2n - p - 1)/2 + (q - p - 1)
__host__ __device__ __forceinline__ int64_t pair_sym(int64_t p, int64_t q, int64_t n) {
  return p * (2 * n - p + 1) / 2 + (q - p);
}
__host__ __device__ __forceinline__ int64_t pair_strict(int64_t p, int64_t q, int64_t n) {
  return p * (2 * n - p - 1) / 2 + (q - p - 1);
}

// ---------------------------------------------------------------- PTX: misc
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void latch_error(Status* st, int code, int where) {
  if (st) {
    atomicCAS(&st->code, 0, code);
    st->where = where;
  }
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with parity `parity`, giving up after
// `timeout_ns` or as soon as another role of the CTA raised `*abort`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > timeout_ns) {
      *abort = 1;
      return false;
    }
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 in, FP32 accumulate).
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 columns of 32-bit TMEM words into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// 32 registers per thread into 32 lanes x 32 columns of TMEM.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// 32 lanes x 16 columns (16 registers per thread), load and store.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- CTA pairs (cluster of 2)
// A pair of CTAs on two SMs runs one tcgen05.mma.cta_group::2: the even CTA
// issues it, A comes from both CTAs' shared memory (128 rows each), B from
// both (half of N each), and each CTA's TMEM holds its 128 rows of D.  Every
// tcgen05 instruction of such a kernel carries .cta_group::2.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Shared::cluster address of the variable at `local` (this CTA's shared
// memory) in the shared memory of CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_rank(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
  return r;
}
// Arrive (release at cluster scope) on an mbarrier given by its shared::cluster address.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// try_wait with acquire at cluster scope (for phases completed by the other CTA of the pair).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t cluster_addr, int4 v) {
  asm volatile("st.shared::cluster.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(cluster_addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// Every thread of both CTAs: all shared-memory writes before it are visible to both after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// TMA tile load into this CTA's shared memory whose completion is counted on
// an mbarrier that may live in the other CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(const CUtensorMap* map, uint32_t bar_cluster, void* dst, int c0,
                                                 int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem, both CTAs] (+)= A[smem, both CTAs] * B[smem, both CTAs]^T, M = 256.
__device__ __forceinline__ void umma_f16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on this CTA's `bar` once every pair MMA issued so far by this thread is done.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Shared-memory matrix descriptor (tcgen05), K-major operand, 64-byte swizzle:
// rows of 64 B (32 BF16 along K), 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;                  // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                           // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                           // layout: 64-byte swizzle
  return d;
}

// Same, 128-byte swizzle: rows of 128 B (64 BF16 along K), 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                           // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                           // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: F16 x F16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                      // D format: FP32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

}  // namespace ccl
