// Helpers of the tensor-core kernels (inline PTX for sm_103a): 5th-generation
// MMA (tcgen05.mma, BF16 operands from shared memory, FP32 accumulators in
// tensor memory), tensor-memory allocation and loads, mbarriers with bounded
// waits, bulk asynchronous copies, and the exact BF16 slicing of float pairs.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace etdm {

constexpr int kTmemCols = 512;
constexpr long kMbarSpin = 4000000;

// byte offset of element (row, k), 0 <= k < 16, in a K-step block of one slice:
// canonical K-major no-swizzle layout with the two 8-column core matrices of a
// row group 128 bytes apart (LBO) and row groups 256 bytes apart (SBO)
__host__ __device__ __forceinline__ int kstep_off(int row, int k) {
  return ((k >> 3) << 7) + ((row >> 3) << 8) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  const uint32_t lbo = 128, sbo = 256;
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (sm_100 family); no swizzle
  return d;
}

// kind::f16 with BF16 A and B, FP32 accumulate, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(mbar))
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}

// bounded wait for the completion of the mbarrier phase with parity `parity`;
// false on timeout or, when `stop` is given, once another role has given up
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity,
                                          const volatile int *stop = nullptr) {
  uint32_t done = 0;
  for (long it = 0; !done; ++it) {
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(su32(mbar)), "r"(parity)
        : "memory");
    if (!done && (it > kMbarSpin || (stop && (it & 255) == 255 && *stop))) return false;
  }
  return true;
}

// bulk asynchronous copy global -> shared, completing `bytes` on the mbarrier
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(mbar))
      : "memory");
}

// Issue the loads of 8 columns (from column address t) of the four slice-order
// accumulators, 128 columns apart, for this warp's lane quarter: r[8k + c] =
// accumulator k, column c.  The registers are valid only after tmem_ld_wait(r).
// the same for streams read once: the lines are marked first for eviction from
// L2, which keeps data that is reused (V's fixed-point sums, O slices) resident
__device__ __forceinline__ void bulk_g2s_stream(void *dst, const void *src, uint32_t bytes,
                                                uint64_t *mbar) {
  asm volatile(
      "{ .reg .b64 pol; createpolicy.fractional.L2::evict_first.b64 pol, 1.0; "
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], pol; }" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(mbar))
      : "memory");
}

// 8 columns of four accumulators st columns apart, lane quarter of the warp
__device__ __forceinline__ void tmem_ld_issue(uint32_t t, uint32_t (&r)[32], uint32_t st) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(t), "r"(t + st), "r"(t + 2 * st), "r"(t + 3 * st));
}
// wait for the issued loads; the registers pass through the statement, so no
// use of them can be scheduled before it
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kTmemCols)
               : "memory");
}

// bits of a BF16 number rounded to nearest from x
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// 2^k for -126 <= k <= 127, built from its bits (exact)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// exponent e with |x| 2^(8-e) < 128 for every |x| <= bound; bounds below
// 2^-102 (whose values do not matter) share e = -100, which keeps 2^(8-e) and
// 2^(e-8) normal floats
__device__ __forceinline__ int slice_exp(float bound) {
  return bound > 0.f ? max(ilogbf(bound) + 2, -100) : -100;
}

// Four slices of the float pair x scaled by the power of two sc (|x sc| <= 128):
// x sc = r0 + r1 + r2 + r3 + O(2^-25) with r_k a multiple of 2^-8k and |r_k| <=
// 128 2^-8k.  Each r_k rounds the remainder to its grid by adding and removing
// 1.5 2^(23-8k); the remainders are exact, only the step that adds the low part
// rounds.
template <int NS>
__device__ __forceinline__ void slice_n(float2 x, float sc, float *r) {
  static_assert(NS >= 2 && NS <= 4, "two to four slices");
  const float C0 = 12582912.f, C1 = 49152.f, C2 = 192.f, C3 = 0.75f;
  r[0] = __fadd_rn(__fmaf_rn(x.x, sc, C0), -C0);
  float u = __fmaf_rn(x.y, sc, __fmaf_rn(x.x, sc, -r[0]));
  r[1] = __fadd_rn(__fadd_rn(u, C1), -C1);
  if (NS == 2) return;
  u = __fadd_rn(u, -r[1]);
  r[2] = __fadd_rn(__fadd_rn(u, C2), -C2);
  if (NS == 3) return;
  u = __fadd_rn(u, -r[2]);
  r[3] = __fadd_rn(__fadd_rn(u, C3), -C3);
}
__device__ __forceinline__ void slice4(float2 x, float sc, float *r) { slice_n<4>(x, sc, r); }

// BF16 pair (lo | hi << 16) of two floats with at most 8 significant bits (exact:
// their low 16 bits are zero)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Five slices of the float pair x scaled by the power of two sc (|x.x sc| <
// 128): x sc = r0 + r1 + r2 + r3 + r4 + O(2^-33), r_k a multiple of 2^-8k
// with |r_k| <= 129 2^-8k (integers of at most 8 significant bits: exact in
// BF16).  The high part's remainders are exact; the low part is added only
// after the two leading slices are removed, so its one rounding falls at
// 2^-34 (the four-slice split above adds it at 2^-25).
__device__ __forceinline__ void slice5(float2 x, float sc, float *r) {
  const float C0 = 12582912.f, C1 = 49152.f, C2 = 192.f, C3 = 0.75f, C4 = 0.0029296875f;
  r[0] = __fadd_rn(__fmaf_rn(x.x, sc, C0), -C0);
  float u = __fmaf_rn(x.x, sc, -r[0]);  // exact: x.x sc on the 2^-16 grid
  r[1] = __fadd_rn(__fadd_rn(u, C1), -C1);
  u = __fadd_rn(u, -r[1]);              // exact, |u| <= 2^-9
  u = __fmaf_rn(x.y, sc, u);            // the one rounding
  r[2] = __fadd_rn(__fadd_rn(u, C2), -C2);
  u = __fadd_rn(u, -r[2]);
  r[3] = __fadd_rn(__fadd_rn(u, C3), -C3);
  u = __fadd_rn(u, -r[3]);
  r[4] = __fadd_rn(__fadd_rn(u, C4), -C4);
}

}  // namespace etdm
