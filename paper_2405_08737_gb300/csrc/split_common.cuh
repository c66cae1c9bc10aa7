// split_common.cuh -- fixed-point digit slicing and tcgen05 helpers of the
// split-precision history slice.
//
// A double v with |v| < 2^e is represented as V = round(v * 2^(31-e)), an
// integer with |V| < 2^31, written in base-256 digits
//   V = d0 2^24 + d1 2^16 + d2 2^8 + d3,
// so v ~= 2^(e-7) (d0 + d1 2^-8 + d2 2^-16 + d3 2^-24).  The history
// operands take the two's-complement bytes of V (d0 = V >> 24 in
// [-128, 127], d1..d3 unsigned in [0, 255]); the small operands take
// balanced digits (d0 in [-128, 128], d1..d3 in [-128, 127]).  Every digit
// is an integer below 2^8 in magnitude, exact in the 16-bit float formats
// of the tensor cores (fp16 here: a byte placed in the mantissa of 1024
// becomes its digit with one packed subtraction); a product of a history
// digit and a small-operand digit is below 2^15 in magnitude and exact in
// FP32, and FP32 sums of such products stay exact while they stay below
// 2^24.  The split path keeps every tensor-core accumulation under that
// bound, forms the digit products of levels d = i + j = 0..4 (the dropped
// levels 5 and 6 weigh below 2^-39 of the product), and folds the
// per-chunk scales in afterwards (Ozaki-style error-free splitting; Ozaki,
// Ogita, Oishi & Rump, Numer. Algorithms 59 (2012)).
//
// Conversions use integer operations on the IEEE-754 bit pattern only (no
// FP64 instructions, which are slow on this part).
#pragma once

#include <cstdint>

namespace kbe {
namespace split {

constexpr int kSlices = 4;       // digits per value
constexpr int kFrac = 31;        // fixed-point bits below the scale
constexpr int kLevels = kSlices + 1;  // digit-product levels d = i + j kept: 0..4

// Unbiased exponent e with |v| < 2^e for the largest magnitude among values
// whose IEEE biased exponent fields have maximum ef (ef = 0 for zero/denormal).
__host__ __device__ __forceinline__ int scale_from_field(int ef) { return ef == 0 ? -1022 : ef - 1022; }

__device__ __forceinline__ int exp_field(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// round(v * 2^(31-e)) as an integer, |v| < 2^e (32-bit integer operations only).
__device__ __forceinline__ int fixed31(double v, int e) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int ef = (hi >> 20) & 0x7FF;
  const int s = 1044 + e - ef;  // right shift of the 53-bit significand, >= 22
  if (ef == 0 || s > 53) return 0;
  const unsigned mh = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
  unsigned V, rb;
  if (s < 32) {
    V = __funnelshift_r(lo, mh, s);
    rb = (lo >> (s - 1)) & 1u;
  } else {
    V = mh >> (s - 32);
    rb = s == 32 ? (lo >> 31) : ((mh >> (s - 33)) & 1u);
  }
  V += rb;
  if (V > 0x7FFFFFFFu) V = 0x7FFFFFFFu;
  return hi < 0 ? -(int)V : (int)V;
}

// round(v * 2^(31-e)) for |v| < 2^e, branch-free in 32-bit operations (the
// same integer as fixed31).  The significand m (53 bits) is shifted right by
// s = 1044 + e - ef >= 22: with x = the top 32 bits of m (m >> 21) and
// t = s - 22, q = x >> t (0 for t > 31) and the rounded quotient is
// (q >> 1) + (q & 1), written so that q = 2^32 - 1 (a value within 2^-32 of
// 2^e, shift 0) gives 2^31 and clamps to 2^31 - 1 instead of wrapping to 0.
__device__ __forceinline__ int fixed31_fast(double v, int e) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int ef = (int)((hi >> 20) & 0x7FFu);
  const unsigned mh = (hi & 0xFFFFFu) | 0x100000u;
  const unsigned x = __funnelshift_l(lo, mh, 11);           // (mh:lo) >> 21, 32 bits
  const unsigned t = (unsigned)(1022 + e - ef);             // s - 22
  const unsigned q = __funnelshift_rc(x, 0u, t);             // shifts of 32 or more give 0
  unsigned V = (q >> 1) + (q & 1u);
  V = ef == 0 ? 0u : min(V, 0x7FFFFFFFu);
  const unsigned sg = (unsigned)((int)hi >> 31);            // 0 or all ones
  return (int)((V ^ sg) - sg);
}

// Digit K of Vr and Vi in the history operands' form (K = 0: the signed
// top byte V >> 24; K = 1..3: the unsigned byte (V >> (24 - 8 K)) & 255) as
// a packed fp16 pair, re in the low half.  One byte permute gathers the two
// bytes, one logic operation puts each into the low mantissa bits of the
// fp16 1024 + b (the top byte with its sign bit flipped: 1152 + d), and one
// packed subtraction of (1024, 1024), resp. (1152, 1152), leaves the digits,
// exactly (fp16 holds every integer of [1024, 2048)).
template <int K>
__device__ __forceinline__ uint32_t digit_pair_f16(int Vr, int Vi) {
  constexpr unsigned kByte = 3 - K;
  const unsigned x = __byte_perm((unsigned)Vr, (unsigned)Vi, kByte | ((kByte + 4) << 8));
  const unsigned bias = K == 0 ? 0x64806480u : 0x64006400u;
  const unsigned w = K == 0 ? ((x & 0x00FF00FFu) ^ 0x64806480u) : ((x & 0x00FF00FFu) | 0x64006400u);
  unsigned r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(w), "r"(bias));
  return r;
}

// Digits as integers (used where the negated digits are needed too).
__device__ __forceinline__ void digits(double v, int e, int d[kSlices]) {
  const int V = fixed31(v, e);
  const unsigned w = (unsigned)V + 0x808080u;
  d[0] = (int)(((long long)V + 0x808080) >> 24);
  d[1] = (int)((w >> 16) & 0xFFu) - 128;
  d[2] = (int)((w >> 8) & 0xFFu) - 128;
  d[3] = (int)(w & 0xFFu) - 128;
}

// fp16 bit pattern of a small integer (|d| <= 2^8, exactly representable):
// d in the low mantissa bits of the fp16 1280 (1280 + d), minus 1280.
__device__ __forceinline__ uint32_t f16_of_int(int d) {
  unsigned r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(0x6500u + (unsigned)d), "r"(0x6500u));
  return r & 0xFFFFu;
}

// Pack (lo, hi) fp16 patterns into one 32-bit word (lo at the lower address).
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) { return (hi << 16) | (lo & 0xFFFFu); }

// ---------------------------------------------------------------- tcgen05 --
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; lbo = byte stride between core matrices along K,
// sbo = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: fp16 x fp16 -> f32, K-major A and B, M = 128.
__host__ __device__ __forceinline__ uint32_t umma_idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(void* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(void* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(void* mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(void* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float v[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// kLevels groups of 4 columns at stride `stride` (the digit-product levels
// of 4 output columns), one wait for all of them.
__device__ __forceinline__ void tmem_ld4xL(uint32_t taddr, int stride, float v[kLevels][4]) {
  uint32_t r[kLevels][4];
#pragma unroll
  for (int d = 0; d < kLevels; ++d)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[d][0]), "=r"(r[d][1]), "=r"(r[d][2]), "=r"(r[d][3])
                 : "r"(taddr + (uint32_t)(d * stride)));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int d = 0; d < kLevels; ++d)
#pragma unroll
    for (int i = 0; i < 4; ++i) v[d][i] = __uint_as_float(r[d][i]);
}

// Zero 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}
// Zero 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(z)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ----------------------------------------------------- double-float sums --
// Error-free sum of two floats (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += x exactly up to the final renormalisation.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  lo += e;
  two_sum(s, lo, hi, lo);
}

// v0 + v1 2^-8 + v2 2^-16 + v3 2^-24 + v4 2^-32 for exact integer levels
// |v_d| < 2^24, as hi + lo: the small levels are folded in FP32 (each
// rounding is below 2^-32 of the level-0 scale), the last step is exact.
__device__ __forceinline__ void combine_levels(const float v[kLevels], float& hi, float& lo) {
  float t = fmaf(v[4], 0.00390625f, v[3]);
  t = fmaf(t, 0.00390625f, v[2]);
  t = fmaf(t, 0.00390625f, v[1]);
  two_sum(v[0], t * 0.00390625f, hi, lo);
}

// Bulk copy global -> shared memory of this CTA, completing on an mbarrier
// (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, void* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
// Arrive on an mbarrier and add `bytes` to its expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(void* mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

// 2^k as a float for k in [-126, 127] (k clamped).
__device__ __forceinline__ float pow2f(int k) {
  k = k < -126 ? -126 : (k > 127 ? 127 : k);
  return __int_as_float((k + 127) << 23);
}

}  // namespace split
}  // namespace kbe
