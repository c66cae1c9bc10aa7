// dfloat.cuh -- double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi),
// about 48 significant bits.  The error-free transformations are the
// classical ones: Knuth's TwoSum (six additions, exact for any order of
// the operands), Dekker's Fast2Sum (|a| >= |b|), and the product error
// through one fused multiply-add.  GB300 issues 64 times more FP32 than
// FP64 operations per clock, so kernels whose FP64 arithmetic would limit
// them below memory bandwidth (the self-energy row) run it here instead.
//
// FP64 <-> double-float conversions use integer operations on the bit
// patterns only (no FP64 or conversion instructions): hi is the double
// rounded to 24 significant bits, lo the remainder kept to 24 bits, so the
// pair represents the double to 2^-48 relative.  Magnitudes outside
// [2^-126, 2^128) are flushed to zero resp. infinity, which the callers'
// finiteness checks report; values below 2^-74 keep only hi.
#pragma once

#include <cstdint>
#include <cstring>

namespace kbe {
namespace df {

struct F2 {
  float hi, lo;
};

__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ float float_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ int clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return v ? __builtin_clz(v) : 32;
#endif
}
__host__ __device__ __forceinline__ float u2f_rn(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(v);
#else
  return (float)v;
#endif
}
__host__ __device__ __forceinline__ float fmaf_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

// FP64 -> double-float by bit manipulation (32-bit integer operations):
// hi = x rounded to 24 significant bits (nearest, ties up), lo = x - hi (at
// most 29 bits, kept to 24 by truncation: 2^-48 relative to x).
__host__ __device__ __forceinline__ F2 from_double(double x) {
  const uint64_t b = bits_of(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t E = (hw >> 20) & 0x7ffu;
  F2 r;
  if (E - 897u >= 254u) {  // |x| < 2^-126 or zero (flushed), |x| >= 2^128, inf, nan
    r.hi = float_of(E < 897u ? sign : (sign | 0x7f800000u | (E == 2047u && ((hw & 0xfffffu) | lw) ? 0x400000u : 0u)));
    r.lo = 0.0f;
    return r;
  }
  const uint32_t rnd = (lw >> 28) & 1u;
  uint32_t h = (0x800000u | ((hw & 0xfffffu) << 3) | (lw >> 29)) + rnd;  // 24 bits, may carry to 2^24
  const int32_t rem = (int32_t)(lw & 0x1fffffffu) - (int32_t)(rnd << 29);  // units of 2^(E-1075)
  const uint32_t carry = h >> 24;
  h >>= carry;
  const uint32_t Eh = E + carry;
  r.hi = float_of(Eh > 1150u ? (sign | 0x7f800000u) : (sign | ((Eh - 896u) << 23) | (h & 0x7fffffu)));
  const uint32_t R = (uint32_t)(rem < 0 ? -rem : rem);
  const uint32_t lsign = rem < 0 ? (sign ^ 0x80000000u) : sign;
  const int p = 31 - clz32(R);             // leading one of R, 0..28 (R != 0)
  const int ef = p + (int)E - 948;         // float exponent field of lo
  if (R == 0u || ef < 1) {
    r.lo = 0.0f;
  } else {
    const uint32_t mant = p >= 23 ? (R >> (p - 23)) : (R << (23 - p));
    r.lo = float_of(lsign | ((uint32_t)ef << 23) | (mant & 0x7fffffu));
  }
  return r;
}

// FP64 -> double-float with fewer integer operations: hi = x truncated to 24
// significant bits, lo = the remaining 29 bits converted to float (rounded)
// and scaled by a power of two.  |lo| <= ulp(hi), error <= 2^-48 relative;
// lo is dropped for |x| < 2^-74.
__host__ __device__ __forceinline__ F2 from_double_fast(double x) {
  const uint64_t b = bits_of(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t E = (hw >> 20) & 0x7ffu;
  F2 r;
  if (E - 897u >= 254u) {  // |x| < 2^-126 or zero (flushed), |x| >= 2^128, inf, nan
    r.hi = float_of(E < 897u ? sign : (sign | 0x7f800000u | (E == 2047u && ((hw & 0xfffffu) | lw) ? 0x400000u : 0u)));
    r.lo = 0.0f;
    return r;
  }
  r.hi = float_of(sign | ((E - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  // lo = (lw mod 2^29) * 2^(E - 1075): the scale's float exponent field is E - 948
  const float scale = E >= 949u ? float_of((E - 948u) << 23) : 0.0f;
  r.lo = float_of(bits_of(u2f_rn(lw & 0x1fffffffu) * scale) | sign);
  return r;
}

// true when the float is neither infinite nor nan
__host__ __device__ __forceinline__ bool finite_bits(float f) { return (bits_of(f) & 0x7f800000u) != 0x7f800000u; }

// The bits of a float f shifted left by 29 (sign kept) are a double equal to
// f * 2^-896 exactly (the 8-bit exponent field lands in the low bits of the
// 11-bit one; float subnormals land on double subnormals), so hi + lo is one
// FP64 addition of two re-biased words, and the exponent is moved back by
// an integer add.  Results below 2^-126 in magnitude are flushed to zero;
// hi must be finite (callers check it on the float words).
__host__ __device__ __forceinline__ double rebias(float f) {
  const uint32_t b = bits_of(f);
  return double_of(((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(b & 0x7fffffffu) << 29));
}
__host__ __device__ __forceinline__ double to_double(F2 a) {
  const double t = rebias(a.hi) + rebias(a.lo);  // (hi + lo) * 2^-896, rounded once
  const uint64_t tb = bits_of(t);
  const uint32_t hw = (uint32_t)(tb >> 32);
  if ((hw & 0x7ff00000u) == 0u) return double_of((uint64_t)(hw & 0x80000000u) << 32);
  return double_of(tb + ((uint64_t)896 << 52));
}

// Knuth's TwoSum: s + e = a + b exactly.
__host__ __device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  const float e = (a - (s - v)) + (b - v);
  return F2{s, e};
}
// Dekker's Fast2Sum (|a| >= |b| or a == 0).
__host__ __device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return F2{s, b - (s - a)};
}

__host__ __device__ __forceinline__ F2 neg(F2 a) { return F2{-a.hi, -a.lo}; }

// a + b, error of order 2^-47 of |a| + |b| (when a.hi + b.hi cancels, the
// final Fast2Sum may split less exactly, which stays within that bound)
__host__ __device__ __forceinline__ F2 add(F2 a, F2 b) {
  F2 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

// a * b
__host__ __device__ __forceinline__ F2 mul(F2 a, F2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf_(a.hi, b.hi, -p);
  e = fmaf_(a.hi, b.lo, e);
  e = fmaf_(a.lo, b.hi, e);
  e = fmaf_(a.lo, b.lo, e);
  return fast_two_sum(p, e);
}

// a*b + sgn*c*d with one final renormalization (sgn = +1 or -1); error of
// order 2^-47 of |a b| + |c d|
__host__ __device__ __forceinline__ F2 dot2(F2 a, F2 b, F2 c, F2 d, float sgn) {
  const float p = a.hi * b.hi;
  const float q = sgn * (c.hi * d.hi);
  float e = fmaf_(a.hi, b.hi, -p);
  float f = fmaf_(sgn * c.hi, d.hi, -q);
  F2 s = two_sum(p, q);
  float t = s.lo + (e + f);
  t = fmaf_(a.hi, b.lo, t);
  t = fmaf_(a.lo, b.hi, t);
  t = fmaf_(sgn * c.hi, d.lo, t);
  t = fmaf_(sgn * c.lo, d.hi, t);
  return fast_two_sum(s.hi, t);
}

// complex double-float
struct C2 {
  F2 re, im;
};
__host__ __device__ __forceinline__ C2 cadd(C2 a, C2 b) { return C2{add(a.re, b.re), add(a.im, b.im)}; }
// a * b
__host__ __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return C2{dot2(a.re, b.re, a.im, b.im, -1.0f), dot2(a.re, b.im, a.im, b.re, 1.0f)};
}
// a * conj(b)
__host__ __device__ __forceinline__ C2 cmul_cj(C2 a, C2 b) {
  return C2{dot2(a.re, b.re, a.im, b.im, 1.0f), dot2(a.im, b.re, a.re, b.im, -1.0f)};
}
// real scale
__host__ __device__ __forceinline__ C2 cscale(F2 s, C2 a) { return C2{mul(s, a.re), mul(s, a.im)}; }

// ------------------------------------------------ compensated dot products --
// Complex double-float values as float4 (re.hi, re.lo, im.hi, im.lo), and
// real sums kept as Ogita-Rump-Oishi pairs: the leading sum s (a TwoSum per
// term) and a float tail c collecting the TwoSum and product errors.
struct Acc {
  float s, c;
};
// a += x y (x, y double-float: hi, lo; the lo*lo term is below 2^-48)
__device__ __forceinline__ void acc_prod(Acc& a, float xh, float xl, float yh, float yl) {
  const float h = xh * yh;
  float e = fmaf(xh, yh, -h);
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  const float s = a.s + h;
  const float v = s - a.s;
  a.c += ((a.s - (s - v)) + (h - v)) + e;
  a.s = s;
}
// (re, im) += p q
__device__ __forceinline__ void cmac(Acc& re, Acc& im, float4 p, float4 q) {
  acc_prod(re, p.x, p.y, q.x, q.y);
  acc_prod(re, -p.z, -p.w, q.z, q.w);
  acc_prod(im, p.x, p.y, q.z, q.w);
  acc_prod(im, p.z, p.w, q.x, q.y);
}
__device__ __forceinline__ float4 c2f(double2 v) {
  const F2 r = from_double_fast(v.x), i = from_double_fast(v.y);
  return make_float4(r.hi, r.lo, i.hi, i.lo);
}
__device__ __forceinline__ float4 cneg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ float4 cconj(float4 v) { return make_float4(v.x, v.y, -v.z, -v.w); }
// double-float complex sum (error of order 2^-47 of |a| + |b|)
__device__ __forceinline__ float4 cadd4(float4 a, float4 b) {
  const F2 r = add(F2{a.x, a.y}, F2{b.x, b.y});
  const F2 i = add(F2{a.z, a.w}, F2{b.z, b.w});
  return make_float4(r.hi, r.lo, i.hi, i.lo);
}
// the pair's value in FP64
__device__ __forceinline__ double acc_value(Acc a) { return (double)a.s + (double)a.c; }

}  // namespace df
}  // namespace kbe
