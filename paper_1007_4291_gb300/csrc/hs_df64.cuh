// Double-float ("df64") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2,
// giving a 48-bit significand (relative rounding ~2^-47) with the exponent
// range of FP32.  The operations below are the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA form of Dekker's product
// (TwoProd: p = a*b, e = fma(a, b, -p) is exact), combined as in Dekker's
// 1971 double-length arithmetic.  All steps use explicitly rounded
// intrinsics so that the compiler cannot contract or reassociate them.
//
// GB300 executes FP32 at 64 times its FP64 rate, so the Krylov vectors of
// the outer solver (unit-norm Arnoldi vectors, residuals, iterates; no value
// near the FP32 range limits) are kept and combined in this format.
#pragma once
#include <cuda_runtime.h>
#include "hs_internal.cuh"

namespace hs {

struct __align__(8) df {
  float h, l;
};
// complex double-float, 16 bytes: (re.h, re.l, im.h, im.l)
struct __align__(16) cdf {
  df re, im;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  const df t = two_sum(a.l, b.l);
  s.l = __fadd_rn(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.h, b);
  p.l = __fmaf_rn(a.l, b, p.l);
  return fast_two_sum(p.h, p.l);
}
// acc += x * y, renormalised
__device__ __forceinline__ void df_fma(df& acc, df x, df y) {
  const df p = two_prod(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l));
  df s = two_sum(acc.h, p.h);
  s.l = __fadd_rn(s.l, __fadd_rn(acc.l, e));
  acc = fast_two_sum(s.h, s.l);
}
// acc += x * y with a float y
__device__ __forceinline__ void df_fma_f(df& acc, df x, float y) {
  const df p = two_prod(x.h, y);
  const float e = __fmaf_rn(x.l, y, p.l);
  df s = two_sum(acc.h, p.h);
  s.l = __fadd_rn(s.l, __fadd_rn(acc.l, e));
  acc = fast_two_sum(s.h, s.l);
}

// Conversions between FP64 and double-float.  Bulk vectors cross this
// boundary (the ABI's complex128 right-hand sides and solutions, the FP64
// right-hand side of the true residual), so both directions work on the
// IEEE-754 bit fields with integer and FP32 instructions and leave at most one
// FP64 operation per value; GB300's FP64 pipe otherwise bounds those passes.
//
// double -> df: h takes the sign, the exponent (rebiased 1023 -> 127) and the
// top 23 of the 52 stored mantissa bits; the 29 remaining bits, scaled by
// 2^(E-52), become l (an integer-to-float conversion, rounded to 24 bits, and
// a multiplication by a power of two); FastTwoSum then restores |l| <=
// ulp(h)/2.  Relative error about 2^-48.  Zero is exact; values outside the
// normal FP32 range, infinities and NaNs take the FP64 route.
// (kept out of line so that the rare FP64 route is a branch, not predicated
// FP64 instructions issued for every value)
static __device__ __noinline__ df df_from_double_fp64(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
  const int fe = e - 896;                       // FP32 exponent field of h
  if (fe >= 1 && fe <= 254) {
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    const float h = __uint_as_float(sgn | ((unsigned)fe << 23) | (unsigned)(m >> 29));
    float l = 0.f;
    const int pe = e - 948;                     // FP32 exponent field of 2^(E-52)
    if (pe >= 1) {
      const float r = __uint2float_rn((unsigned)(m & 0x1FFFFFFFull));
      l = __fmul_rn(r, __uint_as_float((unsigned)pe << 23));
      if (sgn) l = -l;
    }
    return fast_two_sum(h, l);
  }
  if (e == 0) return df{__uint_as_float(sgn), 0.f};   // zero (and FP64 subnormals, far below FP32's range)
  return df_from_double_fp64(x);
}
static __device__ __noinline__ double f2d_fp64(float f) { return (double)f; }
// float -> double by its bit fields (normal numbers and zero; the rest by
// the conversion instruction), then one FP64 addition.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xFF;
  const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
  if (ef >= 1 && ef <= 254)
    return __longlong_as_double((long long)(sg | ((unsigned long long)(ef + 896) << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
  if ((b & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)sg);
  return f2d_fp64(f);
}
__device__ __forceinline__ double df_to_double(df a) { return f2d_bits(a.h) + f2d_bits(a.l); }
__device__ __forceinline__ cdf cdf_from_c128(c128 z) { return cdf{df_from_double(z.re), df_from_double(z.im)}; }
__device__ __forceinline__ c128 cdf_to_c128(cdf z) { return c128{df_to_double(z.re), df_to_double(z.im)}; }

// complex helpers
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// acc += conj(v) * w
__device__ __forceinline__ void cdf_fma_conj(cdf& acc, cdf v, cdf w) {
  df_fma(acc.re, v.re, w.re);
  df_fma(acc.re, v.im, w.im);
  df_fma(acc.im, v.re, w.im);
  df_fma(acc.im, df_neg(v.im), w.re);
}
// acc -= h * v
__device__ __forceinline__ void cdf_fms(cdf& acc, cdf h, cdf v) {
  df_fma(acc.re, df_neg(h.re), v.re);
  df_fma(acc.re, h.im, v.im);
  df_fma(acc.im, df_neg(h.re), v.im);
  df_fma(acc.im, df_neg(h.im), v.re);
}
// acc += h * z with a complex float z
__device__ __forceinline__ void cdf_fma_c64(cdf& acc, cdf h, c64 z) {
  df_fma_f(acc.re, h.re, z.re);
  df_fma_f(acc.re, df_neg(h.im), z.im);
  df_fma_f(acc.im, h.re, z.im);
  df_fma_f(acc.im, h.im, z.re);
}
// h * z, z complex float
__device__ __forceinline__ cdf cdf_mul_c64(cdf h, c64 z) {
  cdf r{df{0.f, 0.f}, df{0.f, 0.f}};
  cdf_fma_c64(r, h, z);
  return r;
}
// a * b (both double-float complex)
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
  cdf r{df{0.f, 0.f}, df{0.f, 0.f}};
  df_fma(r.re, a.re, b.re);
  df_fma(r.re, df_neg(a.im), b.im);
  df_fma(r.im, a.re, b.im);
  df_fma(r.im, a.im, b.re);
  return r;
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }

}  // namespace hs
