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

// conversions that use the FP64 pipe (boundaries and small vectors only)
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }
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
