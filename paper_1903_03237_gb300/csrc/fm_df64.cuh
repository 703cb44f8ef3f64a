// Float-float ("double-float") arithmetic on the FP32 pipes: a value is hi + lo with
// |lo| <= ulp(hi)/2, about 48 significand bits.  GB300's float64 rate is 1/64 of its
// float32 rate, so the M x M solves of the IP update run in this format instead.
//
// Building blocks are the error-free transformations of Knuth (TwoSum), Dekker
// (Fast2Sum) and the FMA-based TwoProduct, composed as in Hida, Li & Bailey, "Library
// for double-double and quad-double arithmetic" (2000) and Joldes, Muller & Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017).  Only additions, multiplications and explicit fmaf are
// used, so the compiler's mul+add contraction cannot change the error terms.
#pragma once
#include <cuda_runtime.h>

namespace fm {

struct df {
  float hi, lo;
};
struct cdf {
  df re, im;
};

__device__ __forceinline__ df df_make(float a) { return df{a, 0.f}; }

// Fast2Sum (|a| >= |b| or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return df{s, b - (s - a)};
}
// TwoSum (no ordering requirement)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df{s, (a - (s - bb)) + (b - bb)};
}
// TwoProduct with FMA
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return df{p, fmaf(a, b, -p)};
}

// Accurate double-word addition (AccurateDWPlusDW)
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  df t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// DWTimesDW (FMA variant)
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  const float t = fmaf(x.hi, y.lo, x.lo * y.hi);
  p.lo += t;
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mulf(df x, float y) {
  df p = two_prod(x.hi, y);
  p.lo = fmaf(x.lo, y, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// Reciprocal: one Newton step on the correctly rounded float32 reciprocal (any float
// range), r = r0 + r0 (1 - x r0), with the residual in float-float.
__device__ __forceinline__ df df_rcp(df x) {
  const float r0 = __frcp_rn(x.hi);
  const df e = df_sub(df_make(1.f), df_mulf(x, r0));  // 1 - x r0
  return df_add(df_make(r0), df_mulf(e, r0));
}
__device__ __forceinline__ df df_div(df a, df b) { return df_mul(a, df_rcp(b)); }

// Square root: s = sqrt(hi); s + (x - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.hi > 0.f)) return df{sqrtf(x.hi), 0.f};
  const float s = sqrtf(x.hi);
  const df e = df_sub(x, two_prod(s, s));
  return fast_two_sum(s, e.hi * (0.5f / s));
}
// 1/sqrt(x) for x > 0: the hardware estimate r0 = rsqrtf(hi), then one Newton-Raphson
// step r = r0 + r0 (1 - x r0^2) / 2 with x r0^2 in float-float (Karp & Markstein, "High-
// precision division and square root", ACM TOMS 1997).  1 - x r0^2 is small, so its float
// value suffices; the relative error is about 1.5 times the square of the estimate's, ~1e-13.
__device__ __forceinline__ df df_rsqrt(df x) {
  // outside [1e-30, 1e30] (r0^2 would leave the normal range): through sqrt and reciprocal
  if (!(x.hi >= 1e-30f && x.hi <= 1e30f)) return df_rcp(df_sqrt(x));
  const float r0 = rsqrtf(x.hi);
  const df t = df_mul(x, two_prod(r0, r0));
  const float e = (1.f - t.hi) - t.lo;  // 1 - t.hi is exact (t.hi is within a few ulp of 1)
  return fast_two_sum(r0, 0.5f * r0 * e);
}
// log(x) for x > 0 to float accuracy of log(hi), plus the first-order term of lo
__device__ __forceinline__ df df_logf(df x) { return two_sum(logf(x.hi), x.lo / x.hi); }

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ df df_from_double(double d) {
  const float hi = (float)d;
  return df{hi, (float)(d - (double)hi)};
}

// ---- complex -------------------------------------------------------------------------
__device__ __forceinline__ cdf cdf_make(float re, float im) { return cdf{df_make(re), df_make(im)}; }
__device__ __forceinline__ cdf cdf_zero() { return cdf{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_conj(cdf a) { return cdf{a.re, df_neg(a.im)}; }
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
  return cdf{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ cdf cdf_cmul(cdf a, cdf b) {
  return cdf{df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }
__device__ __forceinline__ df cdf_abs2(cdf a) { return df_add(df_mul(a.re, a.re), df_mul(a.im, a.im)); }

__device__ __forceinline__ float4 cdf_pack(cdf a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cdf cdf_unpack(float4 v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }

// warp shuffles of df / cdf values
__device__ __forceinline__ df shfl_xor_df(df v, int o) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ cdf shfl_xor_cdf(cdf v, int o) { return cdf{shfl_xor_df(v.re, o), shfl_xor_df(v.im, o)}; }
__device__ __forceinline__ df shfl_df(df v, int src) {
  return df{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ cdf shfl_cdf(cdf v, int src) { return cdf{shfl_df(v.re, src), shfl_df(v.im, src)}; }

}  // namespace fm
