// Double-float ("df64") arithmetic on the FP32 pipe: a value is an unevaluated
// sum hi + lo of two floats (about 48 significant bits).  Error-free
// transformations: Knuth's TwoSum, Dekker's FastTwoSum, and the FMA form of
// Dekker's TwoProduct; division by one Newton correction of the float
// quotient (Dekker 1971, "A floating-point technique for extending the
// available precision").  Used where FP32 alone cannot resolve a quantity and
// FP64 (about 1/70 of the FP32 rate on this GPU) would be too slow.
#pragma once

namespace icrs {

struct df { float hi, lo; };

__device__ __forceinline__ df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}
// p + e = a * b exactly (FMA).
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df_make(p, e);
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mul(df_make(q1, 0.f), b));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ df df_from_double(double x) {
  float h = (float)x;
  return df_make(h, (float)(x - (double)h));
}

struct cdf { df x, y; };

}  // namespace icrs
