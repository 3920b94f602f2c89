// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 runs FP64
// at 1/68 of its FP32 rate, so FP64-class accuracy is reached here with the
// error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based TwoProduct, accumulated as in Ogita-Rump-Oishi's compensated dot
// product (Dot2): every product and every addition error is captured exactly and
// summed into a compensation term.  All operations use the _rn intrinsics so the
// compiler can neither contract nor reassociate them.
#pragma once
#include <cuda_runtime.h>

struct df2 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Compensated accumulator: value = s + c.
struct dacc {
  float s, c;
};

__device__ __forceinline__ dacc dacc_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ dacc dacc_from(df2 v) { return {v.hi, v.lo}; }

// a += p + e, p the leading part (error of the addition captured exactly)
__device__ __forceinline__ void dacc_add2(dacc& a, float p, float e) {
  float s, t;
  two_sum(a.s, p, s, t);
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}
__device__ __forceinline__ void dacc_add(dacc& a, df2 v) { dacc_add2(a, v.hi, v.lo); }
__device__ __forceinline__ void dacc_sub(dacc& a, df2 v) { dacc_add2(a, -v.hi, -v.lo); }

// a += w * z with z an exact FP32 value
__device__ __forceinline__ void dacc_fma(dacc& a, df2 w, float z) {
  float p, e;
  two_prod(w.hi, z, p, e);
  e = __fmaf_rn(w.lo, z, e);
  dacc_add2(a, p, e);
}
// a += x * y, both double-float
__device__ __forceinline__ void dacc_fma(dacc& a, df2 x, df2 y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  dacc_add2(a, p, e);
}

__device__ __forceinline__ df2 dacc_get(dacc a) {
  df2 r;
  two_sum(a.s, a.c, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df2 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df2 df_mul(df2 x, df2 y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df2 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// exact scaling by a power of two
__device__ __forceinline__ df2 df_scale2(df2 a, float pow2) { return {__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

// conversions (FP64 unit: one subtraction per value)
__host__ __device__ __forceinline__ df2 df_from_double(double x) {
  df2 r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__host__ __device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }
