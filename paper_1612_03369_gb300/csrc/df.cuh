// df.cuh -- double-float ("float-float") arithmetic on the FP32 pipe.
//
// GB300 issues FP32 FMAs at ~74x the rate of FP64 ones, so the particle path
// carries its high-precision intermediates as unevaluated sums hi + lo of
// two binary32 numbers (about 48 significant bits), built from error-free
// transformations:
//   two_sum      Knuth, TAOCP vol. 2: s + e == a + b exactly
//   fast_two_sum Dekker 1971, requires |a| >= |b| (or a == 0)
//   two_prod     with a fused multiply-add: p + e == a * b exactly
// (see also Hida, Li & Bailey, "Algorithms for quad-double precision floating
// point arithmetic", ARITH-15, 2001; Ogita, Rump & Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005).
//
// Every step that must be exact uses the __f*_rn intrinsics, which the
// compiler never contracts into an FMA or reorders.
#pragma once

#include <cuda_runtime.h>

namespace pic {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df_make(p, __fmaf_rn(a, b, -p));
}

// Normalise an unevaluated pair so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ df df_norm(df a) { return two_sum(a.hi, a.lo); }

// a + b (sloppy addition: error <= ~2^-47 (|a| + |b|)).
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_make(-b.hi, -b.lo)); }

// a * b, a and b double-float.
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

// a * b, b a single float.
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// Scaling by a power of two is exact.
__device__ __forceinline__ df df_scale2(df a, float pow2) { return df_make(a.hi * pow2, a.lo * pow2); }

// Accumulator for sums of products: the running high part is kept with
// two_sum, every rounding error and low-order part goes into one float.
struct df_acc {
  float s, e;
};

__device__ __forceinline__ df_acc acc_init(df a) {
  df_acc r;
  r.s = a.hi;
  r.e = a.lo;
  return r;
}

__device__ __forceinline__ df_acc acc_zero() {
  df_acc r;
  r.s = 0.f;
  r.e = 0.f;
  return r;
}

// acc += a * b (a, b double-float); a.lo * b.lo (~2^-48 relative) is dropped.
__device__ __forceinline__ void acc_mad(df_acc& acc, df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  float lo = __fmaf_rn(a.hi, b.lo, p.lo);
  lo = __fmaf_rn(a.lo, b.hi, lo);
  const df s = two_sum(acc.s, p.hi);
  acc.s = s.hi;
  acc.e = __fadd_rn(acc.e, __fadd_rn(s.lo, lo));
}

// acc += a * b, b a single float.
__device__ __forceinline__ void acc_mad_f(df_acc& acc, df a, float b) {
  const df p = two_prod(a.hi, b);
  const float lo = __fmaf_rn(a.lo, b, p.lo);
  const df s = two_sum(acc.s, p.hi);
  acc.s = s.hi;
  acc.e = __fadd_rn(acc.e, __fadd_rn(s.lo, lo));
}

// acc += a (double-float).
__device__ __forceinline__ void acc_add(df_acc& acc, df a) {
  const df s = two_sum(acc.s, a.hi);
  acc.s = s.hi;
  acc.e = __fadd_rn(acc.e, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df acc_result(const df_acc& acc) { return fast_two_sum(acc.s, acc.e); }

// Split an FP64 value into a double-float (two conversions and one FP64
// subtraction: these run on the FP64 pipe, so they are kept off inner loops).
__device__ __forceinline__ df df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return df_make(hi, lo);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace pic
