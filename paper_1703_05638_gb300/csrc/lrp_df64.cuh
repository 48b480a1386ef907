// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits. On this
// part FP32 arithmetic runs at 64 times the FP64 rate, so the band kernel
// keeps its implicit-Euler state and computes its refinement residuals in
// this form; every FP64 value entering or leaving the kernel is converted
// at the boundary.
//
// The operations are the error-free transformations of Knuth (TwoSum) and
// Dekker (Fast2Sum, 1971) and the product error from one fused multiply-add
// (exact for FP32 operands); the sum of two double-floats follows the
// accurate variant that adds the low parts with their own error term
// (as in Shewchuk's and Hida-Li-Bailey's double-double arithmetic), so
// cancellation in b - A x keeps close to 48 bits relative to the operands.
#pragma once

#include <cuda_runtime.h>

namespace lrp {

struct df {
  float hi, lo;
};

// s + e = a + b exactly (no precondition)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a + b for a float b
__device__ __forceinline__ df df_add_f(df a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = __fadd_rn(e, a.lo);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// a * b (the error of hi*hi from one FMA; the cross terms rounded once)
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// conversions at the kernel's boundary (one FP64 subtraction each way)
__device__ __forceinline__ df df_from_double(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  return df{hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_load(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}

__device__ __forceinline__ void df_store(float2* p, df a) { *p = make_float2(a.hi, a.lo); }

}  // namespace lrp
