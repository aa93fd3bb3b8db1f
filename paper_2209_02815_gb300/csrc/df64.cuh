// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits. GB300 issues
// FP32 at 64 times its FP64 rate, so a double-float operation (4 to 20 FP32
// instructions) is several times cheaper than an FP64 instruction. The
// building blocks are the classical error-free transformations: Knuth's
// TwoSum, the Fast-TwoSum of Dekker for ordered operands, and the
// FMA-based exact product. Every operation below is written out explicitly
// (no reassociation; the explicit fmaf calls fix where FMAs are used).
#pragma once

#include <cuda_runtime.h>

namespace h1w {

struct df {
  float hi, lo;
};

__host__ __device__ __forceinline__ df df_make(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

// s + e = a + b exactly, valid when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

// Accurate addition: relative error of order 2^-47 of the result.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Product of two double-floats (exact product of the high parts via FMA).
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// Product with a single float.
__device__ __forceinline__ df df_mul_f(df a, float w) {
  const float p = __fmul_rn(a.hi, w);
  float e = __fmaf_rn(a.hi, w, -p);
  e = __fmaf_rn(a.lo, w, e);
  return fast_two_sum(p, e);
}

// FP64 <-> double-float (the conversions run on the FP64 pipe; use them once per vector pass).
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - static_cast<double>(h));
  return df_make(h, l);
}
__device__ __forceinline__ double df_to_double(df a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

inline df df_host(double x) {
  const float h = static_cast<float>(x);
  const float l = static_cast<float>(x - static_cast<double>(h));
  return df_make(h, l);
}

}  // namespace h1w
