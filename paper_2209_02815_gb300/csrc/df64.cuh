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

#include <cstring>

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

#ifdef __CUDACC__
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

#endif  // __CUDACC__

// FP64 -> double-float from the IEEE 754 bit fields with integer arithmetic (the FP64 pipe
// runs at 1/64 of the FP32 rate here). x = m 2^(e - 52) with a 53-bit significand m;
// hi = m rounded to its top 24 bits (to nearest, ties to even) = x rounded to FP32, and the
// remainder rem = m - hm 2^29 (|rem| <= 2^28, exact) gives lo = RN_FP32(rem) 2^(e - 52),
// i.e. x - hi rounded to FP32: the same pair as df_from_double. Exponents outside
// [-60, 126] (zero, tiny, huge, subnormal, inf, NaN) fall back to df_from_double so that
// hi and the scale 2^(e - 52) stay normal FP32 numbers.
__host__ __device__ __forceinline__ unsigned long long df_bits64(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<unsigned long long>(__double_as_longlong(x));
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}
__host__ __device__ __forceinline__ float df_float_of_bits(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof(f));
  return f;
#endif
}
__host__ __device__ __forceinline__ bool df_split_int(double x, df& out) {
  const unsigned long long b = df_bits64(x);
  const int e = static_cast<int>((b >> 52) & 0x7FF) - 1023;
  if (e < -60 || e > 126) return false;
  const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned hm = static_cast<unsigned>(m >> 29);
  int rem = static_cast<int>(m & ((1ull << 29) - 1));
  if (rem > (1 << 28) || (rem == (1 << 28) && (hm & 1u))) {
    hm += 1u;
    rem -= (1 << 29);
  }
  // hm in [2^23, 2^24]; 2^24 means the rounding carried into the next binade
  const unsigned hbits = (hm == (1u << 24)) ? (static_cast<unsigned>(e + 128) << 23)
                                            : ((static_cast<unsigned>(e + 127) << 23) | (hm - (1u << 23)));
  const float scale = df_float_of_bits(static_cast<unsigned>(e - 52 + 127) << 23);
  const int rs = sign ? -rem : rem;  // exact remainder with the sign of x (+0 when zero)
#ifdef __CUDA_ARCH__
  const float lo = __fmul_rn(__int2float_rn(rs), scale);
#else
  const float lo = static_cast<float>(rs) * scale;
#endif
  out.hi = df_float_of_bits(hbits | sign);
  out.lo = lo;
  return true;
}

#ifdef __CUDACC__
__device__ __forceinline__ df df_from_double_fast(double x) {
  df r;
  if (!df_split_int(x, r)) r = df_from_double(x);
  return r;
}

// element k of an array as a double-float: stored so, or FP64 split on the fly
__device__ __forceinline__ df load_df(const df* a, long long k) { return a[k]; }
__device__ __forceinline__ df load_df(const double* a, long long k) { return df_from_double_fast(a[k]); }
#endif  // __CUDACC__

inline df df_host(double x) {
  const float h = static_cast<float>(x);
  const float l = static_cast<float>(x - static_cast<double>(h));
  return df_make(h, l);
}

}  // namespace h1w
