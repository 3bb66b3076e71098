// Double-float ("df64") arithmetic: a value is the unevaluated sum h + l of
// two float32 numbers with |l| <= ulp(h)/2, i.e. a 48-bit significand with
// the float32 exponent range. Error-free transformations after Dekker (1971)
// and Knuth (TAOCP vol. 2): TwoSum, Fast2Sum and the FMA-based TwoProd.
//
// On this GPU the float64 pipe issues about 1/60 of the float32 rate, so all
// n x p block data is stored and combined in df64; float64 is kept for the
// p x p matrices only.
#pragma once
#include <cuda_runtime.h>

namespace gsi {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return make_float2(s, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  float2 t = two_sum(a.y, b.y);
  s.y = __fadd_rn(s.y, t.x);
  s = fast_two_sum(s.x, s.y);
  s.y = __fadd_rn(s.y, t.y);
  return fast_two_sum(s.x, s.y);
}

// acc += a b for a dot product: the product exact to ~2^-48 of |a b|
// (TwoProd of the high words plus the cross terms), one TwoSum into acc's
// high word, the low parts summed in float32; acc stays unnormalised (its
// low word may exceed half an ulp of the high one) until df_acc_done. Half
// the instructions of df_add(acc, df_mul(a, b)), for an error of about 2^-46
// of the sum of |a b| per term.
__device__ __forceinline__ void df_dot_acc(float2& acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  const float2 t = two_sum(acc.x, p);
  acc.x = t.x;
  acc.y = __fadd_rn(acc.y, __fadd_rn(t.y, e));
}
__device__ __forceinline__ float2 df_acc_done(float2 acc) { return two_sum(acc.x, acc.y); }

// df + float
__device__ __forceinline__ float2 df_add_f(float2 a, float b) {
  float2 s = two_sum(a.x, b);
  s.y = __fadd_rn(s.y, a.y);
  return fast_two_sum(s.x, s.y);
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}

// a * b + c, all df
__device__ __forceinline__ float2 df_fma(float2 a, float2 b, float2 c) {
  return df_add(df_mul(a, b), c);
}

__host__ __device__ __forceinline__ float2 df_from_double(double x) {
  float h = (float)x;
  float l = (float)(x - (double)h);
  return make_float2(h, l);
}

__host__ __device__ __forceinline__ double df_to_double(float2 v) {
  return (double)v.x + (double)v.y;
}

// 2^e as a float for -126 <= e <= 127
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

}  // namespace gsi
