// Pair-of-FP32 ("double-float") arithmetic for the residual operator of the
// mixed-precision solve.
//
// A value is hi + lo with hi = fl32(hi + lo); sums and products are formed
// with the error-free transformations of Knuth (two-sum: s = a + b exactly as
// s + e) and of the fused multiply-add (two-product: a b = p + fma(a, b, -p)),
// then renormalised (Dekker's fast two-sum).  The addition is the short form
// (hi parts by two-sum, lo parts added once), with a relative error of a few
// units of 2^-44 away from cancellation; products are within ~2^-45.  That is
// ~1e-12 relative for a whole transform pass, against ~1e-7 in FP32, at FP32
// instruction rates, which on this GPU are 64x the FP64 rate.
//
// Every step uses the _rn intrinsics, which the compiler never contracts into
// fused multiply-adds or reassociates, so the transformations stay exact.
#pragma once
#include "common.cuh"

struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr df(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ constexpr df(double v)
      : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// 16-byte aligned so that a complex value moves as one vector access
struct __align__(16) cdf {
  df x, y;
};
template <> struct cplx_t<df> { typedef cdf type; };

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// quotient by one correction step of the FP32 quotient of the hi parts
__device__ __forceinline__ df operator/(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = a - b * df(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

__device__ __forceinline__ cdf to_cdf(double2 v) { return cdf{df(v.x), df(v.y)}; }
__device__ __forceinline__ double2 to_d2(cdf v) { return make_double2((double)v.x, (double)v.y); }
