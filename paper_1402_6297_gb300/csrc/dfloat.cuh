// Double-single arithmetic: a real number held as an unevaluated sum of two
// floats, hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits, built
// from error-free transformations on the FP32 units (TwoSum, Knuth;
// FastTwoSum, Dekker; TwoProduct by FMA).  On this GPU FP32 arithmetic runs
// about 70 times faster than FP64, so products in this form, accurate to
// ~1e-14, cost far less than complex128 ones.  The templated kernels of the
// A_r product instantiate with R = df, C = dfc unchanged.
#pragma once
#include <cuda_runtime.h>

#include "nfs_complex.cuh"

namespace nfs {

struct df {
  float hi, lo;
  df() = default;
  // from a double: the nearest float and the float nearest the remainder
  __host__ __device__ constexpr df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(int v) : df((double)v) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ df operator+(df a, df b) {
  // the sum of the high parts exactly, the low parts added to its error term
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the high product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }

// 1 / sqrt(x): the float estimate and one Newton step in double-single
__device__ __forceinline__ df rsqrt(df x) {
  const float y0 = rsqrtf(x.hi);
  const df y(y0, 0.f);
  const df e = df(1.0) - x * (y * y);
  return y + df(0.5f * y0, 0.f) * e;
}

struct dfc {
  df x, y;
};

template <> struct CplxOf<df> { using type = dfc; };
template <> struct RealOf<dfc> { using type = df; };
__host__ __device__ __forceinline__ dfc mk(df a, df b) { return dfc{a, b}; }

// The element type of the double-single product in memory: 16 bytes
// (re.hi, re.lo, im.hi, im.lo), loaded and stored as one float4.
__device__ __forceinline__ dfc ldg_c(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{df(v.x, v.y), df(v.z, v.w)};
}

}  // namespace nfs
