// Device-resident CG state and the accumulator of the vector reductions,
// shared by the vector kernels (blas_kernels.cuh) and the product pass that
// can take the CG step itself (matvec_kernels.cuh).  Declarations only.
#pragma once
#include <type_traits>

#include "nfs_complex.cuh"

namespace nfs {

constexpr int kRedBlocks = 304;   // two blocks per SM on a 152-SM GB300
constexpr int kRedThreads = 256;
constexpr int kMaxPartials = 2048;  // >= the product's p^* A p partials, kRedBlocks and kUpdBlocks
constexpr int kUpdBlocks = 608;     // x/r update grid: four blocks of 512 per SM
constexpr int kUpdThreads = 512;

// CG scalar state of one problem, device resident (an array of P).
struct CGState {
  double rr;        // r^* r of the current residual
  double pAp;       // p^* A p
  double alpha, beta;
  double tol2;      // stop when rr <= tol2
  int it, maxit;
  int done;         // 1: converged, broken down or out of iterations
  int status;       // 0, -6 (no convergence) or -7 (breakdown)
  int npart_a;      // number of valid entries of part_a
  unsigned int arrived;  // blocks of the x/r update that have written their partial
  double part_a[kMaxPartials];  // partials of p^* A p (written by the product or k_dot_re)
  double part_b[kMaxPartials];  // partials of r^* r
};
constexpr long long kStateDoubles = sizeof(CGState) / sizeof(double);
constexpr int kStateInts = (int)(sizeof(CGState) / sizeof(int));
static_assert(sizeof(CGState) % sizeof(double) == 0, "CGState must be a whole number of doubles");

// Partial sums of complex products: single-precision data accumulate in FP32
// over short runs that are folded into FP64 (FP64 arithmetic is scarce on
// this GPU); double-precision data accumulate in FP64.
template <typename C>
struct Acc {
  double d = 0.0;
  __device__ __forceinline__ void add(double v) { d += v; }
  __device__ __forceinline__ double total() const { return d; }
};
template <>
struct Acc<float2> {
  double d = 0.0;
  float f = 0.f;
  int k = 0;
  __device__ __forceinline__ void add(float v) {
    f += v;
    if (++k == 16) {
      d += (double)f;
      f = 0.f;
      k = 0;
    }
  }
  __device__ __forceinline__ double total() const { return d + (double)f; }
};

// Per-thread accumulator and block sum of the CG reductions (the partials
// of p^* A p and r^* r).  Complex64 runs accumulate in double-single
// arithmetic on the FP32 units (hi + lo floats, TwoSum: ~1e-14 of the sum of
// the terms' magnitudes) and complex128 runs in FP64.  FP64 arithmetic is
// scarce on this GPU: a block sum of doubles in every CTA of a pass keeps
// the SM's FP64 pipe busy for microseconds.
template <typename T>
struct RedAcc;
template <>
struct RedAcc<double> {
  using value_type = double;
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add_double(double x) { v += x; }
  // the block's total, valid in thread 0; all threads must call it
  template <int NT>
  __device__ __forceinline__ double block_total() {
    __shared__ double sh[NT / 32];
    double t = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
      r = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
  }
};
template <>
struct RedAcc<float> {
  using value_type = float;
  float hi = 0.f, lo = 0.f;
  // (hi, lo) += (bh, bl): TwoSum of the high parts, the rest to the error, renormalised
  __device__ __forceinline__ static void ds_add(float& hi, float& lo, float bh, float bl) {
    const float s = hi + bh;
    const float bb = s - hi;
    const float e = ((hi - (s - bb)) + (bh - bb)) + (lo + bl);
    hi = s + e;
    lo = e - (hi - s);
  }
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
  }
  // a partial stored as a double, split into two floats
  __device__ __forceinline__ void add_double(double x) {
    const float h = (float)x;
    ds_add(hi, lo, h, (float)(x - (double)h));
  }
  template <int NT>
  __device__ __forceinline__ double block_total() {
    __shared__ float2 sh[NT / 32];
    float th = hi, tl = lo;
    ds_add(th, tl, 0.f, 0.f);  // renormalise
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      ds_add(th, tl, __shfl_xor_sync(0xffffffffu, th, o), __shfl_xor_sync(0xffffffffu, tl, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = make_float2(th, tl);
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
      float rh = lane < NT / 32 ? sh[lane].x : 0.f, rl = lane < NT / 32 ? sh[lane].y : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        ds_add(rh, rl, __shfl_xor_sync(0xffffffffu, rh, o), __shfl_xor_sync(0xffffffffu, rl, o));
      if (lane == 0) r = (double)rh + (double)rl;
    }
    __syncthreads();
    return r;
  }
};
// the accumulator for data of real type R (complex64 or complex128 runs)
template <typename R>
using RedAccFor = RedAcc<typename std::conditional<std::is_same<R, float>::value, float, double>::type>;

}  // namespace nfs
