// Device-resident CG state and the accumulator of the vector reductions,
// shared by the vector kernels (blas_kernels.cuh) and the product pass that
// can take the CG step itself (matvec_kernels.cuh).  Declarations only.
#pragma once
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

}  // namespace nfs
