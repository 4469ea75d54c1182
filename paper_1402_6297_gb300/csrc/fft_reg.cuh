// Register-resident small DFTs (lengths dividing 48) with compile-time
// twiddles.  These are the butterflies of the twisted 3-D FFTs that apply T
// and T^* (eq. mtx_T; Section 4.2 applies them as fftn / ifftn).
//
// Sign convention: the forward transform (INV = false) computes
//   X[k] = sum_n x[n] exp(-2 pi i n k / L)     (T^* direction, MATLAB fftn),
// the inverse (INV = true) uses exp(+2 pi i n k / L), unnormalised (T direction).
//
// Composite lengths use one Cooley-Tukey split L = P * Q (P = 4, 3 or 2):
//   n = Q p + q, k = k1 + P k2:
//   Y[q][k1] = w_L^{q k1} * sum_p x[Q p + q] w_P^{p k1}
//   X[k1 + P k2] = sum_q Y[q][k1] w_Q^{q k2}
// After full unrolling every twiddle index is a compile-time constant, so the
// branches in twiddle48() fold away and trivial factors (1, -1, +-i) cost no
// multiplications.
#pragma once
#include "nfs_complex.cuh"

namespace nfs {

// cos(2 pi j / 48) for j = 0..12 (first quadrant), correctly rounded doubles.
__host__ __device__ constexpr double kCosQ48(int j) {
  constexpr double t[13] = {1.0,
                            0.9914448613738104,
                            0.9659258262890683,
                            0.9238795325112867,
                            0.8660254037844386,
                            0.7933533402912352,
                            0.7071067811865476,
                            0.6087614290087207,
                            0.5,
                            0.3826834323650898,
                            0.25881904510252074,
                            0.1305261922200516,
                            0.0};
  return t[j];
}

// cos and sin of 2 pi j / 48 for any j in [0, 48), by quadrant symmetry.
__host__ __device__ constexpr double cos48(int j) {
  return (j <= 12) ? kCosQ48(j)
       : (j <= 24) ? -kCosQ48(24 - j)
       : (j <= 36) ? -kCosQ48(j - 24)
                   : kCosQ48(48 - j);
}
__host__ __device__ constexpr double sin48(int j) {
  return (j <= 12) ? kCosQ48(12 - j)
       : (j <= 24) ? kCosQ48(j - 12)
       : (j <= 36) ? -kCosQ48(36 - j)
                   : -kCosQ48(j - 36);
}

// a * exp(s 2 pi i j / 48), s = +1 for the inverse direction, -1 forward.
template <bool INV, typename C>
__device__ __forceinline__ C twiddle48(C a, int j) {
  using R = typename RealOf<C>::type;
  j %= 48;
  if (j == 0) return a;
  if (j == 24) return cneg(a);
  if (j == 12) return INV ? cmul_i(a) : cmul_mi(a);
  if (j == 36) return INV ? cmul_mi(a) : cmul_i(a);
  const R c = (R)cos48(j);
  const R s = INV ? (R)sin48(j) : -(R)sin48(j);
  return mk(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <int L, bool INV>
struct DFT;

template <bool INV>
struct DFT<1, INV> {
  template <typename C> __device__ __forceinline__ static void run(C*) {}
};

template <bool INV>
struct DFT<2, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <bool INV>
struct DFT<3, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    using R = typename RealOf<C>::type;
    const R h = (R)0.8660254037844386;  // sin(2 pi / 3)
    C s = cadd(x[1], x[2]);
    C d = csub(x[1], x[2]);
    C t = mk(x[0].x - (R)0.5 * s.x, x[0].y - (R)0.5 * s.y);
    x[0] = cadd(x[0], s);
    // forward: X1 = t - i h d, X2 = t + i h d; inverse swaps the signs
    C ihd = mk(-h * d.y, h * d.x);
    if (INV) {
      x[1] = cadd(t, ihd);
      x[2] = csub(t, ihd);
    } else {
      x[1] = csub(t, ihd);
      x[2] = cadd(t, ihd);
    }
  }
};

template <bool INV>
struct DFT<4, INV> {
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
    C c = cadd(x[1], x[3]), d = csub(x[1], x[3]);
    C rd = INV ? cmul_i(d) : cmul_mi(d);  // s i d
    x[0] = cadd(a, c);
    x[2] = csub(a, c);
    x[1] = cadd(b, rd);
    x[3] = csub(b, rd);
  }
};

template <int L, bool INV>
struct DFT {
  static_assert(48 % L == 0, "register DFT lengths must divide 48");
  static constexpr int P = (L % 4 == 0) ? 4 : ((L % 3 == 0) ? 3 : 2);
  static constexpr int Q = L / P;
  template <typename C> __device__ __forceinline__ static void run(C* x) {
    C y[L];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      C t[P];
#pragma unroll
      for (int p = 0; p < P; ++p) t[p] = x[Q * p + q];
      DFT<P, INV>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[q * P + k1] = twiddle48<INV>(t[k1], (q * k1) * (48 / L));
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      C t[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) t[q] = y[q * P + k1];
      DFT<Q, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = t[k2];
    }
  }
};

// Two-level split of a line length N = N1 * N2 used by the shared-memory
// line FFT (see fft_smem.cuh).  The first factor of each length is a tuning
// choice (NFS_N1_<N>, picked by autotune.py into tuning.h); both factors must
// be register DFT lengths (divisors of 48).
#ifndef NFS_N1_24
#define NFS_N1_24 6
#endif
#ifndef NFS_N1_32
#define NFS_N1_32 8
#endif
#ifndef NFS_N1_48
#define NFS_N1_48 8
#endif
#ifndef NFS_N1_64
#define NFS_N1_64 8
#endif
#ifndef NFS_N1_96
#define NFS_N1_96 12
#endif
#ifndef NFS_N1_128
#define NFS_N1_128 16
#endif
template <int N, int F1>
struct SplitOf {
  static_assert(N % F1 == 0 && 48 % F1 == 0 && 48 % (N / F1) == 0, "line split factors must divide 48");
  static constexpr int N1 = F1, N2 = N / F1;
};
template <int N> struct LineSplit;
template <> struct LineSplit<8>   { static constexpr int N1 = 8,  N2 = 1; };
template <> struct LineSplit<12>  { static constexpr int N1 = 12, N2 = 1; };
template <> struct LineSplit<16>  { static constexpr int N1 = 16, N2 = 1; };
template <> struct LineSplit<24>  : SplitOf<24, NFS_N1_24> {};
template <> struct LineSplit<32>  : SplitOf<32, NFS_N1_32> {};
template <> struct LineSplit<48>  : SplitOf<48, NFS_N1_48> {};
template <> struct LineSplit<64>  : SplitOf<64, NFS_N1_64> {};
template <> struct LineSplit<96>  : SplitOf<96, NFS_N1_96> {};
template <> struct LineSplit<128> : SplitOf<128, NFS_N1_128> {};

}  // namespace nfs
