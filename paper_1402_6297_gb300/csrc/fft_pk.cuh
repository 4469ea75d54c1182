// Register DFTs on PAIRS of complex64 lines held in structure-of-arrays form:
// the butterflies of the twisted 3-D FFTs T and T^* (eq. mtx_T; Section 4.2
// applies them as ifftn / fftn) for two fields that share every index and
// every twiddle.
//
// A value of type cp2 holds element j of two lines a and b as two packed
// f32x2 registers, re = (Re a_j, Re b_j) and im = (Im a_j, Im b_j).  Every
// operation of a DFT then treats both lines in one instruction: a complex
// addition costs two packed additions for two complex numbers, a product with
// a constant twiddle four packed multiply/fma instructions for two, and a
// product with +-i only swaps the two registers (the sign goes into the next
// addition).  In the A_r product the two lines are the two fields P_r u1 and
// Q_r u2 of the same component (passes 1, 3) or of the same column (pass 2).
//
// Sign convention as fft_reg.cuh: forward (INV = false) is
// X[k] = sum_n x[n] exp(-2 pi i n k / L), inverse unnormalised with +.
#pragma once
#include "fft_reg.cuh"

namespace nfs {

struct __align__(16) cp2 {
  unsigned long long re, im;
};

__device__ __forceinline__ unsigned long long f2pk(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 pk2f(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ unsigned long long vadd(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long vsub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long vmul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a * b + c
__device__ __forceinline__ unsigned long long vfma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// (s, s)
__device__ __forceinline__ unsigned long long splat(float s) { return f2pk(s, s); }

__device__ __forceinline__ cp2 padd(cp2 a, cp2 b) { return {vadd(a.re, b.re), vadd(a.im, b.im)}; }
__device__ __forceinline__ cp2 psub(cp2 a, cp2 b) { return {vsub(a.re, b.re), vsub(a.im, b.im)}; }
// a + i b and a - i b
__device__ __forceinline__ cp2 padd_i(cp2 a, cp2 b) { return {vsub(a.re, b.im), vadd(a.im, b.re)}; }
__device__ __forceinline__ cp2 psub_i(cp2 a, cp2 b) { return {vadd(a.re, b.im), vsub(a.im, b.re)}; }
__device__ __forceinline__ cp2 pneg(cp2 a) {
  const unsigned long long m = splat(-1.0f);
  return {vmul(a.re, m), vmul(a.im, m)};
}
// real scaling of both lines
__device__ __forceinline__ cp2 pscale(cp2 a, unsigned long long s) { return {vmul(a.re, s), vmul(a.im, s)}; }
// a * (c + i s) with splatted c, s
__device__ __forceinline__ cp2 pmul(cp2 a, unsigned long long c, unsigned long long s, unsigned long long ms) {
  return {vfma(a.im, ms, vmul(a.re, c)), vfma(a.im, c, vmul(a.re, s))};
}
// a * w for a twiddle table entry w = {(c, c), (s, s)} (direction folded in)
__device__ __forceinline__ cp2 pmul_tw(cp2 a, cp2 w) {
  return {vsub(vmul(a.re, w.re), vmul(a.im, w.im)), vfma(a.im, w.re, vmul(a.re, w.im))};
}

// a * exp(s 2 pi i j / 48), s = +1 inverse, -1 forward; j is a compile-time
// constant once the callers are unrolled, so every branch folds away.
template <bool INV>
__device__ __forceinline__ cp2 ptw48(cp2 a, int j) {
  j %= 48;
  if (j == 0) return a;
  if (j == 24) return pneg(a);
  const bool plus_i = (j == 12) == INV;  // the product is +i a (else -i a) for j = 12 or 36
  if (j == 12 || j == 36) {
    if (plus_i) {
      return {vmul(a.im, splat(-1.0f)), a.re};
    }
    return {a.im, vmul(a.re, splat(-1.0f))};
  }
  const float c = (float)cos48(j);
  const float s = INV ? (float)sin48(j) : -(float)sin48(j);
  return pmul(a, splat(c), splat(s), splat(-s));
}

template <int L, bool INV>
struct PDFT;

template <bool INV>
struct PDFT<1, INV> {
  __device__ __forceinline__ static void run(cp2*) {}
};

template <bool INV>
struct PDFT<2, INV> {
  __device__ __forceinline__ static void run(cp2* x) {
    const cp2 a = x[0], b = x[1];
    x[0] = padd(a, b);
    x[1] = psub(a, b);
  }
};

template <bool INV>
struct PDFT<3, INV> {
  __device__ __forceinline__ static void run(cp2* x) {
    const cp2 s = padd(x[1], x[2]);
    const cp2 d = psub(x[1], x[2]);
    // t = x0 - s / 2 ; X0 = x0 + s ; X1, X2 = t -+ i h d (forward), t +- i h d (inverse)
    const unsigned long long mh = splat(-0.5f);
    const cp2 t = {vfma(s.re, mh, x[0].re), vfma(s.im, mh, x[0].im)};
    x[0] = padd(x[0], s);
    const cp2 hd = pscale(d, splat(0.8660254037844386f));
    if (INV) {
      x[1] = padd_i(t, hd);
      x[2] = psub_i(t, hd);
    } else {
      x[1] = psub_i(t, hd);
      x[2] = padd_i(t, hd);
    }
  }
};

template <bool INV>
struct PDFT<4, INV> {
  __device__ __forceinline__ static void run(cp2* x) {
    const cp2 a = padd(x[0], x[2]), b = psub(x[0], x[2]);
    const cp2 c = padd(x[1], x[3]), d = psub(x[1], x[3]);
    x[0] = padd(a, c);
    x[2] = psub(a, c);
    if (INV) {
      x[1] = padd_i(b, d);
      x[3] = psub_i(b, d);
    } else {
      x[1] = psub_i(b, d);
      x[3] = padd_i(b, d);
    }
  }
};

// Composite lengths: one Cooley-Tukey split L = P Q (P = 4, 3 or 2), as DFT<L>
// of fft_reg.cuh.
template <int L, bool INV>
struct PDFT {
  static_assert(48 % L == 0, "register DFT lengths must divide 48");
  static constexpr int P = (L % 4 == 0) ? 4 : ((L % 3 == 0) ? 3 : 2);
  static constexpr int Q = L / P;
  __device__ __forceinline__ static void run(cp2* x) {
    cp2 y[L];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      cp2 t[P];
#pragma unroll
      for (int p = 0; p < P; ++p) t[p] = x[Q * p + q];
      PDFT<P, INV>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[q * P + k1] = ptw48<INV>(t[k1], (q * k1) * (48 / L));
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      cp2 t[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) t[q] = y[q * P + k1];
      PDFT<Q, INV>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = t[k2];
    }
  }
};

// Stage A of a split line DFT (N = N1 N2, see fft_smem.cuh): the radix-N1
// DFT of the items elements n1 N2 + n2 and the twiddles w_N^{n2 k1}; tw is the
// table of the transform's direction, tw[m] = {(cos, cos), (+-sin, +-sin)} of
// 2 pi m / N.
template <bool INV, int N1>
__device__ __forceinline__ void pk_stage_a(cp2 (&r)[N1], const cp2* tw, int n2) {
  PDFT<N1, INV>::run(r);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) r[k1] = pmul_tw(r[k1], tw[n2 * k1]);
}

}  // namespace nfs
