// Batched 1-D DFTs along lines held in shared memory: the building block of
// the 3-D transforms T q and T^* p (eq. mtx_T, applied by FFT in Section 4.2).
//
// Element e of line l lives at buf[l * LS + e * ES].  A length-N line is
// split N = N1 * N2 (LineSplit): stage A runs, for every (line, n2), a
// register DFT of length N1 over elements {n1 N2 + n2}, multiplies by the
// twiddle w_N^{n2 k1} and writes back to slot k1 N2 + n2; stage B runs, for
// every (line, k1), a register DFT of length N2 over slots {k1 N2 + n2} and
// writes the result to its natural position k1 + N1 k2.  Work items take the
// line index fastest across threads: with the odd-padded pitches used by the
// callers every shared-memory access of a warp is conflict-free.
//
// tw[m] = exp(-2 pi i m / N), m < N (forward sign; the inverse conjugates).
// Callers must __syncthreads() before; the routine ends with a barrier.
#pragma once
#include "fft_reg.cuh"

namespace nfs {

template <bool INV, int N, int NLINES, int NT, int LS, int ES, typename C>
__device__ __forceinline__ void smem_fft(C* buf, const C* tw) {
  using S = LineSplit<N>;
  constexpr int N1 = S::N1, N2 = S::N2;
  constexpr int IA = NLINES * N2;
  constexpr int PA = (IA + NT - 1) / NT;
  const int tid = threadIdx.x;

  if constexpr (N2 == 1) {
    // single stage: a work item owns its whole line, so it writes in place
#pragma unroll
    for (int s = 0; s < PA; ++s) {
      const int it = tid + s * NT;
      if ((IA % NT) == 0 || it < IA) {
        C* base = buf + it * LS;
        C r[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) r[k] = base[k * ES];
        DFT<N1, INV>::run(r);
#pragma unroll
        for (int k = 0; k < N1; ++k) base[k * ES] = r[k];
      }
    }
    __syncthreads();
  } else {
    C ra[PA][N1];
#pragma unroll
    for (int s = 0; s < PA; ++s) {
      const int it = tid + s * NT;
      if ((IA % NT) == 0 || it < IA) {
        const int l = it % NLINES, n2 = it / NLINES;
        const C* base = buf + l * LS + n2 * ES;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) ra[s][n1] = base[n1 * N2 * ES];
        DFT<N1, INV>::run(ra[s]);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
          C w = tw[n2 * k1];
          if (INV) w.y = -w.y;
          ra[s][k1] = cmul(ra[s][k1], w);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < PA; ++s) {
      const int it = tid + s * NT;
      if ((IA % NT) == 0 || it < IA) {
        const int l = it % NLINES, n2 = it / NLINES;
        C* base = buf + l * LS + n2 * ES;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) base[k1 * N2 * ES] = ra[s][k1];
      }
    }
    __syncthreads();

    constexpr int IB = NLINES * N1;
    constexpr int PB = (IB + NT - 1) / NT;
    C rb[PB][N2];
#pragma unroll
    for (int s = 0; s < PB; ++s) {
      const int it = tid + s * NT;
      if ((IB % NT) == 0 || it < IB) {
        const int l = it % NLINES, k1 = it / NLINES;
        const C* base = buf + l * LS + k1 * N2 * ES;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) rb[s][n2] = base[n2 * ES];
        DFT<N2, INV>::run(rb[s]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < PB; ++s) {
      const int it = tid + s * NT;
      if ((IB % NT) == 0 || it < IB) {
        const int l = it % NLINES, k1 = it / NLINES;
        C* base = buf + l * LS + k1 * ES;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) base[k2 * N1 * ES] = rb[s][k2];
      }
    }
    __syncthreads();
  }
}

}  // namespace nfs
