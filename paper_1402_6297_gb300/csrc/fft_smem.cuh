// Batched 1-D DFTs along lines held in shared memory: the building block of
// the 3-D transforms T q and T^* p (eq. mtx_T, applied by FFT in Section 4.2).
//
// Element e of line l lives at buf[l * LS + e * ES].  A length-N line is
// split N = N1 * N2 (LineSplit): stage A runs, for every (line, n2), a
// register DFT of length N1 over elements {n1 N2 + n2}, multiplies by the
// twiddle w_N^{n2 k1} and writes back to slot k1 N2 + n2; stage B runs, for
// every (line, k1), a register DFT of length N2 over slots {k1 N2 + n2} and
// writes the result to its natural position k1 + N1 k2.
//
// A thread never holds more than one work item's registers.  Stage A's items
// read and write the same slots and are disjoint, so each thread runs its
// items one after another with a single barrier at the end.  Stage B writes
// to other slots than it reads, so it works on chunks of whole lines: a
// chunk's reads and writes touch only its own lines, and the writes of chunk
// i and the reads of chunk i + 1 share one barrier.  Work items take the line
// index fastest across threads: with the odd-padded pitches of the callers
// every shared-memory access of a warp is conflict-free.
//
// tw[m] = exp(-2 pi i m / N), m < N (forward sign; the inverse conjugates).
// Callers must __syncthreads() before; the routine ends with a barrier.
#pragma once
#include "fft_reg.cuh"



namespace nfs {

template <int ITEMS_PER_LINE, int NLINES, int NT>
struct Chunking {
  // lines per chunk: as many whole lines as the block has threads for
  static constexpr int LPC0 = NT / ITEMS_PER_LINE;
  static constexpr int LPC = LPC0 < 1 ? 1 : (LPC0 > NLINES ? NLINES : LPC0);
  static constexpr int CHUNKS = (NLINES + LPC - 1) / LPC;
  static constexpr int ITEMS = LPC * ITEMS_PER_LINE;  // work items per chunk (<= NT when LPC0 >= 1)
};

// The line DFTs with optional global-memory ends: with IN_GLOBAL the first
// stage reads element e of line l as get(l, e) (natural order) instead of
// from buf; with OUT_GLOBAL the last stage hands element k of line l to
// put(l, k, value) instead of writing buf.  Work items take the line index
// fastest across threads, so when consecutive lines are consecutive in global
// memory those accesses are coalesced.  buf is still the staging area between
// the stages.
template <bool INV, int N, int NLINES, int NT, int LS, int ES, bool IN_GLOBAL, bool OUT_GLOBAL, typename C,
          typename Get, typename Put>
__device__ __forceinline__ void smem_fft_io(C* buf, const C* tw, Get get, Put put) {
  using S = LineSplit<N>;
  constexpr int N1 = S::N1, N2 = S::N2;
  const int tid = threadIdx.x;

  if constexpr (N2 == 1) {
    // single stage: a work item owns its whole line
    constexpr int PA = (NLINES + NT - 1) / NT;
#pragma unroll
    for (int s = 0; s < PA; ++s) {
      const int it = tid + s * NT;
      if ((NLINES % NT) == 0 || it < NLINES) {
        C* base = buf + it * LS;
        C r[N1];
        if constexpr (IN_GLOBAL) {
#pragma unroll
          for (int k = 0; k < N1; ++k) r[k] = get(it, k);
        } else {
#pragma unroll
          for (int k = 0; k < N1; ++k) r[k] = base[k * ES];
        }
        DFT<N1, INV>::run(r);
#pragma unroll
        for (int k = 0; k < N1; ++k) {
          if constexpr (OUT_GLOBAL) {
            put(it, k, r[k]);
          } else {
            base[k * ES] = r[k];
          }
        }
      }
    }
    __syncthreads();
  } else {
    // ---- stage A: items (line, n2) ----
    // the items of stage A read and write the same slots and are disjoint:
    // each thread runs its items one after another, one barrier at the end
    {
      constexpr int ITEMS = NLINES * N2;
      constexpr int PA = (ITEMS + NT - 1) / NT;
#pragma unroll 1
      for (int s = 0; s < PA; ++s) {
        const int it = tid + s * NT;
        if ((ITEMS % NT) == 0 || it < ITEMS) {
          const int l = it % NLINES, n2 = it / NLINES;
          C* base = buf + l * LS + n2 * ES;
          C ra[N1];
          if constexpr (IN_GLOBAL) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) ra[n1] = get(l, n1 * N2 + n2);
          } else {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) ra[n1] = base[n1 * N2 * ES];
          }
          DFT<N1, INV>::run(ra);
#pragma unroll
          for (int k1 = 1; k1 < N1; ++k1) {
            C w = tw[n2 * k1];
            if (INV) w.y = -w.y;
            ra[k1] = cmul(ra[k1], w);
          }
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) base[k1 * N2 * ES] = ra[k1];
        }
      }
      __syncthreads();
    }
    // ---- stage B: items (line, k1) ----
    if constexpr (OUT_GLOBAL) {
      // results leave for global memory: no shared-memory hazards, so each
      // thread runs its items one after another
      constexpr int ITEMS = NLINES * N1;
      constexpr int PB = (ITEMS + NT - 1) / NT;
#pragma unroll 1
      for (int s = 0; s < PB; ++s) {
        const int it = tid + s * NT;
        if ((ITEMS % NT) == 0 || it < ITEMS) {
          const int l = it % NLINES, k1 = it / NLINES;
          const C* base = buf + l * LS + k1 * N2 * ES;
          C rb[N2];
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) rb[n2] = base[n2 * ES];
          DFT<N2, INV>::run(rb);
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) put(l, k1 + N1 * k2, rb[k2]);
        }
      }
      __syncthreads();
    } else {
      using CK = Chunking<N1, NLINES, NT>;
      C rb[N2];
      int l = 0, k1 = 0;
      bool act = false;
#pragma unroll 1
      for (int ch = 0; ch <= CK::CHUNKS; ++ch) {
        if (ch > 0 && act) {
          C* base = buf + l * LS + k1 * ES;
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) base[k2 * N1 * ES] = rb[k2];
        }
        if (ch < CK::CHUNKS) {
          l = ch * CK::LPC + tid % CK::LPC;
          k1 = tid / CK::LPC;
          act = tid < CK::ITEMS && l < NLINES;
          if (act) {
            const C* base = buf + l * LS + k1 * N2 * ES;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) rb[n2] = base[n2 * ES];
            DFT<N2, INV>::run(rb);
          }
        }
        __syncthreads();
      }
    }
  }
}

struct NoGet {
  template <typename L, typename E> __device__ __forceinline__ int operator()(L, E) const { return 0; }
};
struct NoPut {
  template <typename L, typename E, typename V> __device__ __forceinline__ void operator()(L, E, V) const {}
};

// The line DFTs entirely in shared memory (in place).
template <bool INV, int N, int NLINES, int NT, int LS, int ES, typename C>
__device__ __forceinline__ void smem_fft(C* buf, const C* tw) {
  smem_fft_io<INV, N, NLINES, NT, LS, ES, false, false>(buf, tw, NoGet{}, NoPut{});
}

}  // namespace nfs
