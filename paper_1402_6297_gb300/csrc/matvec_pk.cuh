// The complex64 A_r product (eq. factor_mtx, applied as in eq. spd_LS) in the
// paired form: every kernel carries the two fields of the product that share
// all indices and twiddles, P_r u1 and Q_r u2 of one component (passes 1 and
// 3) or of one column (pass 2), as one line pair in structure-of-arrays form
// (fft_pk.cuh).  Same three HBM passes and field layout as matvec_kernels.cuh:
//
//   pass 1  (one CTA per (z-plane i3, component c); no cluster):  spectral
//           assembly of p^_c = (P_r-coefficients)_c and q^_c per voxel from
//           the Lambda tables (the basis is evaluated once for both fields),
//           folded into the first stage of the inverse DFT along x, then the
//           rest of the 2-D inverse DFT; p_c and q_c leave for global memory.
//   pass 2  (one CTA per tile of xy columns):  inverse DFT along z of the six
//           fields, the per-voxel material product, forward DFT along z.
//   pass 3  (one CTA per (z-plane, component)):  forward DFT along y and x
//           of f_c and w_c, in place in the field planes; then a streaming
//           kernel forms the projections P_r^* f and Q_r^* w per voxel from
//           the six transformed fields.  (A cluster of the three component
//           CTAs could project from shared memory, but clusters of three
//           149 KB CTAs co-schedule poorly: a third of the SMs idle.)  The
//           unpaired cluster form of matvec_kernels.cuh is faster at every
//           size measured (96: 38 against 46 us), so this pass is built only
//           with NFS_PK3 = 1.
//
// A CTA of passes 1 and 3 holds its line pair plane as [N][N + 1] elements of
// 16 bytes (odd pitch: row and column accesses of 8 consecutive lanes hit 8
// distinct 16-byte bank groups), 149 KB at N = 96.
#pragma once
#include <cooperative_groups.h>

#include "fft_pk.cuh"
#include "matvec_kernels.cuh"

namespace nfs {

// Paired kernels exist for these plane and z lengths (two stages per line
// DFT); they are used where they measured faster than the unpaired ones on
// GB300: pass 1 at 96 (37.6 against 42.2 us; even at 64, slower at 48), pass
// 2 at 48 to 96 (96: 33.9 against 35.5 us).
__host__ __device__ constexpr bool pk_size(int N) { return N == 24 || N == 32 || N == 48 || N == 64 || N == 96; }
__host__ __device__ constexpr bool pk_plane_used(int N) { return N == 96; }
__host__ __device__ constexpr bool pk_z_used(int N3) { return N3 == 48 || N3 == 64 || N3 == 96; }

// Threads and CTAs per SM of the paired plane passes, per edge length (pass
// 1 keeps a whole stage-A item of N1 voxels' inputs in flight and takes more
// registers per thread than pass 3).
// Pass 1 either folds the spectral assembly into the first DFT stage
// (NFS_PK1_FUSED = 1: a thread loads the inputs of N1 voxels of one row, few
// threads with many registers) or assembles the plane into shared memory
// first (0: every thread assembles voxels in batches with their loads issued
// together, then the DFT stages run from shared memory).
#ifndef NFS_PK1_FUSED
#define NFS_PK1_FUSED 0
#endif
#ifndef NFS_PK1_NT96
#define NFS_PK1_NT96 (NFS_PK1_FUSED ? 384 : 768)
#endif
#ifndef NFS_PK3_NT96
#define NFS_PK3_NT96 768
#endif
__host__ __device__ constexpr int pk_plane_threads(int N, int pass) {
  return N == 96 ? (pass == 1 ? NFS_PK1_NT96 : NFS_PK3_NT96) : N == 64 ? 256 : N == 48 ? 192 : N == 32 ? 128 : 96;
}
__host__ __device__ constexpr int pk_plane_minb(int N, int pass) {
  return N == 96 ? 1 : N == 64 ? (pass == 1 ? 2 : 3) : N == 48 ? (pass == 1 ? 2 : 4) : 4;
}
// xy columns per CTA of the paired z pass (the CG curvature partials are one
// per CTA, so this must equal the unpaired z_tile for complex64), threads and
// CTAs per SM.
constexpr int kPkZTile = 16;
__host__ __device__ constexpr int pk_z_threads(int N3) { return (N3 == 32 || N3 == 24) ? 192 : 384; }
__host__ __device__ constexpr int pk_z_minb(int N3) { return (N3 == 32 || N3 == 24) ? 4 : 2; }

template <int N>
constexpr size_t pk_plane_smem() {
  return (size_t)N * (N + 1) * sizeof(cp2) + 2 * N * sizeof(cp2) + 2 * N * sizeof(float2);
}
template <int N3>
constexpr size_t pk_z_smem() {
  return (size_t)N3 * (3 * kPkZTile + 1) * sizeof(cp2) + 2 * N3 * sizeof(cp2);
}

// Twiddle tables in the paired form, tw[m] = {(cos, cos), (s sin, s sin)} of
// 2 pi m / N with s = -1 forward (the stored float2 table is the forward one).
template <bool INV>
__device__ __forceinline__ cp2 pk_twiddle(float2 w) {
  return {splat(w.x), splat(INV ? -w.y : w.y)};
}

// Stage A in place over NLINES line pairs: element e of line l at
// buf[l LS + e ES]; items (line, n2), line index fastest across threads.
template <bool INV, int N1, int N2, int NT, int NLINES, int LS, int ES>
__device__ __forceinline__ void pk_stage_a_inplace(cp2* buf, const cp2* tw) {
  constexpr int ITEMS = NLINES * N2;
#pragma unroll 1
  for (int it = threadIdx.x; it < ITEMS; it += NT) {
    const int l = it % NLINES, n2 = it / NLINES;
    cp2* base = buf + l * LS + n2 * ES;
    cp2 r[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) r[n1] = base[n1 * N2 * ES];
    pk_stage_a<INV, N1>(r, tw, n2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) base[k1 * N2 * ES] = r[k1];
  }
}

// Stage B in place: items (line, k1) read slots k1 N2 + n2 and write the
// natural positions k1 + N1 k2, so whole lines go per chunk and the writes
// of one chunk share a barrier with the reads of the next (as in
// fft_smem.cuh).  Ends with a barrier.
template <bool INV, int N1, int N2, int NT, int NLINES, int LS, int ES>
__device__ __forceinline__ void pk_stage_b_inplace(cp2* buf) {
  using CK = Chunking<N1, NLINES, NT>;
  cp2 rb[N2];
  int l = 0, k1 = 0;
  bool act = false;
#pragma unroll 1
  for (int ch = 0; ch <= CK::CHUNKS; ++ch) {
    if (ch > 0 && act) {
      cp2* base = buf + l * LS + k1 * ES;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) base[k2 * N1 * ES] = rb[k2];
    }
    if (ch < CK::CHUNKS) {
      l = ch * CK::LPC + (int)threadIdx.x % CK::LPC;
      k1 = (int)threadIdx.x / CK::LPC;
      act = (int)threadIdx.x < CK::ITEMS && l < NLINES;
      if (act) {
        const cp2* base = buf + l * LS + k1 * N2 * ES;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) rb[n2] = base[n2 * ES];
        PDFT<N2, INV>::run(rb);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------
template <int N, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_pk_pass1(const float2* u, float2* __restrict__ fld, const float2* __restrict__ lam,
           const float2* __restrict__ twx, const float2* __restrict__ twy, int n3, float alpha, float beta,
           const int* __restrict__ skip, const float2* __restrict__ cg_r, const double* __restrict__ cg_beta,
           float2* __restrict__ p_out, BatchStrides bs) {
  using S = LineSplit<N>;
  constexpr int N1 = S::N1, N2 = S::N2;
  constexpr int PITCH = N + 1;
  constexpr int NE = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cp2* buf = reinterpret_cast<cp2*>(smem_raw);
  cp2* tx = buf + N * PITCH;
  cp2* ty = tx + N;
  float2* a1s = reinterpret_cast<float2*>(ty + N);
  float2* a2s = a1s + N;
  const int c = blockIdx.x;
  const int prob = blockIdx.y / n3, i3 = blockIdx.y % n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  u += prob * bs.su;
  fld += prob * bs.sfld;
  lam += (long long)prob * bs.slam;
  float bt = 0.f;
  if (cg_r != nullptr) {
    cg_r += prob * bs.su;
    p_out += prob * bs.su;
    bt = (float)cg_beta[(long long)prob * bs.sstate];
  }
  for (int i = threadIdx.x; i < N; i += NT) {
    tx[i] = pk_twiddle<true>(twx[i]);
    ty[i] = pk_twiddle<true>(twy[i]);
    a1s[i] = lam[i];
    a2s[i] = lam[N + i];
  }
  __syncthreads();
  const long long n = (long long)NE * n3;
  const float2 a3 = lam[2 * N + i3];
  const float2* ub = u + (long long)i3 * NE;
  const float2* rb = cg_r != nullptr ? cg_r + (long long)i3 * NE : nullptr;
  float2* pb = cg_r != nullptr ? p_out + (long long)i3 * NE : nullptr;
  // the component-c basis of eq. mtx_QdPd at voxel (x, y, i3) and the spectral
  // assembly p^ = -c u1a + x u1b, q^ = conj(x) u2a + conj(c) u2b, packed
  auto assemble = [&](int x, float2 a2, float2 v0, float2 v1, float2 v2, float2 v3) -> cp2 {
    const float2 a1 = a1s[x];
    const float2 p1 = mk(beta * a3.x - a2.x, beta * a3.y - a2.y);  // Lambda_p = t x a, t = (alpha, beta, 1)
    const float2 p2 = mk(a1.x - alpha * a3.x, a1.y - alpha * a3.y);
    const float2 p3 = mk(alpha * a2.x - beta * a1.x, alpha * a2.y - beta * a1.y);
    const float rp = rsqrtf(cabs2(p1) + cabs2(p2) + cabs2(p3));
    const float rq = rsqrtf(cabs2(a1) + cabs2(a2) + cabs2(a3));
    // component c of c = Lambda_p / |Lambda_p| and of x = (a x conj(c)) / sqrt(Lambda_q):
    //   x_1 = a2 conj(c_3) - a3 conj(c_2), x_2 = a3 conj(c_1) - a1 conj(c_3), x_3 = a1 conj(c_2) - a2 conj(c_1)
    float2 pc, aa, pa, ab, pbb;
    if (c == 0) {
      pc = p1; aa = a2; pa = p3; ab = a3; pbb = p2;
    } else if (c == 1) {
      pc = p2; aa = a3; pa = p1; ab = a1; pbb = p3;
    } else {
      pc = p3; aa = a1; pa = p2; ab = a2; pbb = p1;
    }
    const float2 cc = mk(pc.x * rp, pc.y * rp);
    const float sc = rp * rq;
    const float2 xd = csub(cmulc(pa, aa), cmulc(pbb, ab));
    const float2 xc = mk(xd.x * sc, xd.y * sc);
    const float2 ph = csub(cmul(xc, v1), cmul(cc, v0));
    const float2 qh = cadd(cmulc(xc, v2), cmulc(cc, v3));
    return {f2pk(ph.x, qh.x), f2pk(ph.y, qh.y)};
  };
#if NFS_PK1_FUSED
  // stage A along x with the spectral assembly: item (row y, n2) holds the
  // voxels x = n1 N2 + n2 of row y (n2 fastest across threads: coalesced loads)
#pragma unroll 1
  for (int it = threadIdx.x; it < N * N2; it += NT) {
    const int n2 = it % N2, y = it / N2;
    const float2 a2 = a2s[y];
    cp2 r[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int x = n1 * N2 + n2;
      const int e = y * N + x;
      float2 v0 = ub[e], v1 = ub[n + e], v2 = ub[2 * n + e], v3 = ub[3 * n + e];
      if (rb != nullptr) {
        // CG direction p = r + beta p_old, written (once per voxel) to p_out
        const float2 g0 = rb[e], g1 = rb[n + e], g2 = rb[2 * n + e], g3 = rb[3 * n + e];
        v0 = mk(g0.x + bt * v0.x, g0.y + bt * v0.y);
        v1 = mk(g1.x + bt * v1.x, g1.y + bt * v1.y);
        v2 = mk(g2.x + bt * v2.x, g2.y + bt * v2.y);
        v3 = mk(g3.x + bt * v3.x, g3.y + bt * v3.y);
        if (c == 0) {
          pb[e] = v0;
          pb[n + e] = v1;
          pb[2 * n + e] = v2;
          pb[3 * n + e] = v3;
        }
      }
      r[n1] = assemble(x, a2, v0, v1, v2, v3);
    }
    pk_stage_a<true, N1>(r, tx, n2);
    cp2* row = buf + y * PITCH;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) row[k1 * N2 + n2] = r[k1];
  }
  __syncthreads();
#else
  // spectral assembly into the plane buffer in natural order, AB voxels per
  // thread at a time with all their loads issued together
  constexpr int AB = 4;
#pragma unroll 1
  for (int eb = threadIdx.x; eb < NE; eb += AB * NT) {
    float2 v[AB][4];
#pragma unroll
    for (int b = 0; b < AB; ++b) {
      const int e = eb + b * NT;
      if (NE % (AB * NT) == 0 || e < NE) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[b][q] = ub[q * n + e];
      }
    }
    if (rb != nullptr) {
      // CG direction p = r + beta p_old, written (once per voxel) to p_out
#pragma unroll
      for (int b = 0; b < AB; ++b) {
        const int e = eb + b * NT;
        if (NE % (AB * NT) == 0 || e < NE) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 g = rb[q * n + e];
            v[b][q] = mk(g.x + bt * v[b][q].x, g.y + bt * v[b][q].y);
            if (c == 0) pb[q * n + e] = v[b][q];
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < AB; ++b) {
      const int e = eb + b * NT;
      if (NE % (AB * NT) == 0 || e < NE) {
        const int x = e % N, y = e / N;
        buf[y * PITCH + x] = assemble(x, a2s[y], v[b][0], v[b][1], v[b][2], v[b][3]);
      }
    }
  }
  __syncthreads();
  pk_stage_a_inplace<true, N1, N2, NT, N, PITCH, 1>(buf, tx);  // along x (rows)
  __syncthreads();
#endif
  pk_stage_b_inplace<true, N1, N2, NT, N, PITCH, 1>(buf);          // along x (rows)
  pk_stage_a_inplace<true, N1, N2, NT, N, 1, PITCH>(buf, ty);      // along y (columns)
  __syncthreads();
  // stage B along y, results to global memory: element y = k1 + N1 k2 of column x
  float2* op = fld + ((long long)c * n3 + i3) * NE;
  float2* oq = fld + ((long long)(3 + c) * n3 + i3) * NE;
#pragma unroll 1
  for (int it = threadIdx.x; it < N * N1; it += NT) {
    const int x = it % N, k1 = it / N;
    cp2 rr[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) rr[n2] = buf[(k1 * N2 + n2) * PITCH + x];
    PDFT<N2, true>::run(rr);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int yy = k1 + N1 * k2;
      const float2 re = pk2f(rr[k2].re), im = pk2f(rr[k2].im);
      op[yy * N + x] = mk(re.x, im.x);
      oq[yy * N + x] = mk(re.y, im.y);
    }
  }
}

// The material of one voxel (Section 4.3 with diagonal eps and mu), loaded
// ahead of its use, and the product of eq. factor_mtx with it:
//   w = Phi^{-1} (xi mu^{-1} p + q),   f = mu^{-1} (zeta w + p)
// (the arithmetic of material_apply in matvec_kernels.cuh).
struct MatVals {
  float ip[3], im[3], g[3];
  __device__ __forceinline__ void load(const MatView<float>& m, long long v) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ip[c] = __ldg(m.inv_phi + c * m.n + v);
      im[c] = m.inv_mu ? __ldg(m.inv_mu + c * m.n + v) : 1.0f;
    }
    if (m.kind == kMediumChiral) {
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] = __ldg(m.gam + c * m.n + v);
    } else {
      g[0] = __ldg(m.gam + v);
      g[1] = g[2] = g[0];
    }
  }
  __device__ __forceinline__ void apply(const MatView<float>& m, const float2* p, const float2* q, float2* f,
                                        float2* w, float scale) const {
    if (m.kind == kMediumChiral) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // xi mu^{-1} p = i g im p;  w = ip (q + i g im p);  zeta w = -i g w;  f = im (p - i g w)
        const float gi = g[c] * im[c];
        const float2 sv = mk(q[c].x - gi * p[c].y, q[c].y + gi * p[c].x);
        const float2 wc = cscale(sv, ip[c]);
        const float2 fc = mk(p[c].x + g[c] * wc.y, p[c].y - g[c] * wc.x);
        w[c] = cscale(wc, scale);
        f[c] = cscale(fc, im[c] * scale);
      }
    } else {
      // pseudochiral pair (a, b): (xi mu^{-1} p)_a = i g im_b p_b and vice versa
      const int a = m.ax_a, b = m.ax_b;
      const float gg = g[0];
      float2 wc[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int o = c == a ? b : (c == b ? a : -1);
        float2 xmp = mk(0.f, 0.f);
        if (o >= 0) {
          const float2 po = pick3<float>(o, p[0], p[1], p[2]);
          const float imo = o == 0 ? im[0] : (o == 1 ? im[1] : im[2]);
          xmp = cmul_i(cscale(po, gg * imo));
        }
        wc[c] = cscale(cadd(q[c], xmp), ip[c]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int o = c == a ? b : (c == b ? a : -1);
        float2 zw = mk(0.f, 0.f);
        if (o >= 0) zw = cmul_mi(cscale(pick3<float>(o, wc[0], wc[1], wc[2]), gg));  // (zeta w)_c = -i g w_o
        w[c] = cscale(wc[c], scale);
        f[c] = cscale(cadd(p[c], zw), im[c] * scale);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// pass 2: inverse z-DFT, material product of eq. factor_mtx, forward z-DFT
// ---------------------------------------------------------------------------
template <int N3, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_pk_pass2(float2* __restrict__ fld, MatView<float> mat, const float2* __restrict__ twz, int ncols, float inv_n,
           const int* __restrict__ skip, double* __restrict__ dot_part, BatchStrides bs) {
  using S = LineSplit<N3>;
  constexpr int N1 = S::N1, N2 = S::N2;
  constexpr int TX = kPkZTile;
  constexpr int LINES = 3 * TX;  // line l = c TX + column: component c, fields p/f and q/w paired
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cp2* buf = reinterpret_cast<cp2*>(smem_raw);
  cp2* ti = buf + N3 * PITCH;
  cp2* tf = ti + N3;
  const int tiles = ncols / TX;
  const int prob = blockIdx.x / tiles;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  fld += prob * bs.sfld;
  mat.inv_phi += prob * bs.smat;
  mat.gam += prob * bs.smat;
  if (mat.inv_mu) mat.inv_mu += prob * bs.smat;
  for (int i = threadIdx.x; i < N3; i += NT) {
    const float2 w = twz[i];
    ti[i] = pk_twiddle<true>(w);
    tf[i] = pk_twiddle<false>(w);
  }
  const int col0 = (blockIdx.x % tiles) * TX;
  const long long n = (long long)ncols * N3;
  __syncthreads();
  // stage A of the inverse DFT from global memory: item (line, n2)
#pragma unroll 1
  for (int it = threadIdx.x; it < LINES * N2; it += NT) {
    const int l = it % LINES, n2 = it / LINES;
    const float2* gp = fld + (long long)(l / TX) * n + col0 + (l % TX);
    const float2* gq = gp + 3 * n;
    cp2 r[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const long long z = (long long)(n1 * N2 + n2) * ncols;
      const float2 p = ldg_c(gp + z), q = ldg_c(gq + z);
      r[n1] = {f2pk(p.x, q.x), f2pk(p.y, q.y)};
    }
    pk_stage_a<true, N1>(r, ti, n2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[(k1 * N2 + n2) * PITCH + l] = r[k1];
  }
  __syncthreads();
  pk_stage_b_inplace<true, N1, N2, NT, LINES, 1, PITCH>(buf);
  // material product per voxel; CG curvature u^* A_r u = sum Re(conj(p) f + conj(q) w)
  // (Parseval; the DFTs carry the factor n that inv_n removes).  The material
  // of all this thread's voxels is loaded first (one memory latency, not one
  // per voxel).
  constexpr int MV = (N3 * TX + NT - 1) / NT;
  MatVals mv[MV];
#pragma unroll
  for (int b = 0; b < MV; ++b) {
    const int idx = threadIdx.x + b * NT;
    if ((N3 * TX) % NT == 0 || idx < N3 * TX) mv[b].load(mat, (long long)(idx / TX) * ncols + col0 + idx % TX);
  }
  RedAcc<float> dot_acc;
#pragma unroll
  for (int b = 0; b < MV; ++b) {
    const int idx = threadIdx.x + b * NT;
    if ((N3 * TX) % NT != 0 && idx >= N3 * TX) continue;
    const int col = idx % TX, z = idx / TX;
    cp2* cell = buf + z * PITCH + col;
    float2 p[3], q[3], f[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const cp2 v = cell[k * TX];
      const float2 re = pk2f(v.re), im = pk2f(v.im);
      p[k] = mk(re.x, im.x);
      q[k] = mk(re.y, im.y);
    }
    mv[b].apply(mat, p, q, f, w, inv_n);
    if (dot_part != nullptr) {
      float sacc = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) sacc += p[k].x * f[k].x + p[k].y * f[k].y + q[k].x * w[k].x + q[k].y * w[k].y;
      dot_acc.add(sacc);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) cell[k * TX] = {f2pk(f[k].x, w[k].x), f2pk(f[k].y, w[k].y)};
  }
  if (dot_part != nullptr) {
    const double tot = dot_acc.block_total<NT>();  // its barriers also order the material writes
    if (threadIdx.x == 0) dot_part[(long long)prob * bs.sstate + blockIdx.x % tiles] = tot;
  } else {
    __syncthreads();
  }
  pk_stage_a_inplace<false, N1, N2, NT, LINES, 1, PITCH>(buf, tf);
  __syncthreads();
  // stage B of the forward DFT, results to global memory
#pragma unroll 1
  for (int it = threadIdx.x; it < LINES * N1; it += NT) {
    const int l = it % LINES, k1 = it / LINES;
    float2* gp = fld + (long long)(l / TX) * n + col0 + (l % TX);
    float2* gq = gp + 3 * n;
    cp2 r[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) r[n2] = buf[(k1 * N2 + n2) * PITCH + l];
    PDFT<N2, false>::run(r);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const long long z = (long long)(k1 + N1 * k2) * ncols;
      const float2 re = pk2f(r[k2].re), im = pk2f(r[k2].im);
      gp[z] = mk(re.x, im.x);
      gq[z] = mk(re.y, im.y);
    }
  }
}

// ---------------------------------------------------------------------------
// pass 3: forward DFT along y and x of the pair (f_c, w_c), in place in fld
// (one CTA per (z-plane, component), no cluster), then the projections in a
// streaming kernel that reads all six transformed fields per voxel
// ---------------------------------------------------------------------------
template <int N, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_pk_pass3(float2* __restrict__ fld, const float2* __restrict__ twx, const float2* __restrict__ twy, int n3,
           const int* __restrict__ skip, BatchStrides bs) {
  using S = LineSplit<N>;
  constexpr int N1 = S::N1, N2 = S::N2;
  constexpr int PITCH = N + 1;
  constexpr int NE = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cp2* buf = reinterpret_cast<cp2*>(smem_raw);
  cp2* tx = buf + N * PITCH;
  cp2* ty = tx + N;
  const int c = blockIdx.x;
  const int prob = blockIdx.y / n3, i3 = blockIdx.y % n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  fld += prob * bs.sfld;
  for (int i = threadIdx.x; i < N; i += NT) {
    tx[i] = pk_twiddle<false>(twx[i]);
    ty[i] = pk_twiddle<false>(twy[i]);
  }
  __syncthreads();
  float2* fp = fld + ((long long)c * n3 + i3) * NE;
  float2* fq = fld + ((long long)(3 + c) * n3 + i3) * NE;
  // stage A along y from global memory: item (column x, n2), elements y = n1 N2 + n2
#pragma unroll 1
  for (int it = threadIdx.x; it < N * N2; it += NT) {
    const int x = it % N, n2 = it / N;
    cp2 r[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int e = (n1 * N2 + n2) * N + x;
      const float2 f = fp[e], w = fq[e];
      r[n1] = {f2pk(f.x, w.x), f2pk(f.y, w.y)};
    }
    pk_stage_a<false, N1>(r, ty, n2);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[(k1 * N2 + n2) * PITCH + x] = r[k1];
  }
  __syncthreads();
  pk_stage_b_inplace<false, N1, N2, NT, N, 1, PITCH>(buf);      // along y (columns)
  pk_stage_a_inplace<false, N1, N2, NT, N, PITCH, 1>(buf, tx);  // along x (rows)
  __syncthreads();
  pk_stage_b_inplace<false, N1, N2, NT, N, PITCH, 1>(buf);
  // results back to the field planes, row by row (coalesced; every CTA read
  // its own planes completely before its first barrier)
#pragma unroll 4
  for (int e = threadIdx.x; e < NE; e += NT) {
    const cp2 v = buf[(e / N) * PITCH + e % N];
    const float2 re = pk2f(v.re), im = pk2f(v.im);
    fp[e] = mk(re.x, im.x);
    fq[e] = mk(re.y, im.y);
  }
}

// The projections of eq. factor_mtx per spectral voxel from the transformed
// fields: Au = [P_r^* f ; Q_r^* w] with
//   P_r^* f = [-sum conj(c) f ; sum conj(x) f],  Q_r^* w = [sum x w ; sum c w].
// Each thread takes V voxels along x, all loads first.
constexpr int kProjThreads = 256;
constexpr int kProjV = 2;
template <int N>
__global__ void __launch_bounds__(kProjThreads)
k_pk_project(const float2* __restrict__ fld, float2* __restrict__ Au, const float2* __restrict__ lam, int n3,
             float alpha, float beta, const int* __restrict__ skip, BatchStrides bs) {
  constexpr int NE = N * N;
  constexpr int PER_CTA = kProjThreads * kProjV;
  constexpr int CTAS_PER_PLANE = (NE + PER_CTA - 1) / PER_CTA;
  const int plane = blockIdx.x / CTAS_PER_PLANE;
  const int prob = plane / n3, i3 = plane % n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  fld += prob * bs.sfld;
  Au += prob * bs.su;
  lam += (long long)prob * bs.slam;
  const long long n = (long long)NE * n3;
  const int e0 = (blockIdx.x % CTAS_PER_PLANE) * PER_CTA + (int)threadIdx.x;
  const float2* f0 = fld + (long long)i3 * NE;
  float2 v[kProjV][6];
#pragma unroll
  for (int b = 0; b < kProjV; ++b) {
    const int e = e0 + b * kProjThreads;
    if (e < NE) {
#pragma unroll
      for (int k = 0; k < 6; ++k) v[b][k] = ldg_c(f0 + k * n + e);
    }
  }
  const float2 a3 = lam[2 * N + i3];
  float2* o = Au + (long long)i3 * NE;
#pragma unroll
  for (int b = 0; b < kProjV; ++b) {
    const int e = e0 + b * kProjThreads;
    if (e < NE) {
      const int x = e % N, y = e / N;
      Basis<float> B;
      make_basis<float>(lam[x], lam[N + y], a3, alpha, beta, B);
      const float2* f = v[b];
      const float2* w = v[b] + 3;
      o[e] = cneg(cadd(cadd(cmulc(B.c[0], f[0]), cmulc(B.c[1], f[1])), cmulc(B.c[2], f[2])));
      o[n + e] = cadd(cadd(cmulc(B.x[0], f[0]), cmulc(B.x[1], f[1])), cmulc(B.x[2], f[2]));
      o[2 * n + e] = cadd(cadd(cmul(B.x[0], w[0]), cmul(B.x[1], w[1])), cmul(B.x[2], w[2]));
      o[3 * n + e] = cadd(cadd(cmul(B.c[0], w[0]), cmul(B.c[1], w[1])), cmul(B.c[2], w[2]));
    }
  }
}

}  // namespace nfs
