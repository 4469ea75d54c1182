// The A_r matrix-vector product of the HHPD-NFGEP (eq. factor_mtx, applied
// as in eq. spd_LS) in three HBM passes:
//
//   pass 1  (cluster of 3 CTAs per (z-plane i3, group)):  spectral assembly
//           p^ = P_r-coefficients, q^ = Q_r-coefficients per voxel, then the
//           inverse DFT along x and y.  Group 0 builds p = P_r [u1a; u1b],
//           group 1 builds q = Q_r [u2a; u2b]; CTA rank c owns component c.
//           Each CTA assembles all three components of its third of the
//           plane and the CTAs exchange them through shared memory (Stage).
//   pass 2  (one CTA per tile of xy columns):  inverse DFT along z, the
//           per-voxel material product of eq. factor_mtx, forward DFT along z
//           (the tile goes between global memory and registers directly).
//   pass 3  (cluster of 3 CTAs per (z-plane, group)):  forward DFT along y
//           and x, then the projections P_r^* f (group 0) or Q_r^* w (group 1)
//           from the three transformed components (remote shared loads).
//
// Planes too large for shared memory take the five-pass form of
// matvec_split.cuh.
//
// Basis per spectral voxel (Section 2), with a = (Lambda_1, Lambda_2, Lambda_3),
// t = (alpha, beta, 1), Lambda_p = t x a, Lambda_q = |a|^2:
//   c  = Lambda_p / |Lambda_p|                  (= conj Pi_2, eq. mtx_Pi_2)
//   x  = (a / sqrt(Lambda_q)) x conj(c)          (= Pi_0 x Pi_2 = conj Pi_1)
// so that P_r = (I3 (x) T)[-c, x] and Q_r = (I3 (x) T)[conj x, conj c]
// (eq. mtx_QdPd, SVD theorem thm:svd_C).  x equals conj(Pi_1) because
// Pi_1 = (conj(a) x Lambda_p) / sqrt(Lambda_q |Lambda_p|^2), the unit-norm
// reading of eq. mtx_Pi_1.
//
// The Bloch twist D of T (eq. mtx_T) is a per-voxel unit scalar and commutes
// with the per-voxel material product, so it cancels between T and T^*: the
// kernels run plain DFTs.  The two unnormalised DFTs give a factor n, removed
// in pass 2 (T = D U / sqrt(n)).
//
// Field buffer layout: fld[g][c][i3][j2][j1], g in {p/f, q/w}, c in {x, y, z};
// z is spectral in passes 1 -> 2 and 2 -> 3, x and y are real-space.
#pragma once
#include <cooperative_groups.h>

#include <type_traits>

#include "cg_state.cuh"
#include "fft_smem.cuh"
#include "matvec.h"

namespace nfs {
namespace cg = cooperative_groups;

constexpr int kMediumChiral = 0;
constexpr int kMediumPseudochiral = 1;

// Per-voxel real-space material (Section 4.3 with diagonal eps and mu):
//   inv_phi[3][n] = 1 / Phi_c, Phi = eps - xi mu^{-1} zeta (diagonal here)
//   gam     chiral [3][n] gamma_c; pseudochiral [n] gamma
//   inv_mu  [3][n] = 1 / mu_c, or nullptr for mu = 1
template <typename R>
struct MatView {
  const R* inv_phi;
  const R* gam;
  const R* inv_mu;
  int kind;
  int ax_a, ax_b;
  long long n;
};

// 16-byte vector type holding 16 / sizeof(C) complex elements.
template <typename C> struct Vec16;
template <> struct Vec16<float2> { using type = float4; };
template <> struct Vec16<double2> { using type = double2; };

// How the passes move elements between global and shared memory: EPV
// consecutive elements per lane in one vector V.  One element per lane
// (8-byte accesses for complex64, still 256 contiguous bytes per warp) keeps
// every shared-memory access of a warp on consecutive addresses, free of bank
// conflicts; pairs (16-byte accesses) halve the instruction count but make
// 8-byte shared accesses stride 16 bytes, a two-way conflict.
#ifndef NFS_C64_PAIRS
#define NFS_C64_PAIRS 0
#endif
template <typename C>
struct Lane {
  static constexpr int EPV = (sizeof(C) == 8 && NFS_C64_PAIRS) ? 2 : 1;
  using V = typename std::conditional<EPV == 2, float4, C>::type;
};

// Sum of one double per thread over the block (result valid in thread 0).
template <int NT>
__device__ __forceinline__ double block_sum_dbl(double v) {
  __shared__ double sh[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
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

template <typename R>
struct Basis {
  cplx<R> c[3];
  cplx<R> x[3];
};

template <typename R>
__device__ __forceinline__ void make_basis(cplx<R> a1, cplx<R> a2, cplx<R> a3, R al, R be, Basis<R>& B) {
  using C = cplx<R>;
  // Lambda_p = t x a  (eq. mtx_Lambda_p_q)
  const C p1 = mk(be * a3.x - a2.x, be * a3.y - a2.y);
  const C p2 = mk(a1.x - al * a3.x, a1.y - al * a3.y);
  const C p3 = mk(al * a2.x - be * a1.x, al * a2.y - be * a1.y);
  const R lp2 = cabs2(p1) + cabs2(p2) + cabs2(p3);
  const R lq = cabs2(a1) + cabs2(a2) + cabs2(a3);
  const R rp = rsqrt(lp2);
  const R rq = rsqrt(lq);
  B.c[0] = cscale(p1, rp);
  B.c[1] = cscale(p2, rp);
  B.c[2] = cscale(p3, rp);
  // x = (a / sqrt(Lq)) x conj(c):  x_1 = a2 conj(c3) - a3 conj(c2), cyclic
  B.x[0] = cscale(csub(cmulc(B.c[2], a2), cmulc(B.c[1], a3)), rq);
  B.x[1] = cscale(csub(cmulc(B.c[0], a3), cmulc(B.c[2], a1)), rq);
  B.x[2] = cscale(csub(cmulc(B.c[1], a1), cmulc(B.c[0], a2)), rq);
}

// The basis of spectral voxel v: from the table when there is one, else from
// the Lambda tables.
template <typename R>
__device__ __forceinline__ void voxel_basis(const cplx<R>* __restrict__ table, long long n, long long v, cplx<R> a1,
                                            cplx<R> a2, cplx<R> a3, R al, R be, Basis<R>& B) {
  if (table != nullptr) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      B.c[k] = table[k * n + v];
      B.x[k] = table[(3 + k) * n + v];
    }
  } else {
    make_basis<R>(a1, a2, a3, al, be, B);
  }
}

// Table of the basis (complex128 products use it: double-precision square
// roots are scarce on this GPU).  Grid-stride over P x n voxels.
template <typename R>
__global__ void k_basis_table(const cplx<R>* __restrict__ lam, int n1, int n2, int n3, R al, R be,
                              cplx<R>* __restrict__ table, int P, int slam, long long sbasis) {
  const long long n = (long long)n1 * n2 * n3;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n * P; g += (long long)gridDim.x * blockDim.x) {
    const long long p = g / n, v = g % n;
    const int i1 = (int)(v % n1), i2 = (int)((v / n1) % n2), i3 = (int)(v / ((long long)n1 * n2));
    const cplx<R>* L = lam + p * slam;
    Basis<R> B;
    make_basis<R>(L[i1], L[n1 + i2], L[n1 + n2 + i3], al, be, B);
    cplx<R>* t = table + p * sbasis;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      t[k * n + v] = B.c[k];
      t[(3 + k) * n + v] = B.x[k];
    }
  }
}

// ---------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------

// Element range [e0, e1) of cluster rank r over a plane of NE elements, with
// even boundaries so that 16-byte vectors never straddle two ranks.
template <int NE>
__device__ __forceinline__ int third_bound(int r) {
  return r >= 3 ? NE : ((r * NE) / 3) & ~1;
}

template <typename R>
__device__ __forceinline__ cplx<R> pick3(int k, cplx<R> a, cplx<R> b, cplx<R> c) {
  return k == 0 ? a : (k == 1 ? b : c);
}

// Shared-memory staging of pass 1's exchange.  Rank r computes all three
// components of its third of the plane; its own component goes to its final
// place, the other two to staging gaps of its plane buffer (outside its own
// third's final positions), from which the partner CTAs load them.
template <int NX, int NY>
struct Stage {
  static constexpr int PITCH = NX + 1, NE = NX * NY, TOTAL = NY * PITCH;
  __host__ __device__ static constexpr int pos(int e) { return (e / NX) * PITCH + e % NX; }
  __host__ __device__ static constexpr int e0(int r) { return r >= 3 ? NE : ((r * NE) / 3) & ~1; }
  // start of the staging run of rank r's values of component r + k (k = 1, 2)
  __host__ __device__ static constexpr int base(int r, int k) {
    const int s = e0(r + 1) - e0(r);
    const int lo = pos(e0(r)), hi = pos(e0(r + 1) - 1) + 1, rhi = (hi + 1) & ~1;
    if (lo >= s && TOTAL - rhi >= s) return k == 1 ? 0 : rhi;
    if (TOTAL - rhi >= 2 * s) return k == 1 ? rhi : rhi + s;
    return k == 1 ? 0 : s;
  }
};

// Pass 1's input handling: 0 loads every input block first (all loads in
// flight together), 1 handles one block at a time (fewer live registers).
#ifndef NFS_PASS1_FUSED_LOAD
#define NFS_PASS1_FUSED_LOAD 0
#endif

template <typename R, int NX, int NY, int NT, int MINB>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(NT, MINB)
k_pass1_assemble_ifft_xy(const cplx<R>* u, cplx<R>* __restrict__ fld,
                         const cplx<R>* __restrict__ lam, const cplx<R>* __restrict__ twx,
                         const cplx<R>* __restrict__ twy, int n3, R alpha, R beta,
                         const int* __restrict__ skip, const cplx<R>* __restrict__ cg_r,
                         const double* __restrict__ cg_beta, const cplx<R>* __restrict__ basis, BatchStrides bs) {
  using C = cplx<R>;
  constexpr int PITCH = NX + 1;
  constexpr int NE = NX * NY;
  constexpr int EPV = Lane<C>::EPV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* plane = reinterpret_cast<C*>(smem_raw);
  C* stx = plane + NY * PITCH;
  C* sty = stx + NX;
  cg::cluster_group cl = cg::this_cluster();
  const int prob = blockIdx.z / n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;  // uniform across the cluster
  const int rank = (int)cl.block_rank();
  const int grp = blockIdx.y;
  const int i3 = blockIdx.z % n3;
  u += prob * bs.su;
  fld += prob * bs.sfld;
  lam += (long long)prob * bs.slam;
  if (basis != nullptr) basis += prob * bs.sbasis;
  if (cg_r != nullptr) {
    cg_r += prob * bs.su;
    cg_beta += prob * bs.sstate;
  }
  for (int i = threadIdx.x; i < NX; i += NT) stx[i] = twx[i];
  for (int i = threadIdx.x; i < NY; i += NT) sty[i] = twy[i];

  const long long n = (long long)NE * n3;
  const int e0 = third_bound<NE>(rank), e1 = third_bound<NE>(rank + 1);
  const C* ua = u + (2 * grp) * n + (long long)i3 * NE + e0;
  const C* ub = ua + n;
  // this rank's inputs, loaded into registers (both halves in flight together)
  using V = typename Lane<C>::V;
  constexpr int NVMAX = (NE / 3 + 2) / EPV;
  constexpr int PER = (NVMAX + NT - 1) / NT;
  const int nv = (e1 - e0) / EPV;
#if NFS_PASS1_FUSED_LOAD
  // one block of inputs at a time: load, CG update, assembly and staging, so
  // that only one block's inputs are live (no register spills at 96 x 96
  // with three CTAs per SM)
  const C a3 = lam[NX + NY + i3];
  using SG = Stage<NX, NY>;
  const int sb1 = SG::base(rank, 1), sb2 = SG::base(rank, 2);
  const int r1 = rank == 2 ? 0 : rank + 1, r2 = rank == 0 ? 2 : rank - 1;
  const R bt = cg_r != nullptr ? (R)*cg_beta : (R)0;
  const long long goff = (2 * grp) * n + (long long)i3 * NE + e0;
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int v = b * NT + (int)threadIdx.x;
    if (v < nv) {
      V ra = reinterpret_cast<const V*>(ua)[v];
      V rb = reinterpret_cast<const V*>(ub)[v];
      if (cg_r != nullptr) {
        // CG direction update fused into the load: u = r + beta u, stored back
        const V qa = ldg_c(reinterpret_cast<const V*>(cg_r + goff) + v);
        const V qb = ldg_c(reinterpret_cast<const V*>(cg_r + goff + n) + v);
        if constexpr (EPV == 2) {
          ra = make_float4(qa.x + bt * ra.x, qa.y + bt * ra.y, qa.z + bt * ra.z, qa.w + bt * ra.w);
          rb = make_float4(qb.x + bt * rb.x, qb.y + bt * rb.y, qb.z + bt * rb.z, qb.w + bt * rb.w);
        } else {
          ra = mk(qa.x + bt * ra.x, qa.y + bt * ra.y);
          rb = mk(qb.x + bt * rb.x, qb.y + bt * rb.y);
        }
        reinterpret_cast<V*>(const_cast<C*>(ua))[v] = ra;
        reinterpret_cast<V*>(const_cast<C*>(ub))[v] = rb;
      }
#pragma unroll
      for (int h = 0; h < EPV; ++h) {
        const int e = e0 + v * EPV + h;
        C va, vb;
        if constexpr (EPV == 2) {
          va = h == 0 ? mk(ra.x, ra.y) : mk(ra.z, ra.w);
          vb = h == 0 ? mk(rb.x, rb.y) : mk(rb.z, rb.w);
        } else {
          va = ra;
          vb = rb;
        }
        const int i1 = e % NX, i2 = e / NX;
        Basis<R> B;
        voxel_basis<R>(basis, n, (long long)i3 * NE + e, lam[i1], lam[NX + i2], a3, alpha, beta, B);
        C o[3];
        if (grp == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) o[k] = csub(cmul(B.x[k], vb), cmul(B.c[k], va));
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) o[k] = cadd(cmulc(B.x[k], va), cmulc(B.c[k], vb));
        }
        const int sidx = i2 * PITCH + i1;
        plane[sidx] = pick3<R>(rank, o[0], o[1], o[2]);
        plane[sb1 + (e - e0)] = pick3<R>(r1, o[0], o[1], o[2]);
        plane[sb2 + (e - e0)] = pick3<R>(r2, o[0], o[1], o[2]);
      }
    }
  }
#else
  V ra[PER], rb[PER];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int v = b * NT + (int)threadIdx.x;
    if (v < nv) {
      ra[b] = reinterpret_cast<const V*>(ua)[v];
      rb[b] = reinterpret_cast<const V*>(ub)[v];
    }
  }
  if (cg_r != nullptr) {
    // CG direction update fused into the load: u = r + beta u, stored back
    const R bt = (R)*cg_beta;
    const long long off = (2 * grp) * n + (long long)i3 * NE + e0;
    const V* rva = reinterpret_cast<const V*>(cg_r + off);
    const V* rvb = reinterpret_cast<const V*>(cg_r + off + n);
    V* wa = reinterpret_cast<V*>(const_cast<C*>(ua));
    V* wb = reinterpret_cast<V*>(const_cast<C*>(ub));
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int v = b * NT + (int)threadIdx.x;
      if (v < nv) {
        const V qa = ldg_c(rva + v), qb = ldg_c(rvb + v);
        if constexpr (EPV == 2) {
          ra[b] = make_float4(qa.x + bt * ra[b].x, qa.y + bt * ra[b].y, qa.z + bt * ra[b].z, qa.w + bt * ra[b].w);
          rb[b] = make_float4(qb.x + bt * rb[b].x, qb.y + bt * rb[b].y, qb.z + bt * rb[b].z, qb.w + bt * rb[b].w);
        } else {
          ra[b] = mk(qa.x + bt * ra[b].x, qa.y + bt * ra[b].y);
          rb[b] = mk(qb.x + bt * rb[b].x, qb.y + bt * rb[b].y);
        }
        wa[v] = ra[b];
        wb[v] = rb[b];
      }
    }
  }
  const C a3 = lam[NX + NY + i3];
  // exchange through shared memory: all three components of this third are
  // computed here; this rank's goes to its final place, the other two to
  // staging runs that the partner CTAs load after the cluster barrier
  using SG = Stage<NX, NY>;
  const int sb1 = SG::base(rank, 1), sb2 = SG::base(rank, 2);
  const int r1 = rank == 2 ? 0 : rank + 1, r2 = rank == 0 ? 2 : rank - 1;
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int v = b * NT + (int)threadIdx.x;
    if (v < nv) {
#pragma unroll
      for (int h = 0; h < EPV; ++h) {
        const int e = e0 + v * EPV + h;
        C va, vb;
        if constexpr (EPV == 2) {
          va = h == 0 ? mk(ra[b].x, ra[b].y) : mk(ra[b].z, ra[b].w);
          vb = h == 0 ? mk(rb[b].x, rb[b].y) : mk(rb[b].z, rb[b].w);
        } else {
          va = ra[b];
          vb = rb[b];
        }
        const int i1 = e % NX, i2 = e / NX;
        Basis<R> B;
        voxel_basis<R>(basis, n, (long long)i3 * NE + e, lam[i1], lam[NX + i2], a3, alpha, beta, B);
        C o[3];
        if (grp == 0) {
          // p^ = -c u1a + x u1b
#pragma unroll
          for (int k = 0; k < 3; ++k) o[k] = csub(cmul(B.x[k], vb), cmul(B.c[k], va));
        } else {
          // q^ = conj(x) u2a + conj(c) u2b
#pragma unroll
          for (int k = 0; k < 3; ++k) o[k] = cadd(cmulc(B.x[k], va), cmulc(B.c[k], vb));
        }
        const int sidx = i2 * PITCH + i1;
        plane[sidx] = pick3<R>(rank, o[0], o[1], o[2]);
        plane[sb1 + (e - e0)] = pick3<R>(r1, o[0], o[1], o[2]);
        plane[sb2 + (e - e0)] = pick3<R>(r2, o[0], o[1], o[2]);
      }
    }
  }
#endif
  cl.sync();  // staging complete in every CTA of the cluster
  {
    // load this rank's component of the two other thirds from the partners'
    // staging runs, then (after every CTA has read) put them in place
    using V = typename Lane<C>::V;
    constexpr int S_MAX = (NE / 3 + 2) / EPV;
    constexpr int PER2 = (S_MAX + NT - 1) / NT;
    V g[2][PER2];
    int gt[2], gn[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int t = q == 0 ? r1 : r2;               // partner rank (its third)
      const int k = q == 0 ? 2 : 1;                 // this rank = t + k (mod 3)
      const V* src = reinterpret_cast<const V*>(cl.map_shared_rank(plane, t) + SG::base(t, k));
      gt[q] = t;
      gn[q] = (SG::e0(t + 1) - SG::e0(t)) / EPV;
#pragma unroll
      for (int b = 0; b < PER2; ++b) {
        const int v = b * NT + (int)threadIdx.x;
        if (v < gn[q]) g[q][b] = src[v];
      }
    }
    cl.sync();  // every CTA has read its partners' staging
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int te0 = SG::e0(gt[q]);
#pragma unroll
      for (int b = 0; b < PER2; ++b) {
        const int v = b * NT + (int)threadIdx.x;
        if (v < gn[q]) {
#pragma unroll
          for (int h = 0; h < EPV; ++h) {
            const int e = te0 + v * EPV + h;
            C val;
            if constexpr (EPV == 2) {
              val = h == 0 ? mk(g[q][b].x, g[q][b].y) : mk(g[q][b].z, g[q][b].w);
            } else {
              val = g[q][b];
            }
            plane[(e / NX) * PITCH + (e % NX)] = val;
          }
        }
      }
    }
    __syncthreads();
  }
  smem_fft<true, NX, NY, NT, PITCH, 1>(plane, stx);  // along x (rows)
  // along y (columns), the results leaving for global memory from registers
  C* out = fld + ((long long)(grp * 3 + rank) * n3 + i3) * NE;
  smem_fft_io<true, NY, NX, NT, 1, PITCH, false, true>(plane, sty, NoGet{},
                                                      [&](int i1, int i2, C v) { out[i2 * NX + i1] = v; });
}

// ---------------------------------------------------------------------------
// pass 2: the material product of eq. factor_mtx, per real-space voxel:
//   w = Phi^{-1} (xi mu^{-1} p + q),   f = mu^{-1} (zeta w + p)
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ void material_apply(const MatView<R>& m, long long v, const cplx<R>* p,
                                               const cplx<R>* q, cplx<R>* f, cplx<R>* w, R scale) {
  using C = cplx<R>;
  R ip[3], im[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ip[c] = m.inv_phi[c * m.n + v];
    im[c] = m.inv_mu ? m.inv_mu[c * m.n + v] : (R)1;
  }
  if (m.kind == kMediumChiral) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R g = m.gam[c * m.n + v];
      // xi mu^{-1} p = i g im p;  w = ip (q + i g im p)
      const R gi = g * im[c];
      const C s = mk(q[c].x - gi * p[c].y, q[c].y + gi * p[c].x);
      const C wc = cscale(s, ip[c]);
      // zeta w = -i g w;  f = im (p - i g w)
      const C fc = mk(p[c].x + g * wc.y, p[c].y - g * wc.x);
      w[c] = cscale(wc, scale);
      f[c] = cscale(fc, im[c] * scale);
    }
  } else {
    const R g = m.gam[v];
    const int a = m.ax_a, b = m.ax_b;
    // partner component of each axis in the coupled pair (-1: uncoupled)
    C wc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int o = c == a ? b : (c == b ? a : -1);
      C xmp = mk((R)0, (R)0);
      if (o >= 0) {
        // (xi mu^{-1} p)_c = i g im_o p_o
        const C po = pick3<R>(o, p[0], p[1], p[2]);
        const R imo = o == 0 ? im[0] : (o == 1 ? im[1] : im[2]);
        xmp = cmul_i(cscale(po, g * imo));
      }
      wc[c] = cscale(cadd(q[c], xmp), ip[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int o = c == a ? b : (c == b ? a : -1);
      C zw = mk((R)0, (R)0);
      if (o >= 0) zw = cmul_mi(cscale(pick3<R>(o, wc[0], wc[1], wc[2]), g));  // (zeta w)_c = -i g w_o
      w[c] = cscale(wc[c], scale);
      f[c] = cscale(cadd(p[c], zw), im[c] * scale);
    }
  }
}

template <typename R, int N3, int TX, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_pass2_z_material(cplx<R>* __restrict__ fld, MatView<R> mat, const cplx<R>* __restrict__ twz, int ncols,
                   R inv_n, const int* __restrict__ skip, double* __restrict__ dot_part, BatchStrides bs) {
  using C = cplx<R>;
  constexpr int LINES = 6 * TX;
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* stw = buf + N3 * PITCH;
  const int tiles = ncols / TX;
  const int prob = blockIdx.x / tiles;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  fld += prob * bs.sfld;
  mat.inv_phi += prob * bs.smat;
  mat.gam += prob * bs.smat;
  if (mat.inv_mu) mat.inv_mu += prob * bs.smat;
  for (int i = threadIdx.x; i < N3; i += NT) stw[i] = twz[i];
  const int col0 = (blockIdx.x % tiles) * TX;
  const long long n = (long long)ncols * N3;
  // line l = f * TX + c of the tile is field f, column col0 + c; its element
  // z lives at fld[f n + z ncols + col0 + c] (consecutive lines, consecutive
  // addresses within a field)
  C* tile = fld + col0;
  auto gaddr = [&](int l, int z) { return tile + (long long)(l / TX) * n + (long long)z * ncols + (l % TX); };
  __syncthreads();  // twiddles
  smem_fft_io<true, N3, LINES, NT, 1, PITCH, true, false>(buf, stw, [&](int l, int z) { return ldg_c(gaddr(l, z)); },
                                                         NoPut{});
  // CG curvature from the real-space fields (Parseval; the DFTs carry the
  // factor n that inv_n removes): u^* A_r u = sum Re(conj(P) f + conj(Q) w)
  RedAccFor<R> dot_acc;
  for (int idx = threadIdx.x; idx < N3 * TX; idx += NT) {
    const int c = idx % TX, z = idx / TX;
    C* row = buf + z * PITCH + c;
    C p[3] = {row[0], row[TX], row[2 * TX]};
    C q[3] = {row[3 * TX], row[4 * TX], row[5 * TX]};
    C fo[3], wo[3];
    material_apply<R>(mat, (long long)z * ncols + col0 + c, p, q, fo, wo, inv_n);
    if (dot_part != nullptr) {
      R sacc = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        sacc += p[k].x * fo[k].x + p[k].y * fo[k].y + q[k].x * wo[k].x + q[k].y * wo[k].y;
      dot_acc.add(static_cast<typename RedAccFor<R>::value_type>(sacc));
    }
    row[0] = fo[0];
    row[TX] = fo[1];
    row[2 * TX] = fo[2];
    row[3 * TX] = wo[0];
    row[4 * TX] = wo[1];
    row[5 * TX] = wo[2];
  }
  if (dot_part != nullptr) {
    const double tot = dot_acc.template block_total<NT>();  // (its barriers also order the material writes)
    if (threadIdx.x == 0) dot_part[(long long)prob * bs.sstate + blockIdx.x % tiles] = tot;
  } else {
    __syncthreads();
  }
  smem_fft_io<false, N3, LINES, NT, 1, PITCH, false, true>(buf, stw, NoGet{},
                                                          [&](int l, int z, C v) { *gaddr(l, z) = v; });
}

// ---------------------------------------------------------------------------
// pass 3
// ---------------------------------------------------------------------------
template <typename R, int NX, int NY, int NT, int MINB>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(NT, MINB)
k_pass3_fft_xy_project(const cplx<R>* __restrict__ fld, cplx<R>* __restrict__ Au,
                       const cplx<R>* __restrict__ lam, const cplx<R>* __restrict__ twx,
                       const cplx<R>* __restrict__ twy, int n3, R alpha, R beta,
                       const int* __restrict__ skip, const cplx<R>* __restrict__ basis, BatchStrides bs,
                       CgFuse<R> cg) {
  using C = cplx<R>;
  constexpr int PITCH = NX + 1;
  constexpr int NE = NX * NY;
  constexpr int EPV = Lane<C>::EPV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* plane = reinterpret_cast<C*>(smem_raw);
  C* stx = plane + NY * PITCH;
  C* sty = stx + NX;
  cg::cluster_group cl = cg::this_cluster();
  const int prob = blockIdx.z / n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  const int rank = (int)cl.block_rank();
  const int grp = blockIdx.y;
  const int i3 = blockIdx.z % n3;
  fld += prob * bs.sfld;
  Au += prob * bs.su;
  lam += (long long)prob * bs.slam;
  if (basis != nullptr) basis += prob * bs.sbasis;
  for (int i = threadIdx.x; i < NX; i += NT) stx[i] = twx[i];
  for (int i = threadIdx.x; i < NY; i += NT) sty[i] = twy[i];
  const C* in = fld + ((long long)(grp * 3 + rank) * n3 + i3) * NE;
  // fused CG step: alpha from pass 2's partials of p^* A p, summed in the same
  // fixed order by every CTA (so all agree); no state is written until the
  // last CTA of the launch (the `done` flag every CTA reads at its start must
  // not change while the launch runs)
  __shared__ double s_cg_alpha;
  __shared__ int s_cg_ok, s_cg_last;
  // (only complex64 and complex128 run CG; the double-single product never does)
  constexpr bool CGT = std::is_same<R, float>::value || std::is_same<R, double>::value;
  CGState* cst = (CGT && cg.st != nullptr) ? cg.st + prob : nullptr;
  if (cst != nullptr) {
    RedAccFor<R> pa;
    for (int i = threadIdx.x; i < cst->npart_a; i += NT) pa.add_double(cst->part_a[i]);
    const double pAp = pa.template block_total<NT>();
    if (threadIdx.x == 0) {
      s_cg_alpha = cst->rr / pAp;
      s_cg_ok = (pAp > 0.0) && (s_cg_alpha == s_cg_alpha);  // also catches NaN
      if (blockIdx.x == 0 && blockIdx.y == 0 && i3 == 0) {
        cst->pAp = pAp;
        cst->alpha = s_cg_alpha;
      }
    }
  }
  __syncthreads();  // twiddles (and alpha)
  // the 2-D DFT along y first (columns, read from global memory straight into
  // registers), then along x
  smem_fft_io<false, NY, NX, NT, 1, PITCH, true, false>(plane, sty,
                                                       [&](int i1, int i2) { return ldg_c(in + i2 * NX + i1); }, NoPut{});
  smem_fft<false, NX, NY, NT, PITCH, 1>(plane, stx);
  cl.sync();
  const C* src0 = cl.map_shared_rank(plane, 0);
  const C* src1 = cl.map_shared_rank(plane, 1);
  const C* src2 = cl.map_shared_rank(plane, 2);
  const long long n = (long long)NE * n3;
  C* o0 = Au + (2 * grp) * n + (long long)i3 * NE;
  C* o1 = o0 + n;
  const C a3 = lam[NX + NY + i3];
  const int e0 = third_bound<NE>(rank), e1 = third_bound<NE>(rank + 1);
  using V = typename Lane<C>::V;
  V* o0v = reinterpret_cast<V*>(o0);
  V* o1v = reinterpret_cast<V*>(o1);
  const bool cg_on = cst != nullptr;
  const bool cg_upd = cg_on && s_cg_ok;
  const R cg_al = cg_on ? (R)s_cg_alpha : (R)0;
  const long long cg_off = prob * bs.su + (2 * grp) * n + (long long)i3 * NE;
  RedAccFor<R> cg_acc;
  // EPV consecutive elements per lane (e0, e1 even)
  for (int ev = e0 / EPV + (int)threadIdx.x; ev < e1 / EPV; ev += NT) {
    C r0[EPV], r1[EPV];
#pragma unroll
    for (int h = 0; h < EPV; ++h) {
      const int e = ev * EPV + h;
      const int i1 = e % NX, i2 = e / NX;
      const int s = i2 * PITCH + i1;
      const C f[3] = {src0[s], src1[s], src2[s]};
      Basis<R> B;
      voxel_basis<R>(basis, n, (long long)i3 * NE + e, lam[i1], lam[NX + i2], a3, alpha, beta, B);
      if (grp == 0) {
        // P_r^* f = [-sum conj(c) f ; sum conj(x) f]
        r0[h] = cneg(cadd(cadd(cmulc(B.c[0], f[0]), cmulc(B.c[1], f[1])), cmulc(B.c[2], f[2])));
        r1[h] = cadd(cadd(cmulc(B.x[0], f[0]), cmulc(B.x[1], f[1])), cmulc(B.x[2], f[2]));
      } else {
        // Q_r^* w = [sum x w ; sum c w]
        r0[h] = cadd(cadd(cmul(B.x[0], f[0]), cmul(B.x[1], f[1])), cmul(B.x[2], f[2]));
        r1[h] = cadd(cadd(cmul(B.c[0], f[0]), cmul(B.c[1], f[1])), cmul(B.c[2], f[2]));
      }
    }
    if (cg_on) {
      // x += alpha p, r -= alpha A_r p (this CTA's third of its two quarters)
      if constexpr (CGT) if (cg_upd) {
#pragma unroll
        for (int h = 0; h < EPV; ++h) {
          const long long i0 = cg_off + ev * EPV + h, i1 = i0 + n;
          const C pa = cg.p[i0], pb = cg.p[i1];
          C xa = cg.x[i0], xb = cg.x[i1], ra = cg.r[i0], rb = cg.r[i1];
          xa = mk(xa.x + cg_al * pa.x, xa.y + cg_al * pa.y);
          xb = mk(xb.x + cg_al * pb.x, xb.y + cg_al * pb.y);
          ra = mk(ra.x - cg_al * r0[h].x, ra.y - cg_al * r0[h].y);
          rb = mk(rb.x - cg_al * r1[h].x, rb.y - cg_al * r1[h].y);
          cg.x[i0] = xa;
          cg.x[i1] = xb;
          cg.r[i0] = ra;
          cg.r[i1] = rb;
          cg_acc.add(static_cast<typename RedAccFor<R>::value_type>(ra.x * ra.x + ra.y * ra.y + rb.x * rb.x +
                                                                   rb.y * rb.y));
        }
      }
    } else if constexpr (EPV == 2) {
      o0v[ev] = make_float4(r0[0].x, r0[0].y, r0[1].x, r0[1].y);
      o1v[ev] = make_float4(r1[0].x, r1[0].y, r1[1].x, r1[1].y);
    } else {
      o0v[ev] = r0[0];
      o1v[ev] = r1[0];
    }
  }
  if (cg_on) {
    // this CTA's partial of the new r^* r; the last CTA to arrive (atomic
    // count, no waiting) sums them in fixed order and sets beta, the
    // iteration count and the convergence state for the next launch
    const int ncta = 6 * n3;
    const int cta = rank + 3 * (grp + 2 * i3);
    const double part = cg_acc.template block_total<NT>();
    if (threadIdx.x == 0) {
      cst->part_b[cta] = part;
      __threadfence();
      s_cg_last = atomicAdd(&cst->arrived, 1u) == (unsigned)ncta - 1;
    }
    __syncthreads();
    if (s_cg_last) {
      __threadfence();
      RedAccFor<R> rb_acc;
      for (int i = threadIdx.x; i < ncta; i += NT) rb_acc.add_double(((volatile double*)cst->part_b)[i]);
      const double rr = rb_acc.template block_total<NT>();
      if (threadIdx.x == 0) {
        cst->arrived = 0;
        if (!s_cg_ok) {
          cst->status = -7;  // breakdown: x, r left untouched
          cst->done = 1;
        } else {
          cst->it += 1;
          if (!(rr == rr)) {
            cst->status = -7;
            cst->done = 1;
          } else if (rr <= cst->tol2) {
            cst->done = 1;
          } else if (cst->it >= cst->maxit) {
            cst->status = -6;
            cst->done = 1;
          }
          cst->beta = rr / cst->rr;
          cst->rr = rr;
        }
      }
    }
  }
  cl.sync();  // keep this CTA's plane alive until the cluster finished reading it
}

}  // namespace nfs
