// The A_r product for xy planes too large for shared memory (complex128 at
// 128 x 128: 264 KB), in five passes instead of three.  The arithmetic is the
// same as in matvec_kernels.cuh (eq. factor_mtx; the Bloch twist cancels, the
// two unnormalised DFTs give the factor n removed in pass 2); the planes are
// split into tiles of rows or columns, with an extra trip through global
// memory between the x and y DFTs:
//
//   pass 1a  (tile of RT rows, group):  spectral assembly of all three
//            components (no cluster exchange needed: a CTA owns every
//            component of its rows), inverse DFT along x.
//   pass 1b  (tile of CT columns, field):  inverse DFT along y.
//   pass 2   unchanged (k_pass2_z_material).
//   pass 3a  (tile of CT columns, field):  forward DFT along y.
//   pass 3b  (tile of RT rows, group):  forward DFT along x, projections.
//
// CG fusion as in the three-pass product: pass 1a forms p = r + beta p while
// loading u, pass 3b emits the p^* A p partials (one per CTA).
#pragma once
#include "matvec_kernels.cuh"

namespace nfs {

template <typename R, int NX, int RT, int NT>
__global__ void __launch_bounds__(NT, 1)
k_pass1a_assemble_fft_x(const cplx<R>* u, cplx<R>* __restrict__ fld, const cplx<R>* __restrict__ lam,
                        const cplx<R>* __restrict__ twx, int n2, int n3, R alpha, R beta,
                        const int* __restrict__ skip, const cplx<R>* __restrict__ cg_r,
                        const double* __restrict__ cg_beta, const cplx<R>* __restrict__ basis, BatchStrides bs) {
  using C = cplx<R>;
  constexpr int PITCH = NX + 1;
  constexpr int LINES = 3 * RT;  // line (c, r): component c of row row0 + r
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  C* stx = tile + LINES * PITCH;
  const int prob = blockIdx.z / n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  const int i3 = blockIdx.z % n3;
  const int grp = blockIdx.y;
  const int row0 = blockIdx.x * RT;
  u += prob * bs.su;
  fld += prob * bs.sfld;
  lam += (long long)prob * bs.slam;
  if (basis != nullptr) basis += prob * bs.sbasis;
  const R bt = cg_r != nullptr ? (R)cg_beta[(long long)prob * bs.sstate] : (R)0;
  if (cg_r != nullptr) cg_r += prob * bs.su;
  for (int i = threadIdx.x; i < NX; i += NT) stx[i] = twx[i];
  const long long n = (long long)NX * n2 * n3;
  const long long NE = (long long)NX * n2;
  const C a3 = lam[NX + n2 + i3];
  for (int idx = threadIdx.x; idx < RT * NX; idx += NT) {
    const int r = idx / NX, i1 = idx % NX;
    const int i2 = row0 + r;
    const long long e = (long long)i2 * NX + i1;
    const long long off = (2 * grp) * n + (long long)i3 * NE + e;
    C va = u[off], vb = u[off + n];
    if (cg_r != nullptr) {
      // CG direction update fused into the load: u = r + beta u, stored back
      const C ga = cg_r[off], gb = cg_r[off + n];
      va = mk(ga.x + bt * va.x, ga.y + bt * va.y);
      vb = mk(gb.x + bt * vb.x, gb.y + bt * vb.y);
      const_cast<C*>(u)[off] = va;
      const_cast<C*>(u)[off + n] = vb;
    }
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
#pragma unroll
    for (int k = 0; k < 3; ++k) tile[(k * RT + r) * PITCH + i1] = o[k];
  }
  __syncthreads();
  smem_fft<true, NX, LINES, NT, PITCH, 1>(tile, stx);  // along x
  for (int idx = threadIdx.x; idx < LINES * NX; idx += NT) {
    const int l = idx / NX, i1 = idx % NX;
    const int k = l / RT, r = l % RT;
    fld[((long long)(grp * 3 + k) * n3 + i3) * NE + (long long)(row0 + r) * NX + i1] = tile[l * PITCH + i1];
  }
}

// DFT along y of a tile of CT columns of one field plane, in place in global
// memory (pass 1b: inverse; pass 3a: forward).
template <bool INV, typename R, int NY, int CT, int NT>
__global__ void __launch_bounds__(NT)
k_fft_y_columns(cplx<R>* __restrict__ fld, const cplx<R>* __restrict__ twy, int n1, int n3,
                const int* __restrict__ skip, BatchStrides bs) {
  using C = cplx<R>;
  constexpr int PITCH = CT + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  C* sty = tile + NY * PITCH;
  const int prob = blockIdx.z / n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  const int i3 = blockIdx.z % n3;
  const int f = blockIdx.y;
  const int col0 = blockIdx.x * CT;
  fld += prob * bs.sfld;
  for (int i = threadIdx.x; i < NY; i += NT) sty[i] = twy[i];
  C* plane = fld + ((long long)f * n3 + i3) * (long long)n1 * NY + col0;
  __syncthreads();  // twiddles
  // line l = column col0 + l; element i2 at plane[i2 n1 + l] (consecutive
  // lines, consecutive addresses)
  smem_fft_io<INV, NY, CT, NT, 1, PITCH, true, true>(
      tile, sty, [&](int l, int i2) { return plane[(long long)i2 * n1 + l]; },
      [&](int l, int i2, C v) { plane[(long long)i2 * n1 + l] = v; });
}

template <typename R, int NX, int RT, int NT>
__global__ void __launch_bounds__(NT, 1)
k_pass3b_fft_x_project(const cplx<R>* __restrict__ fld, cplx<R>* __restrict__ Au, const cplx<R>* __restrict__ lam,
                       const cplx<R>* __restrict__ twx, int n2, int n3, R alpha, R beta,
                       const int* __restrict__ skip, const cplx<R>* __restrict__ u, double* __restrict__ dot_part,
                       const cplx<R>* __restrict__ basis, BatchStrides bs) {
  using C = cplx<R>;
  constexpr int PITCH = NX + 1;
  constexpr int LINES = 3 * RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  C* stx = tile + LINES * PITCH;
  const int prob = blockIdx.z / n3;
  if (skip != nullptr && skip[(long long)prob * bs.sskip]) return;
  const int i3 = blockIdx.z % n3;
  const int grp = blockIdx.y;
  const int row0 = blockIdx.x * RT;
  fld += prob * bs.sfld;
  Au += prob * bs.su;
  lam += (long long)prob * bs.slam;
  if (basis != nullptr) basis += prob * bs.sbasis;
  if (dot_part != nullptr) {
    u += prob * bs.su;
    dot_part += prob * bs.sstate;
  }
  for (int i = threadIdx.x; i < NX; i += NT) stx[i] = twx[i];
  const long long n = (long long)NX * n2 * n3;
  const long long NE = (long long)NX * n2;
  for (int idx = threadIdx.x; idx < LINES * NX; idx += NT) {
    const int l = idx / NX, i1 = idx % NX;
    const int k = l / RT, r = l % RT;
    tile[l * PITCH + i1] = ldg_c(fld + ((long long)(grp * 3 + k) * n3 + i3) * NE + (long long)(row0 + r) * NX + i1);
  }
  __syncthreads();
  smem_fft<false, NX, LINES, NT, PITCH, 1>(tile, stx);  // along x
  const C a3 = lam[NX + n2 + i3];
  double dot_acc = 0.0;
  for (int idx = threadIdx.x; idx < RT * NX; idx += NT) {
    const int r = idx / NX, i1 = idx % NX;
    const int i2 = row0 + r;
    const long long e = (long long)i2 * NX + i1;
    const C f[3] = {tile[(0 * RT + r) * PITCH + i1], tile[(1 * RT + r) * PITCH + i1], tile[(2 * RT + r) * PITCH + i1]};
    Basis<R> B;
    voxel_basis<R>(basis, n, (long long)i3 * NE + e, lam[i1], lam[NX + i2], a3, alpha, beta, B);
    C r0, r1;
    if (grp == 0) {
      r0 = cneg(cadd(cadd(cmulc(B.c[0], f[0]), cmulc(B.c[1], f[1])), cmulc(B.c[2], f[2])));
      r1 = cadd(cadd(cmulc(B.x[0], f[0]), cmulc(B.x[1], f[1])), cmulc(B.x[2], f[2]));
    } else {
      r0 = cadd(cadd(cmul(B.x[0], f[0]), cmul(B.x[1], f[1])), cmul(B.x[2], f[2]));
      r1 = cadd(cadd(cmul(B.c[0], f[0]), cmul(B.c[1], f[1])), cmul(B.c[2], f[2]));
    }
    const long long off = (2 * grp) * n + (long long)i3 * NE + e;
    Au[off] = r0;
    Au[off + n] = r1;
    if (dot_part != nullptr) {
      const C pa = u[off], pb = u[off + n];
      dot_acc += (double)(pa.x * r0.x + pa.y * r0.y + pb.x * r1.x + pb.y * r1.y);
    }
  }
  if (dot_part != nullptr) {
    const double tot = block_sum_dbl<NT>(dot_acc);
    if (threadIdx.x == 0) dot_part[((long long)i3 * 2 + grp) * gridDim.x + blockIdx.x] = tot;
  }
}

}  // namespace nfs
