// complex128 instantiation of the three-pass A_r product; the eigenvalue
// gradient and eigenvector-field passes that share its pass-1 fields; the
// residual of the original GEP.
#include <algorithm>
#include <cmath>
#include "matvec_impl.cuh"

namespace nfs {
NFS_INSTANTIATE_MATVEC(double)

// Gradient of omega with respect to the per-component permittivity and the
// chirality, for one eigenvector y of B_r y = theta A_r y (mu = 1):
//   d omega = y^* (dA_r) y / (y^* B_r y),
//   y^* A_r y = sum_c |s_c|^2 / Phi_c + |p_c|^2,  s = xi p + q,
// with (p, q) = (P_r y1, Q_r y2) in real space (eq. factor_mtx with mu = 1,
// zeta = xi^*).  Hence, per voxel and component,
//   d/d eps_c   : -|s_c|^2 / Phi_c^2
//   d/d gamma_c : 2 Re(conj(s_c) i p_c) / Phi_c + 2 gamma_c |s_c|^2 / Phi_c^2   (chiral)
// and for the pseudochiral pair (a, b) with one gamma per voxel the two
// coupled components' terms add (s_a = i gamma p_b + q_a, s_b = i gamma p_a + q_b).
// `scale` carries weight / (n y^* B_r y): pass 1 leaves sqrt(n) p, sqrt(n) q.
template <int N3, int TX, int NT>
__global__ void __launch_bounds__(NT)
k_grad_z(const double2* __restrict__ fld, const double2* __restrict__ twz, int ncols, const double* __restrict__ inv_phi,
         const double* __restrict__ gam, int kind, int ax_a, int ax_b, double scale, double* __restrict__ d_eps,
         double* __restrict__ d_gamma) {
  using C = double2;
  constexpr int LINES = 6 * TX;
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* stw = buf + N3 * PITCH;
  for (int i = threadIdx.x; i < N3; i += NT) stw[i] = twz[i];
  const int col0 = blockIdx.x * TX;
  const long long n = (long long)ncols * N3;
  for (int idx = threadIdx.x; idx < N3 * LINES; idx += NT) {
    const int c = idx % TX;
    const int t = idx / TX;
    const int f = t % 6, z = t / 6;
    buf[z * PITCH + f * TX + c] = fld[f * n + (long long)z * ncols + col0 + c];
  }
  __syncthreads();
  smem_fft<true, N3, LINES, NT, 1, PITCH>(buf, stw);
  for (int idx = threadIdx.x; idx < N3 * TX; idx += NT) {
    const int c = idx % TX, z = idx / TX;
    const long long v = (long long)z * ncols + col0 + c;
    const C* row = buf + z * PITCH + c;
    const C p[3] = {row[0], row[TX], row[2 * TX]};
    const C q[3] = {row[3 * TX], row[4 * TX], row[5 * TX]};
    double ip[3];
    for (int k = 0; k < 3; ++k) ip[k] = inv_phi[k * n + v];
    if (kind == kMediumChiral) {
      for (int k = 0; k < 3; ++k) {
        const double g = gam[k * n + v];
        const C s = mk(q[k].x - g * p[k].y, q[k].y + g * p[k].x);   // q + i g p
        const double s2 = cabs2(s);
        const C ipk = cmul_i(p[k]);
        const double re = s.x * ipk.x + s.y * ipk.y;                  // Re(conj(s) i p)
        if (d_eps) d_eps[k * n + v] += scale * (-s2 * ip[k] * ip[k]);
        if (d_gamma) d_gamma[k * n + v] += scale * (2.0 * re * ip[k] + 2.0 * g * s2 * ip[k] * ip[k]);
      }
    } else {
      const double g = gam[v];
      C s[3] = {q[0], q[1], q[2]};
      s[ax_a] = cadd(q[ax_a], cmul_i(cscale(p[ax_b], g)));
      s[ax_b] = cadd(q[ax_b], cmul_i(cscale(p[ax_a], g)));
      double dg = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double s2 = cabs2(s[k]);
        if (d_eps) d_eps[k * n + v] += scale * (-s2 * ip[k] * ip[k]);
        if (k == ax_a || k == ax_b) {
          const C ipo = cmul_i(p[k == ax_a ? ax_b : ax_a]);
          const double re = s[k].x * ipo.x + s[k].y * ipo.y;
          dg += 2.0 * re * ip[k] + 2.0 * g * s2 * ip[k] * ip[k];
        }
      }
      if (d_gamma) d_gamma[v] += scale * dg;
    }
  }
}

template <int N3>
static cudaError_t grad_prep_n3() {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  return cudaFuncSetAttribute(k_grad_z<N3, TX, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)z_smem<double, N3>());
}

template <int N3>
static cudaError_t grad_launch_n3(const GradArgs& a) {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  const int ncols = a.n1 * a.n2;
  k_grad_z<N3, TX, NT><<<ncols / TX, NT, z_smem<double, N3>(), a.stream>>>(
      a.fld, a.tw3, ncols, a.inv_phi, a.gam, a.kind, a.ax_a, a.ax_b, a.scale, a.d_eps, a.d_gamma);
  return cudaGetLastError();
}

cudaError_t grad_prepare(int n1, int n2, int n3) {
  if (!matvec_supported<double>(n1, n2, n3)) return cudaErrorInvalidValue;
  switch (n3) {
#define NFS_CASE(N) case N: return grad_prep_n3<N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t grad_launch(const GradArgs& a) {
  switch (a.n3) {
#define NFS_CASE(N) case N: return grad_launch_n3<N>(a);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

// Physical fields of one eigenvector (Algorithm 1, final step):
//   x = [E; H] = B^{-1} diag(P_r, Q_r) y,   B = i [[zeta, mu], [-eps, -xi]].
// By eq. B_inv, B^{-1} [p; q] = [i w; -i f] with the same
//   w = Phi^{-1} (xi mu^{-1} p + q),   f = mu^{-1} (zeta w + p)
// that the middle factors of A_r form (material_apply), so this is pass 1,
// the inverse DFT along z and the material step of the product.  The product
// never needs the Bloch twist D of T = n^{-1/2} D U (eq. mtx_T: it cancels
// against T^*); the fields do, so it is applied here from the three 1-D
// diagonals D_l[j] = exp(i 2 pi k.a_l j / n_l).  The two unnormalised DFTs
// leave sqrt(n) p, sqrt(n) q; inv_sqrt_n removes that factor.
template <int N3, int TX, int NT>
__global__ void __launch_bounds__(NT)
k_fields_z(const double2* __restrict__ fld, const double2* __restrict__ twz, int n1, int ncols, MatView<double> mat,
           const double2* __restrict__ bloch, double inv_sqrt_n, double2* __restrict__ X) {
  using C = double2;
  constexpr int LINES = 6 * TX;
  constexpr int PITCH = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* stw = buf + N3 * PITCH;
  for (int i = threadIdx.x; i < N3; i += NT) stw[i] = twz[i];
  const int col0 = blockIdx.x * TX;
  const long long n = (long long)ncols * N3;
  for (int idx = threadIdx.x; idx < N3 * LINES; idx += NT) {
    const int c = idx % TX;
    const int t = idx / TX;
    const int f = t % 6, z = t / 6;
    buf[z * PITCH + f * TX + c] = fld[f * n + (long long)z * ncols + col0 + c];
  }
  __syncthreads();
  smem_fft<true, N3, LINES, NT, 1, PITCH>(buf, stw);
  const int n2 = ncols / n1;
  for (int idx = threadIdx.x; idx < N3 * TX; idx += NT) {
    const int c = idx % TX, z = idx / TX;
    const int col = col0 + c;
    const long long v = (long long)z * ncols + col;
    const C* row = buf + z * PITCH + c;
    const C p[3] = {row[0], row[TX], row[2 * TX]};
    const C q[3] = {row[3 * TX], row[4 * TX], row[5 * TX]};
    C f[3], w[3];
    material_apply<double>(mat, v, p, q, f, w, inv_sqrt_n);
    const C d = cmul(cmul(bloch[col % n1], bloch[n1 + col / n1]), bloch[n1 + n2 + z]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      X[k * n + v] = cmul_i(cmul(d, w[k]));         // E = i D w
      X[(3 + k) * n + v] = cmul_mi(cmul(d, f[k]));  // H = -i D f
    }
  }
}

template <int N3>
static cudaError_t fields_prep_n3() {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  return cudaFuncSetAttribute(k_fields_z<N3, TX, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)z_smem<double, N3>());
}

template <int N3>
static cudaError_t fields_launch_n3(const FieldsArgs& a) {
  constexpr int TX = z_tile(N3, 16);
  constexpr int NT = z_threads(N3, 16);
  const int ncols = a.n1 * a.n2;
  const MatView<double> mat{a.inv_phi, a.gam, a.inv_mu, a.kind, a.ax_a, a.ax_b, (long long)ncols * N3};
  k_fields_z<N3, TX, NT><<<ncols / TX, NT, z_smem<double, N3>(), a.stream>>>(
      a.fld, a.tw3, a.n1, ncols, mat, a.bloch, 1.0 / std::sqrt((double)ncols * N3), a.X);
  return cudaGetLastError();
}

cudaError_t fields_prepare(int n1, int n2, int n3) {
  if (!matvec_supported<double>(n1, n2, n3)) return cudaErrorInvalidValue;
  switch (n3) {
#define NFS_CASE(N) case N: return fields_prep_n3<N>();
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t fields_launch(const FieldsArgs& a) {
  switch (a.n3) {
#define NFS_CASE(N) case N: return fields_launch_n3<N>(a);
    NFS_FOR_EACH_SIZE(NFS_CASE)
#undef NFS_CASE
  }
  return cudaErrorInvalidValue;
}

// Residual of an eigenpair (omega, x = [E; H]) in the GEP of eq.
// discrete_GEP_EH, diag(C, C^*) x = omega B x, with the Yee curl applied as
// its stencil (eqs. mtx_C, mtx_C123, mtx_K_n1): C_l is the forward difference
// along axis l over delta_l, the step past the last cell wrapping to the first
// times exp(i 2 pi k.a_l); C_l^* is the backward difference, wrapping with the
// conjugate phase.  Per voxel
//   B x = i [zeta E + mu H ; -eps E - xi H],
// with eps recovered from the stored 1 / Phi: chiral eps_c = Phi_c + gamma_c^2
// / mu_c, pseudochiral eps_a = Phi_a + gamma^2 / mu_b (and a <-> b).  Each
// block leaves two partial sums, |diag(C, C^*) x - omega B x|^2 and |B x|^2.
__global__ void __launch_bounds__(256) k_gep_residual(GepResidualArgs a) {
  using C = double2;
  const long long n1 = a.n1, n2 = a.n2, n3 = a.n3;
  const long long s3 = n1 * n2, n = s3 * n3;
  const C* X = a.X;
  double racc = 0.0, bacc = 0.0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long i1 = v % n1, i2 = (v / n1) % n2, i3 = v / s3;
    // neighbours: forward (E) and backward (H) along each axis
    const bool fw[3] = {i1 == n1 - 1, i2 == n2 - 1, i3 == n3 - 1};
    const bool bw[3] = {i1 == 0, i2 == 0, i3 == 0};
    const long long step[3] = {1, n1, s3};
    const long long len[3] = {n1, n2, n3};
    C E[3], H[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      E[k] = X[k * n + v];
      H[k] = X[(3 + k) * n + v];
    }
    // fwd(c, l) = (C_l E_c)(v), bwd(c, l) = (C_l^* H_c)(v)
    auto fwd = [&](int c, int l) {
      const long long u = fw[l] ? v - (len[l] - 1) * step[l] : v + step[l];
      C e = X[c * n + u];
      if (fw[l]) e = cmul(a.wrap[l], e);
      return cscale(csub(e, E[c]), a.inv_delta[l]);
    };
    auto bwd = [&](int c, int l) {
      const long long u = bw[l] ? v + (len[l] - 1) * step[l] : v - step[l];
      C h = X[(3 + c) * n + u];
      if (bw[l]) h = cmulc(a.wrap[l], h);
      return cscale(csub(h, H[c]), a.inv_delta[l]);
    };
    const C CE[3] = {csub(fwd(2, 1), fwd(1, 2)), csub(fwd(0, 2), fwd(2, 0)), csub(fwd(1, 0), fwd(0, 1))};
    const C CH[3] = {csub(bwd(1, 2), bwd(2, 1)), csub(bwd(2, 0), bwd(0, 2)), csub(bwd(0, 1), bwd(1, 0))};
    double ip[3], im[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ip[k] = a.inv_phi[k * n + v];
      im[k] = a.inv_mu ? a.inv_mu[k * n + v] : 1.0;
    }
    C zE[3], xH[3];
    double eps[3];
    if (a.kind == kMediumChiral) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double g = a.gam[k * n + v];
        eps[k] = 1.0 / ip[k] + g * g * im[k];
        zE[k] = cmul_mi(cscale(E[k], g));  // zeta = -i gamma
        xH[k] = cmul_i(cscale(H[k], g));   // xi = i gamma
      }
    } else {
      const double g = a.gam[v];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int o = k == a.ax_a ? a.ax_b : (k == a.ax_b ? a.ax_a : -1);
        if (o >= 0) {
          eps[k] = 1.0 / ip[k] + g * g * im[o];
          zE[k] = cmul_mi(cscale(E[o], g));
          xH[k] = cmul_i(cscale(H[o], g));
        } else {
          eps[k] = 1.0 / ip[k];
          zE[k] = mk(0.0, 0.0);
          xH[k] = mk(0.0, 0.0);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const C bt = cmul_i(cadd(zE[k], cscale(H[k], 1.0 / im[k])));  // i (zeta E + mu H)
      const C bb = cmul_mi(cadd(cscale(E[k], eps[k]), xH[k]));      // -i (eps E + xi H)
      racc += cabs2(csub(CE[k], cscale(bt, a.omega))) + cabs2(csub(CH[k], cscale(bb, a.omega)));
      bacc += cabs2(bt) + cabs2(bb);
    }
  }
  const double rt = block_sum_dbl<256>(racc);
  const double bt = block_sum_dbl<256>(bacc);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = rt;
    a.part[2 * blockIdx.x + 1] = bt;
  }
}

cudaError_t gep_residual_launch(const GepResidualArgs& a, int blocks, cudaStream_t stream) {
  k_gep_residual<<<blocks, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t basis_table_launch(const double2* lam, int n1, int n2, int n3, double alpha, double beta, double2* basis,
                               int P, int slam, long long sbasis, cudaStream_t stream) {
  const long long total = (long long)n1 * n2 * n3 * P;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_basis_table<double><<<blocks, 256, 0, stream>>>(lam, n1, n2, n3, alpha, beta, basis, P, slam, sbasis);
  return cudaGetLastError();
}

}  // namespace nfs
