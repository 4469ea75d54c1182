// complex128 instantiation of the three-pass A_r product, and the eigenvalue
// gradient pass that shares its pass-1 fields.
#include <algorithm>
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

cudaError_t basis_table_launch(const double2* lam, int n1, int n2, int n3, double alpha, double beta, double2* basis,
                               int P, int slam, long long sbasis, cudaStream_t stream) {
  const long long total = (long long)n1 * n2 * n3 * P;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_basis_table<double><<<blocks, 256, 0, stream>>>(lam, n1, n2, n3, alpha, beta, basis, P, slam, sbasis);
  return cudaGetLastError();
}

}  // namespace nfs
