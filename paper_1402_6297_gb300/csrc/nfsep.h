// Device pieces of the null space free standard problem for any nonsingular
// B (eq. NFSEP_org, Algorithm 1's second branch), complex128 (nfsep.cu):
//
//   M y = [Sigma_r^{1/2} Q_r^* e ; Sigma_r^{1/2} P_r^* h],
//   [e; h] = B^{-1} [P_r Sigma_r^{1/2} y1 ; Q_r Sigma_r^{1/2} y2],
//
// run as: nfsep_prescale (Sigma_r^{1/2}), pass 1 of the A_r product
// (assembly, inverse DFTs along x and y), nfsep_pass2 (inverse DFT along z,
// B^{-1} per voxel with h into fields 0-2 and e into fields 3-5, forward DFT
// along z), pass 3 of the A_r product (which then yields [P_r^* h; Q_r^* e])
// and nfsep_post (the two halves exchanged, Sigma_r^{1/2}, optionally minus
// sigma y).  B^{-1} is stored per voxel and component as the 2 x 2 block
// coupling (p_c, q_c) to (e_c, h_c): binv[(4 c + t) n + v], t = 00, 01, 10, 11.
#pragma once
#include <cuda_runtime.h>

namespace nfs {

// t = Sigma_r^{1/2} y: each quarter times Lambda_q^{1/4} at its index
cudaError_t nfsep_prescale(const double2* y, double2* t, const double2* lam, int n1, int n2, int n3,
                           cudaStream_t s);
// out = [Sigma^{1/2} a_2; Sigma^{1/2} a_1] - sigma v (quarters: out_0 from a_2,
// out_1 from a_3, out_2 from a_0, out_3 from a_1); v may be nullptr
cudaError_t nfsep_post(const double2* a, double2* out, const double2* lam, int n1, int n2, int n3,
                       const double2* v, double2 sigma, cudaStream_t s);
cudaError_t nfsep_prepare(int n3);
cudaError_t nfsep_pass2(double2* fld, const double2* binv, const double2* tw3, int n1, int n2, int n3,
                        cudaStream_t s);
// Algorithm 1 (second branch): X = [E; H] = D [e; h] / sqrt(n) from the pass-1
// fields of Sigma_r^{1/2} y (D: the Bloch twist, from its three 1-D diagonals)
cudaError_t nfsep_fields(const double2* fld, const double2* binv, const double2* tw3, const double2* bloch,
                         int n1, int n2, int n3, double2* X, cudaStream_t s);

// Long-vector operations of the Krylov drivers (complex128):
// w -= sign * sum_{j<m} c_j V_j, c device interleaved complex, V_j at V + j N
cudaError_t zaxpy_basis(double2* w, const double2* V, long long N, const double* c, int m, double sign,
                        cudaStream_t s);
// dst = scale * src
cudaError_t zscale_copy(const double2* src, double2* dst, double scale, long long N, cudaStream_t s);
// V_i <- sum_{r<m} V_r Y[r k + i], i < k, in place (Y device interleaved complex)
cudaError_t zrotate(double2* V, int m, const double* Y, int k, long long N, cudaStream_t s);

// Restarted GMRES for the shifted systems (M - sigma I) z = b with the long-
// vector work on the device and no host round trip per step: the two
// classical Gram-Schmidt passes write their coefficients to device memory
// and the updates read them there, and a one-block kernel per step forms
// the Hessenberg column and the scale of the next basis vector.  The host
// reads a batch of columns at once and keeps the small least-squares problem
// (nfs::host::GivensLS, krylov.h).
constexpr int kGmresMax = 128;  // largest restart length
struct GmresDev {
  int done;       // 1 once h_{j+1,j} = 0 (an invariant Krylov space): later steps of the cycle store zeros
  int pad[3];
  double inv_h;   // 1 / h_{j+1,j} of the last step, 0 once done
  double pad2;
  double2 Hc[kGmresMax * (kGmresMax + 1)];  // column j of H at Hc[j (kGmresMax + 1) + i], i <= j + 1
};

// Chunks (S) of the Gram-Schmidt dot products for vectors of length N, and
// the blocks of gs_axpy / gmres_residual (the number of norm partials).
int gs_chunks(long long N);
int gs_norm_blocks(long long N);
// part[(s m + j) 2 + {0, 1}] = chunk s's share of V_j^* w, j < m (m <= kGmresMax)
cudaError_t gs_dots(const double2* V, int m, const double2* w, long long N, double* part, cudaStream_t s);
// complex128 elements of the scratch gs_axpy needs for vectors of length N
// and m <= kGmresMax basis vectors (0: none)
long long gs_axpy_tmp_len(long long N);
// w -= sum_{j<m} c_j V_j with c_j = sum_s part[(s m + j)]; with nrm_part,
// nrm_part[b] = block b's share of ||w||^2 after the update.  Short vectors
// split the sum over the basis across blocks (partial sums in tmp) so that
// enough of the GPU works on it.
cudaError_t gs_axpy(double2* w, const double2* V, long long N, int m, const double* part, double* nrm_part,
                    double2* tmp, cudaStream_t s);
int gs_axpy_kernels(long long N);  // kernel launches one gs_axpy makes
// w = b - w and the partials of ||w||^2
cudaError_t gmres_residual(const double2* b, double2* w, long long N, double* nrm_part, cudaStream_t s);
// Step j: column j of H from the two passes' partials (S chunks each, over
// j + 1 vectors) and h_{j+1,j} from nb norm partials; inv_h and done.  A
// no-op once done.
cudaError_t gmres_column(int j, const double* part1, const double* part2, int S, const double* nrm_part, int nb,
                         GmresDev* st, cudaStream_t s);
// dst = inv_h * w
cudaError_t gmres_store(const double2* w, double2* dst, const GmresDev* st, long long N, cudaStream_t s);

}  // namespace nfs
