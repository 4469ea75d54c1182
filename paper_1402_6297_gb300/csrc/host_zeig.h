// Dense complex non-Hermitian eigensolver for the projected matrices of an
// Arnoldi (Krylov-Schur) eigensolve of the null space free standard problem
// (eq. NFSEP_org; its operator is not Hermitian once the medium leaves the
// Assumption).  At most a few hundred rows, FP64, host only.  Matrices are
// row-major m x m arrays of std::complex<double>.
#pragma once
#include <complex>
#include <vector>

namespace nfs {
namespace host {

using cplxd = std::complex<double>;

// Complex Schur decomposition A = Q T Q^* (Q unitary, T upper triangular):
// Householder reduction to upper Hessenberg form, then shifted QR steps
// (Wilkinson shift, exceptional shifts when a block stalls) with deflation.
// On entry A holds the matrix; on return it holds T, and Q the Schur vectors.
// Returns false if the QR iteration did not converge.
bool complex_schur(int m, std::vector<cplxd>& A, std::vector<cplxd>& Q);

// Reorder a Schur form so that the diagonal entries with select[i] != 0 come
// first, in their original order, keeping A = Q T Q^* (T and Q updated by
// unitary swaps of adjacent diagonal entries).
void schur_reorder(int m, std::vector<cplxd>& T, std::vector<cplxd>& Q, const std::vector<int>& select);

// Eigenvectors of the upper triangular T by back substitution: column j of V
// (row-major m x m) solves T v = T_jj v with v_j = 1 and v_i = 0 for i > j,
// then is scaled to unit 2-norm.
void triangular_eigvecs(int m, const std::vector<cplxd>& T, std::vector<cplxd>& V);

}  // namespace host
}  // namespace nfs
