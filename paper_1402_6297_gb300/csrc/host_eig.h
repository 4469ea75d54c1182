// Host-side dense symmetric eigensolver used by the Lanczos driver.
#pragma once
#include <vector>

namespace nfs {
namespace host {

// Eigen-decomposition of the real symmetric m x m matrix A (row-major):
// eigenvalues w ascending and orthonormal eigenvectors in the columns of Z
// (row-major m x m), or only the last row of Z (1 x m) when last_row_only.
// Returns false if the QR iteration cap was hit.
bool sym_eig(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& Z,
             bool last_row_only = false);

}  // namespace host
}  // namespace nfs
