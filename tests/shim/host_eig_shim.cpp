// Test shim: exposes the library's host symmetric eigensolver with a C ABI so
// that the CPU test-suite can compare it with LAPACK (numpy.linalg.eigh).
#include <vector>

#include "../../paper_1402_6297_gb300/csrc/host_eig.h"

extern "C" int shim_sym_eig(int m, const double* A, double* w, double* Z) {
  std::vector<double> a(A, A + (size_t)m * m), ww, zz;
  const bool ok = nfs::host::sym_eig(m, a, ww, zz);
  for (int i = 0; i < m; ++i) w[i] = ww[i];
  for (size_t i = 0; i < (size_t)m * m; ++i) Z[i] = zz[i];
  return ok ? 0 : 1;
}

extern "C" int shim_sym_eig_last_row(int m, const double* A, double* w, double* zlast) {
  std::vector<double> a(A, A + (size_t)m * m), ww, zz;
  const bool ok = nfs::host::sym_eig(m, a, ww, zz, true);
  for (int i = 0; i < m; ++i) {
    w[i] = ww[i];
    zlast[i] = zz[i];
  }
  return ok ? 0 : 1;
}
