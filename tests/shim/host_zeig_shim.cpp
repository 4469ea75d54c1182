// Test shim: exposes the library's host complex Schur routines with a C ABI
// (interleaved re, im doubles) so that the CPU test-suite can compare them
// with LAPACK through numpy.
#include <complex>
#include <vector>

#include "../../paper_1402_6297_gb300/csrc/host_zeig.h"

using nfs::host::cplxd;

static std::vector<cplxd> load(int m, const double* a) {
  std::vector<cplxd> v((size_t)m * m);
  for (size_t i = 0; i < v.size(); ++i) v[i] = cplxd(a[2 * i], a[2 * i + 1]);
  return v;
}
static void store(const std::vector<cplxd>& v, double* a) {
  for (size_t i = 0; i < v.size(); ++i) {
    a[2 * i] = v[i].real();
    a[2 * i + 1] = v[i].imag();
  }
}

extern "C" int shim_complex_schur(int m, const double* A, double* T, double* Q) {
  std::vector<cplxd> a = load(m, A), q;
  const bool ok = nfs::host::complex_schur(m, a, q);
  store(a, T);
  store(q, Q);
  return ok ? 0 : 1;
}

extern "C" void shim_schur_reorder(int m, double* T, double* Q, const int* select) {
  std::vector<cplxd> t = load(m, T), q = load(m, Q);
  nfs::host::schur_reorder(m, t, q, std::vector<int>(select, select + m));
  store(t, T);
  store(q, Q);
}

extern "C" void shim_triangular_eigvecs(int m, const double* T, double* V) {
  std::vector<cplxd> t = load(m, T), v;
  nfs::host::triangular_eigvecs(m, t, v);
  store(v, V);
}
