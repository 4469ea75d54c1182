// Dense real symmetric eigensolver for the Lanczos projected matrix (at most a
// few hundred rows): Householder reduction to tridiagonal form followed by
// implicit symmetric QR steps with the Wilkinson shift, accumulating the
// orthogonal transformations.  FP64, host only.
#include "host_eig.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace nfs {
namespace host {

namespace {

// A (row-major m x m, symmetric) -> tridiagonal (a: diagonal, b: b[i] couples
// i and i+1) with A = Q T Q^T; Q row-major.
void tridiagonalise(int m, std::vector<double>& A, std::vector<double>& Q, std::vector<double>& a,
                    std::vector<double>& b) {
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * m + j]; };
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<double> v(m), p(m), q(m);
  for (int k = 0; k + 2 < m; ++k) {
    // column k below the sub-diagonal
    double tail = 0.0;
    for (int i = k + 2; i < m; ++i) tail += at(i, k) * at(i, k);
    if (tail == 0.0) continue;  // already tridiagonal in this column
    const double x0 = at(k + 1, k);
    const double nrm = std::sqrt(tail + x0 * x0);
    const double alpha = x0 >= 0 ? -nrm : nrm;
    std::fill(v.begin(), v.end(), 0.0);
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < m; ++i) v[i] = at(i, k);
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    // H = I - 2 v v^T / vv ;  H A H = A - v q^T - q v^T with
    // p = (2/vv) A v, K = (v^T p) / vv, q = p - K v
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += at(i, j) * v[j];
      p[i] = 2.0 * s / vv;
    }
    double vp = 0.0;
    for (int i = k + 1; i < m; ++i) vp += v[i] * p[i];
    const double K = vp / vv;
    for (int i = 0; i < m; ++i) q[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) at(i, j) -= v[i] * q[j] + q[i] * v[j];
    // Q <- Q H
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += Q[(size_t)i * m + j] * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < m; ++j) Q[(size_t)i * m + j] -= s * v[j];
    }
  }
  a.resize(m);
  b.assign(m > 0 ? m - 1 : 0, 0.0);
  for (int i = 0; i < m; ++i) a[i] = at(i, i);
  for (int i = 0; i + 1 < m; ++i) b[i] = 0.5 * (at(i + 1, i) + at(i, i + 1));
}

// One implicit QR step with the Wilkinson shift on the window [lo, hi] of the
// symmetric tridiagonal (a, b); the rotations are also applied to the columns
// of Z (rows x m, row-major).
void qr_step(int m, int rows, int lo, int hi, std::vector<double>& a, std::vector<double>& b,
             std::vector<double>& Z) {
  const double t = 0.5 * (a[hi - 1] - a[hi]);
  const double bb = b[hi - 1];
  const double den = t + (t >= 0 ? 1.0 : -1.0) * std::hypot(t, bb);
  const double mu = den != 0.0 ? a[hi] - bb * bb / den : a[hi];
  double x = a[lo] - mu, z = b[lo];
  for (int k = lo; k < hi; ++k) {
    // rotation J on (k, k+1) with J^T [x; z] = [r; 0]: c = x / r, s = -z / r
    const double r = std::hypot(x, z);
    double c = 1.0, s = 0.0;
    if (r != 0.0) {
      c = x / r;
      s = -z / r;
    }
    if (k > lo) b[k - 1] = r;
    const double p = a[k], q = a[k + 1], e = b[k];
    a[k] = p * c * c - 2.0 * e * c * s + q * s * s;
    a[k + 1] = p * s * s + 2.0 * e * c * s + q * c * c;
    b[k] = (p - q) * c * s + e * (c * c - s * s);
    if (k + 1 < hi) {
      // bulge in (k, k+2)
      z = -s * b[k + 1];
      b[k + 1] = c * b[k + 1];
      x = b[k];
    }
    for (int i = 0; i < rows; ++i) {
      const double zk = Z[(size_t)i * m + k], zk1 = Z[(size_t)i * m + k + 1];
      Z[(size_t)i * m + k] = c * zk - s * zk1;
      Z[(size_t)i * m + k + 1] = s * zk + c * zk1;
    }
  }
}

}  // namespace

bool sym_eig(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& Z, bool last_row_only) {
  if (m <= 0) return true;
  std::vector<double> a, b, Q;
  tridiagonalise(m, A, Q, a, b);
  const int rows = last_row_only ? 1 : m;
  if (last_row_only) {
    Z.assign(Q.begin() + (size_t)(m - 1) * m, Q.begin() + (size_t)m * m);
  } else {
    Z.swap(Q);
  }
  const double eps = 2.220446049250313e-16;
  long long iters = 0;
  const long long cap = 60LL * m + 100;
  int hi = m - 1;
  while (hi > 0) {
    // deflate negligible couplings at the bottom
    if (std::fabs(b[hi - 1]) <= eps * (std::fabs(a[hi - 1]) + std::fabs(a[hi]))) {
      b[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(b[lo - 1]) > eps * (std::fabs(a[lo - 1]) + std::fabs(a[lo]))) --lo;
    if (lo > 0) b[lo - 1] = 0.0;
    if (++iters > cap) return false;
    qr_step(m, rows, lo, hi, a, b, Z);
  }
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return a[i] < a[j]; });
  w.resize(m);
  std::vector<double> Zs((size_t)rows * m);
  for (int c2 = 0; c2 < m; ++c2) {
    w[c2] = a[idx[c2]];
    for (int r = 0; r < rows; ++r) Zs[(size_t)r * m + c2] = Z[(size_t)r * m + idx[c2]];
  }
  Z.swap(Zs);
  return true;
}

}  // namespace host
}  // namespace nfs
