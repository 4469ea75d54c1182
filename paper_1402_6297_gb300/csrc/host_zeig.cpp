// Complex Schur decomposition, its reordering and the eigenvectors of the
// triangular factor (see host_zeig.h).
#include "host_zeig.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace nfs {
namespace host {

namespace {

constexpr double kEps = std::numeric_limits<double>::epsilon();

// Unitary 2 x 2 rotation G = [[c, s], [-conj(s), c]] (c real) with
// G [a; b] = [r; 0], |r| = sqrt(|a|^2 + |b|^2).
void givens(cplxd a, cplxd b, double& c, cplxd& s) {
  const double na = std::abs(a), nb = std::abs(b);
  if (nb == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (na == 0.0) {
    c = 0.0;
    s = std::conj(b) / nb;
    return;
  }
  const double r = std::hypot(na, nb);
  c = na / r;
  s = (a / na) * std::conj(b) / r;
}

// rows (i, i+1) <- G rows, columns [j0, j1)
void rot_rows(int m, std::vector<cplxd>& A, int i, double c, cplxd s, int j0, int j1) {
  for (int j = j0; j < j1; ++j) {
    const cplxd x = A[(size_t)i * m + j], y = A[(size_t)(i + 1) * m + j];
    A[(size_t)i * m + j] = c * x + s * y;
    A[(size_t)(i + 1) * m + j] = -std::conj(s) * x + c * y;
  }
}

// columns (k, k+1) <- columns G^*, rows [r0, r1)
void rot_cols(int m, std::vector<cplxd>& A, int k, double c, cplxd s, int r0, int r1) {
  for (int r = r0; r < r1; ++r) {
    const cplxd u = A[(size_t)r * m + k], v = A[(size_t)r * m + k + 1];
    A[(size_t)r * m + k] = u * c + v * std::conj(s);
    A[(size_t)r * m + k + 1] = -u * s + v * c;
  }
}

// A -> upper Hessenberg H = Q^* A Q by Householder reflections.
void hessenberg(int m, std::vector<cplxd>& A, std::vector<cplxd>& Q) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<cplxd> v(m);
  for (int k = 0; k + 2 < m; ++k) {
    double tail = 0.0;
    for (int i = k + 2; i < m; ++i) tail += std::norm(A[(size_t)i * m + k]);
    if (tail == 0.0) continue;
    const cplxd x0 = A[(size_t)(k + 1) * m + k];
    const double nrm = std::sqrt(tail + std::norm(x0));
    const cplxd phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplxd(1.0);
    const cplxd alpha = -phase * nrm;  // v = x - alpha e1 avoids cancellation
    std::fill(v.begin(), v.end(), cplxd(0.0));
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < m; ++i) v[i] = A[(size_t)i * m + k];
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += std::norm(v[i]);
    const double beta = 2.0 / vv;
    // A <- H A, H = I - beta v v^*
    for (int j = 0; j < m; ++j) {
      cplxd d = 0.0;
      for (int i = k + 1; i < m; ++i) d += std::conj(v[i]) * A[(size_t)i * m + j];
      d *= beta;
      for (int i = k + 1; i < m; ++i) A[(size_t)i * m + j] -= v[i] * d;
    }
    // A <- A H, Q <- Q H
    for (std::vector<cplxd>* M : {&A, &Q}) {
      for (int r = 0; r < m; ++r) {
        cplxd d = 0.0;
        for (int i = k + 1; i < m; ++i) d += (*M)[(size_t)r * m + i] * v[i];
        d *= beta;
        for (int i = k + 1; i < m; ++i) (*M)[(size_t)r * m + i] -= d * std::conj(v[i]);
      }
    }
    for (int i = k + 2; i < m; ++i) A[(size_t)i * m + k] = 0.0;
  }
}

// eigenvalue of [[a, b], [c, d]] nearer d
cplxd wilkinson(cplxd a, cplxd b, cplxd c, cplxd d) {
  const cplxd half = 0.5 * (a - d);
  const cplxd disc = std::sqrt(half * half + b * c);
  const cplxd l1 = d + half + disc, l2 = d + half - disc;
  return std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
}

}  // namespace

bool complex_schur(int m, std::vector<cplxd>& A, std::vector<cplxd>& Q) {
  if (m <= 0) return true;
  hessenberg(m, A, Q);
  auto H = [&](int i, int j) -> cplxd& { return A[(size_t)i * m + j]; };
  double anorm = 0.0;
  for (const cplxd& x : A) anorm = std::max(anorm, std::abs(x));
  std::vector<double> cs(m);
  std::vector<cplxd> ss(m);
  int hi = m - 1, iter = 0, total = 0;
  const int max_total = 100 * m + 100;
  while (hi > 0) {
    // the unreduced block [lo, hi]
    int lo = hi;
    while (lo > 0) {
      const double sub = std::abs(H(lo, lo - 1));
      double scale = std::abs(H(lo, lo)) + std::abs(H(lo - 1, lo - 1));
      if (scale == 0.0) scale = anorm;
      if (sub <= kEps * scale) {
        H(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // a 1 x 1 block has converged
      --hi;
      iter = 0;
      continue;
    }
    if (++total > max_total) return false;
    ++iter;
    cplxd mu;
    if (iter % 11 == 0) {
      // exceptional shift: break a cycle of the Wilkinson shift
      mu = H(hi, hi) + cplxd(0.75, 0.4375) * std::abs(H(hi, hi - 1));
    } else {
      mu = wilkinson(H(hi - 1, hi - 1), H(hi - 1, hi), H(hi, hi - 1), H(hi, hi));
    }
    // explicit shifted QR step on [lo, hi]: H - mu I = G^* R, H <- R G^* + mu I,
    // with the rotations carried across the whole matrix (full Schur form)
    for (int i = lo; i <= hi; ++i) H(i, i) -= mu;
    for (int k = lo; k < hi; ++k) {
      givens(H(k, k), H(k + 1, k), cs[k], ss[k]);
      rot_rows(m, A, k, cs[k], ss[k], k, m);
      H(k + 1, k) = 0.0;
    }
    for (int k = lo; k < hi; ++k) {
      rot_cols(m, A, k, cs[k], ss[k], 0, std::min(k + 2, hi) + 1);
      rot_cols(m, Q, k, cs[k], ss[k], 0, m);
    }
    for (int i = lo; i <= hi; ++i) H(i, i) += mu;
  }
  for (int i = 1; i < m; ++i)
    for (int j = 0; j < i; ++j) H(i, j) = 0.0;
  return true;
}

void schur_reorder(int m, std::vector<cplxd>& T, std::vector<cplxd>& Q, const std::vector<int>& select) {
  std::vector<int> sel(select.begin(), select.end());
  int placed = 0;
  for (int i = 0; i < m; ++i) {
    if (!sel[i]) continue;
    // move entry i to position `placed` by adjacent swaps
    for (int k = i - 1; k >= placed; --k) {
      const cplxd t11 = T[(size_t)k * m + k], t22 = T[(size_t)(k + 1) * m + k + 1];
      const cplxd t12 = T[(size_t)k * m + k + 1];
      // Z = [z, z_perp] with z the eigenvector of the block for t22:
      // (T - t22 I) z = 0 gives z ~ [t12, t22 - t11]
      cplxd z0 = t12, z1 = t22 - t11;
      const double r = std::hypot(std::abs(z0), std::abs(z1));
      if (r == 0.0) {
        std::swap(sel[k], sel[k + 1]);
        continue;  // equal entries and no coupling: the swap changes nothing
      }
      z0 /= r;
      z1 /= r;
      // rows (k, k+1) <- Z^* rows; columns (k, k+1) <- columns Z
      for (int j = k; j < m; ++j) {
        const cplxd x = T[(size_t)k * m + j], y = T[(size_t)(k + 1) * m + j];
        T[(size_t)k * m + j] = std::conj(z0) * x + std::conj(z1) * y;
        T[(size_t)(k + 1) * m + j] = -z1 * x + z0 * y;
      }
      for (std::vector<cplxd>* M : {&T, &Q}) {
        const int rows = M == &T ? k + 2 : m;
        for (int rr = 0; rr < rows; ++rr) {
          const cplxd u = (*M)[(size_t)rr * m + k], v = (*M)[(size_t)rr * m + k + 1];
          (*M)[(size_t)rr * m + k] = u * z0 + v * z1;
          (*M)[(size_t)rr * m + k + 1] = -u * std::conj(z1) + v * std::conj(z0);
        }
      }
      T[(size_t)(k + 1) * m + k] = 0.0;
      std::swap(sel[k], sel[k + 1]);
    }
    ++placed;
  }
}

void triangular_eigvecs(int m, const std::vector<cplxd>& T, std::vector<cplxd>& V) {
  V.assign((size_t)m * m, 0.0);
  double tnorm = 0.0;
  for (const cplxd& x : T) tnorm = std::max(tnorm, std::abs(x));
  const double small = std::max(tnorm, 1.0) * kEps;
  std::vector<cplxd> v(m);
  for (int j = 0; j < m; ++j) {
    std::fill(v.begin(), v.end(), cplxd(0.0));
    v[j] = 1.0;
    const cplxd lam = T[(size_t)j * m + j];
    for (int i = j - 1; i >= 0; --i) {
      cplxd acc = 0.0;
      for (int k = i + 1; k <= j; ++k) acc += T[(size_t)i * m + k] * v[k];
      cplxd den = T[(size_t)i * m + i] - lam;
      if (std::abs(den) < small) den = small;  // equal eigenvalues: perturbed
      v[i] = -acc / den;
    }
    double nrm = 0.0;
    for (int i = 0; i <= j; ++i) nrm += std::norm(v[i]);
    nrm = std::sqrt(nrm);
    for (int i = 0; i <= j; ++i) V[(size_t)i * m + j] = v[i] / nrm;
  }
}

}  // namespace host
}  // namespace nfs
