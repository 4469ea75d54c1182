// Restarted GMRES and Krylov-Schur Arnoldi drivers (see krylov.h).
#include "krylov.h"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "host_zeig.h"

namespace nfs {
namespace host {

namespace {

constexpr int kOk = 0;
constexpr int kNoConv = -6;
constexpr int kBreakdown = -7;

#define KRY_TRY(call)          \
  do {                         \
    const int r_ = (call);     \
    if (r_ != kOk) return r_;  \
  } while (0)

// G = [[c, s], [-conj(s), c]], c real, with G [a; b] = [r; 0]
void rotation(cplxd a, cplxd b, double& c, cplxd& s) {
  const double na = std::abs(a), nb = std::abs(b);
  if (nb == 0.0) {
    c = 1.0;
    s = 0.0;
  } else if (na == 0.0) {
    c = 0.0;
    s = std::conj(b) / nb;
  } else {
    const double r = std::hypot(na, nb);
    c = na / r;
    s = (a / na) * std::conj(b) / r;
  }
}

// Two classical Gram-Schmidt passes of w against V_0 .. V_{n-1}; the summed
// coefficients are returned (the Arnoldi column).
int orthogonalise(KrylovOps& ops, int n, std::vector<cplxd>& h) {
  std::vector<cplxd> c1, c2;
  KRY_TRY(ops.dots(n, c1));
  KRY_TRY(ops.axpy(n, c1));
  KRY_TRY(ops.dots(n, c2));
  KRY_TRY(ops.axpy(n, c2));
  h.assign(n, 0.0);
  for (int i = 0; i < n; ++i) h[i] = c1[i] + c2[i];
  return kOk;
}

}  // namespace

void GivensLS::reset(int m, double beta) {
  m_ = m;
  k_ = 0;
  R_.assign((size_t)(m + 1) * m, cplxd(0.0));
  g_.assign(m + 1, cplxd(0.0));
  sn_.assign(m, cplxd(0.0));
  cs_.assign(m, 0.0);
  g_[0] = beta;
}

double GivensLS::add_column(const cplxd* col, double h) {
  const int j = k_;
  auto Rc = [&](int r, int cc) -> cplxd& { return R_[(size_t)r * m_ + cc]; };
  for (int i = 0; i <= j; ++i) Rc(i, j) = col[i];
  Rc(j + 1, j) = h;
  for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
    const cplxd x = Rc(i, j), y = Rc(i + 1, j);
    Rc(i, j) = cs_[i] * x + sn_[i] * y;
    Rc(i + 1, j) = -std::conj(sn_[i]) * x + cs_[i] * y;
  }
  rotation(Rc(j, j), Rc(j + 1, j), cs_[j], sn_[j]);
  const cplxd x = Rc(j, j), y = Rc(j + 1, j);
  Rc(j, j) = cs_[j] * x + sn_[j] * y;
  Rc(j + 1, j) = 0.0;
  const cplxd gj = g_[j];
  g_[j] = cs_[j] * gj;
  g_[j + 1] = -std::conj(sn_[j]) * gj;
  k_ = j + 1;
  return std::abs(g_[j + 1]);
}

bool GivensLS::solve(std::vector<cplxd>& y) const {
  y.assign(k_, cplxd(0.0));
  for (int i = k_ - 1; i >= 0; --i) {
    cplxd acc = g_[i];
    for (int q = i + 1; q < k_; ++q) acc -= R_[(size_t)i * m_ + q] * y[q];
    const cplxd d = R_[(size_t)i * m_ + i];
    if (d == cplxd(0.0)) return false;
    y[i] = acc / d;
  }
  return true;
}

int gmres(GmresOps& ops, int m, double tol, double bnorm, int maxit, GmresResult& out) {
  out = GmresResult{};
  if (m < 1 || !(tol > 0.0)) return -1;
  if (!(bnorm > 0.0)) return kOk;  // b = 0: x is left as it is
  GivensLS ls;
  std::vector<cplxd> col;
  for (;;) {
    KRY_TRY(ops.residual());
    double beta = 0.0;
    KRY_TRY(ops.norm(beta));
    out.relres = beta / bnorm;
    if (beta <= tol * bnorm) return kOk;
    if (out.iterations >= maxit) {
      out.status = kNoConv;
      return kOk;
    }
    KRY_TRY(ops.store(0, 1.0 / beta));
    ls.reset(m, beta);
    for (int j = 0; j < m; ++j) {
      KRY_TRY(ops.apply(j));
      ++out.iterations;
      KRY_TRY(orthogonalise(ops, j + 1, col));
      double h = 0.0;
      KRY_TRY(ops.norm(h));
      const double res = ls.add_column(col.data(), h);
      const bool done = res <= tol * bnorm || out.iterations >= maxit || h == 0.0;
      if (!done && j + 1 < m) KRY_TRY(ops.store(j + 1, 1.0 / h));
      if (done) break;
    }
    // y = R^{-1} g over the cycle's columns, x += V y
    std::vector<cplxd> y;
    if (!ls.solve(y)) return kBreakdown;
    KRY_TRY(ops.update(ls.columns(), y));
    ++out.restarts;
  }
}

int krylov_schur(KrylovOps& ops, int nev, int m, double tol, int max_restarts, ArnoldiResult& res) {
  res = ArnoldiResult{};
  if (nev < 1 || m < nev + 2 || !(tol > 0.0)) return -1;
  // normalise the start vector
  KRY_TRY(ops.load(0));
  double nrm = 0.0;
  KRY_TRY(ops.norm(nrm));
  if (!(nrm > 0.0)) return kBreakdown;
  KRY_TRY(ops.store(0, 1.0 / nrm));
  // S: (m + 1) x m, Op V_{0..m-1} = V_{0..m} S
  std::vector<cplxd> S((size_t)(m + 1) * m, 0.0), col;
  auto Sx = [&](int r, int c) -> cplxd& { return S[(size_t)r * m + c]; };
  const int keep = std::max(nev + 1, std::min(m - 1, nev + (m - nev) / 2));
  int k0 = 0;
  unsigned long long injections = 0;
  for (;;) {
    for (int j = k0; j < m; ++j) {
      KRY_TRY(ops.apply(j));
      ++res.steps;
      KRY_TRY(orthogonalise(ops, j + 1, col));
      double colnorm = 0.0;
      for (int i = 0; i <= j; ++i) {
        Sx(i, j) = col[i];
        colnorm += std::norm(col[i]);
      }
      double h = 0.0;
      KRY_TRY(ops.norm(h));
      if (!(h == h)) return kBreakdown;  // NaN
      colnorm = std::sqrt(colnorm + h * h);
      if (!(h > 1e-13 * colnorm)) {
        // invariant subspace: continue from a random direction orthogonal to
        // the basis, uncoupled (S(j+1, j) = 0)
        KRY_TRY(ops.random(0x9E3779B97F4A7C15ull * ++injections + 12345));
        ++res.injections;
        std::vector<cplxd> discard;
        KRY_TRY(orthogonalise(ops, j + 1, discard));
        KRY_TRY(orthogonalise(ops, j + 1, discard));
        double r = 0.0;
        KRY_TRY(ops.norm(r));
        if (!(r > 0.0)) return kBreakdown;
        Sx(j + 1, j) = 0.0;
        KRY_TRY(ops.store(j + 1, 1.0 / r));
        continue;
      }
      Sx(j + 1, j) = h;
      KRY_TRY(ops.store(j + 1, 1.0 / h));
    }
    // Schur form of the m x m projection, the `keep` values of largest
    // modulus first
    std::vector<cplxd> T(S.begin(), S.begin() + (size_t)m * m), Q;
    if (!complex_schur(m, T, Q)) return kBreakdown;
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return std::abs(T[(size_t)a * m + a]) > std::abs(T[(size_t)b * m + b]);
    });
    std::vector<int> sel(m, 0);
    for (int i = 0; i < keep; ++i) sel[order[i]] = 1;
    schur_reorder(m, T, Q, sel);
    // b^T Q: the coupling of the residual vector V_m to the Schur vectors
    std::vector<cplxd> bq(m, 0.0);
    for (int c = 0; c < m; ++c)
      for (int r = 0; r < m; ++r) bq[c] += Sx(m, r) * Q[(size_t)r * m + c];
    // the nev of largest modulus among the kept ones, and their Ritz residuals
    std::vector<int> want(keep);
    std::iota(want.begin(), want.end(), 0);
    std::stable_sort(want.begin(), want.end(), [&](int a, int b) {
      return std::abs(T[(size_t)a * m + a]) > std::abs(T[(size_t)b * m + b]);
    });
    want.resize(nev);
    std::vector<cplxd> Z;
    triangular_eigvecs(m, T, Z);
    int nconv = 0;
    double maxres = 0.0;
    for (int i : want) {
      cplxd r = 0.0;
      for (int q = 0; q <= i; ++q) r += bq[q] * Z[(size_t)q * m + i];
      const double rel = std::abs(r) / std::abs(T[(size_t)i * m + i]);
      maxres = std::max(maxres, rel);
      if (rel <= tol) ++nconv;
    }
    res.nconv = nconv;
    res.max_residual = maxres;
    if (nconv == nev || res.restarts >= max_restarts) {
      if (nconv < nev) res.status = kNoConv;
      // eigenvectors: V Q z_i, in order of decreasing modulus
      std::vector<cplxd> C((size_t)m * nev, 0.0);
      res.theta.resize(nev);
      for (int e = 0; e < nev; ++e) {
        const int i = want[e];
        res.theta[e] = T[(size_t)i * m + i];
        for (int r = 0; r < m; ++r) {
          cplxd acc = 0.0;
          for (int q = 0; q <= i; ++q) acc += Q[(size_t)r * m + q] * Z[(size_t)q * m + i];
          C[(size_t)r * nev + e] = acc;
        }
      }
      KRY_TRY(ops.rotate(m, C, nev));
      return kOk;
    }
    // restart: V_{0..keep-1} = V Q(:, :keep), V_keep = V_m, S = [T_keep; b^T Q_keep]
    std::vector<cplxd> Qk((size_t)m * keep);
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < keep; ++c) Qk[(size_t)r * keep + c] = Q[(size_t)r * m + c];
    KRY_TRY(ops.rotate(m, Qk, keep));
    KRY_TRY(ops.copy(keep, m));
    std::fill(S.begin(), S.end(), cplxd(0.0));
    for (int r = 0; r < keep; ++r)
      for (int c = r; c < keep; ++c) Sx(r, c) = T[(size_t)r * m + c];
    for (int c = 0; c < keep; ++c) Sx(keep, c) = bq[c];
    k0 = keep;
    ++res.restarts;
  }
}

}  // namespace host
}  // namespace nfs
