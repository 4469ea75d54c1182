// Test shim: the library's host Krylov drivers (krylov.cpp) run on host
// vectors with a dense operator, exposed with a C ABI (interleaved re, im
// doubles) for the CPU test-suite.
#include <complex>
#include <random>
#include <vector>

#include "../../paper_1402_6297_gb300/csrc/krylov.h"

using nfs::host::cplxd;
using Vec = std::vector<cplxd>;

namespace {

std::vector<cplxd> load(size_t len, const double* a) {
  std::vector<cplxd> v(len);
  for (size_t i = 0; i < len; ++i) v[i] = cplxd(a[2 * i], a[2 * i + 1]);
  return v;
}

// Op = A - shift I (row-major dense N x N) on host vectors
struct DenseBasis : virtual nfs::host::KrylovOps {
  int N;
  const Vec* A;
  cplxd shift;
  std::vector<Vec> V;
  Vec w;
  DenseBasis(int n, const Vec* a, cplxd sh, int cap) : N(n), A(a), shift(sh), V(cap, Vec(n)), w(n) {}
  void mul(const Vec& x, Vec& y) const {
    for (int r = 0; r < N; ++r) {
      cplxd acc = 0.0;
      for (int c = 0; c < N; ++c) acc += (*A)[(size_t)r * N + c] * x[c];
      y[r] = acc - shift * x[r];
    }
  }
  int apply(int j) override { mul(V[j], w); return 0; }
  int dots(int m, Vec& c) override {
    c.assign(m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int r = 0; r < N; ++r) c[i] += std::conj(V[i][r]) * w[r];
    return 0;
  }
  int axpy(int m, const Vec& c) override {
    for (int i = 0; i < m; ++i)
      for (int r = 0; r < N; ++r) w[r] -= c[i] * V[i][r];
    return 0;
  }
  int norm(double& nrm) override {
    double s = 0.0;
    for (const cplxd& x : w) s += std::norm(x);
    nrm = std::sqrt(s);
    return 0;
  }
  int store(int j, double scale) override {
    for (int r = 0; r < N; ++r) V[j][r] = scale * w[r];
    return 0;
  }
  int rotate(int m, const Vec& Q, int k) override {
    std::vector<Vec> out(k, Vec(N, 0.0));
    for (int i = 0; i < k; ++i)
      for (int r = 0; r < m; ++r)
        for (int q = 0; q < N; ++q) out[i][q] += V[r][q] * Q[(size_t)r * k + i];
    for (int i = 0; i < k; ++i) V[i] = out[i];
    return 0;
  }
  int copy(int dst, int src) override { V[dst] = V[src]; return 0; }
  int load(int j) override { w = V[j]; return 0; }
  int random(unsigned long long seed) override {
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd;
    for (int r = 0; r < N; ++r) w[r] = cplxd(nd(rng), nd(rng));
    return 0;
  }
};

struct DenseGmres : DenseBasis, nfs::host::GmresOps {
  Vec b, x;
  DenseGmres(int n, const Vec* a, cplxd sh, int cap, Vec rhs)
      : DenseBasis(n, a, sh, cap), b(std::move(rhs)), x(n, 0.0) {}
  int residual() override {
    mul(x, w);
    for (int r = 0; r < N; ++r) w[r] = b[r] - w[r];
    return 0;
  }
  int update(int m, const Vec& y) override {
    for (int i = 0; i < m; ++i)
      for (int r = 0; r < N; ++r) x[r] += y[i] * V[i][r];
    return 0;
  }
};

// Op = (A - sigma I)^{-1}, each application one GMRES solve
struct ShiftInvert : DenseBasis {
  int inner_m;
  double inner_tol;
  int inner_its = 0;
  ShiftInvert(int n, const Vec* a, cplxd sigma, int cap, int im, double it)
      : DenseBasis(n, a, sigma, cap), inner_m(im), inner_tol(it) {}
  int apply(int j) override {
    DenseGmres g(N, A, shift, inner_m + 1, V[j]);
    double bn = 0.0;
    for (const cplxd& v : V[j]) bn += std::norm(v);
    nfs::host::GmresResult gr;
    const int rc = nfs::host::gmres(g, inner_m, inner_tol, std::sqrt(bn), 100000, gr);
    if (rc != 0) return rc;
    if (gr.status != 0) return gr.status;
    inner_its += gr.iterations;
    w = g.x;
    return 0;
  }
};

void start(DenseBasis& ops, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd;
  for (int r = 0; r < ops.N; ++r) ops.V[0][r] = cplxd(nd(rng), nd(rng));
}

void out_vec(const Vec& v, double* o) {
  for (size_t i = 0; i < v.size(); ++i) {
    o[2 * i] = v[i].real();
    o[2 * i + 1] = v[i].imag();
  }
}

}  // namespace

extern "C" int shim_gmres(int N, const double* A, double sre, double sim, const double* b, double* x, int m,
                          double tol, int maxit, int* iters, double* relres) {
  const Vec a = load((size_t)N * N, A);
  DenseGmres g(N, &a, cplxd(sre, sim), m + 1, load(N, b));
  double bn = 0.0;
  for (const cplxd& v : g.b) bn += std::norm(v);
  nfs::host::GmresResult r;
  const int rc = nfs::host::gmres(g, m, tol, std::sqrt(bn), maxit, r);
  out_vec(g.x, x);
  *iters = r.iterations;
  *relres = r.relres;
  return rc != 0 ? rc : r.status;
}

// the nev eigenvalues of A of largest modulus
extern "C" int shim_krylov_schur(int N, const double* A, int nev, int m, double tol, int max_restarts,
                                 unsigned seed, double* theta, double* Y, int* steps, int* restarts) {
  const Vec a = load((size_t)N * N, A);
  DenseBasis ops(N, &a, 0.0, m + 1);
  start(ops, seed);
  nfs::host::ArnoldiResult r;
  const int rc = nfs::host::krylov_schur(ops, nev, m, tol, max_restarts, r);
  if (rc != 0) return rc;
  out_vec(r.theta, theta);
  for (int e = 0; e < nev; ++e)
    for (int q = 0; q < N; ++q) {
      Y[2 * ((size_t)e * N + q)] = ops.V[e][q].real();
      Y[2 * ((size_t)e * N + q) + 1] = ops.V[e][q].imag();
    }
  *steps = r.steps;
  *restarts = r.restarts;
  return r.status;
}

// as shim_krylov_schur from a given start vector v0
extern "C" int shim_krylov_schur_from(int N, const double* A, const double* v0, int nev, int m, double tol,
                                      int max_restarts, double* theta, int* steps, int* injections) {
  const Vec a = load((size_t)N * N, A);
  DenseBasis ops(N, &a, 0.0, m + 1);
  ops.V[0] = load(N, v0);
  nfs::host::ArnoldiResult r;
  const int rc = nfs::host::krylov_schur(ops, nev, m, tol, max_restarts, r);
  if (rc != 0) return rc;
  out_vec(r.theta, theta);
  *steps = r.steps;
  *injections = r.injections;
  return r.status;
}

// the nev eigenvalues of A nearest sigma by shift-and-invert Arnoldi
extern "C" int shim_shift_invert(int N, const double* A, double sre, double sim, int nev, int m, double tol,
                                 int inner_m, double inner_tol, unsigned seed, double* lam, int* steps,
                                 int* inner_its) {
  const Vec a = load((size_t)N * N, A);
  const cplxd sigma(sre, sim);
  ShiftInvert ops(N, &a, sigma, m + 1, inner_m, inner_tol);
  start(ops, seed);
  nfs::host::ArnoldiResult r;
  const int rc = nfs::host::krylov_schur(ops, nev, m, tol, 100, r);
  if (rc != 0) return rc;
  Vec l(nev);
  for (int e = 0; e < nev; ++e) l[e] = sigma + 1.0 / r.theta[e];
  out_vec(l, lam);
  *steps = r.steps;
  *inner_its = ops.inner_its;
  return r.status;
}
