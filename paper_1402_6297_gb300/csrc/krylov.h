// Host drivers of the non-Hermitian Krylov methods for the null space free
// standard problem M y = omega y (eq. NFSEP_org) outside the Assumption:
// restarted GMRES for the shifted systems (M - sigma I) z = b, and
// Krylov-Schur Arnoldi on (M - sigma I)^{-1} for the eigenvalues nearest the
// shift (shift-and-invert Arnoldi, Section 4).  The drivers own the small
// projected matrices; every operation on the long vectors goes through a
// KrylovOps object, so the same driver runs on device vectors (the library)
// or on host vectors (the CPU tests).  The library's inner GMRES solves run
// the same iteration with the Gram-Schmidt coefficients kept on the device
// and the Hessenberg columns read in batches (nfsep.h), the least-squares
// part through GivensLS below; gmres() is the host statement of that
// iteration, exercised on host operators by the CPU tests.
#pragma once
#include <complex>
#include <vector>

namespace nfs {
namespace host {

using cplxd = std::complex<double>;

// A basis V_0 .. V_{cap-1} of long vectors and one work vector w.  Every
// call returns 0 (NFS_OK) or a negative library error code.
struct KrylovOps {
  virtual ~KrylovOps() = default;
  virtual int apply(int j) = 0;                                   // w = Op V_j
  virtual int dots(int m, std::vector<cplxd>& c) = 0;             // c_i = V_i^* w, i < m
  virtual int axpy(int m, const std::vector<cplxd>& c) = 0;       // w -= sum_{i<m} c_i V_i
  virtual int norm(double& nrm) = 0;                              // ||w||_2
  virtual int store(int j, double scale) = 0;                     // V_j = scale w
  // V_i <- sum_{r<m} V_r Q[r * k + i] for i < k (Q row-major m x k)
  virtual int rotate(int m, const std::vector<cplxd>& Q, int k) = 0;
  virtual int copy(int dst, int src) = 0;                         // V_dst = V_src
  virtual int load(int j) = 0;                                    // w = V_j
  // w = a random vector (counter-based, from seed)
  virtual int random(unsigned long long seed) = 0;
};

// Operations GMRES needs beyond the basis: the right-hand side, the
// iterate x and the residual.
struct GmresOps : virtual KrylovOps {
  virtual int residual() = 0;                                     // w = b - Op x
  virtual int update(int m, const std::vector<cplxd>& y) = 0;     // x += sum_{i<m} y_i V_i
};

struct GmresResult {
  int iterations = 0;   // operator applications
  int restarts = 0;
  double relres = 0.0;  // final ||b - Op x|| / ||b||
  int status = 0;       // 0 or NFS_ENOCONV (-6)
};

// The small least-squares problem of a GMRES cycle, min ||beta e_0 - H y||
// over the (j + 2) x (j + 1) upper Hessenberg H, kept factored by Givens
// rotations G = [[c, s], [-conj(s), c]] as the columns arrive: after column j
// the residual norm of the cycle's best iterate is |g_{j+1}|.
class GivensLS {
 public:
  void reset(int m, double beta);
  // column j of H: col[0..j], h = h_{j+1,j} >= 0; returns |g_{j+1}|
  double add_column(const cplxd* col, double h);
  int columns() const { return k_; }
  // y = R^{-1} g over the columns so far; false on a zero pivot
  bool solve(std::vector<cplxd>& y) const;

 private:
  int m_ = 0, k_ = 0;
  std::vector<cplxd> R_, g_, sn_;  // R_ row-major (m + 1) x m
  std::vector<double> cs_;
};

// Restarted GMRES(m) from the iterate the ops hold, modified Gram-Schmidt
// with one re-orthogonalisation pass, Givens rotations on the Hessenberg
// matrix.  Stops at ||r|| <= tol ||b|| (bnorm = ||b||) or after maxit
// operator applications.
int gmres(GmresOps& ops, int m, double tol, double bnorm, int maxit, GmresResult& out);

struct ArnoldiResult {
  std::vector<cplxd> theta;  // the nev eigenvalues of Op of largest modulus
  int steps = 0;             // operator applications
  int restarts = 0;
  int nconv = 0;
  double max_residual = 0.0; // max |h_{m+1,m} s_m| / |theta| over the nev
  int injections = 0;        // random directions taken at invariant subspaces
  int status = 0;            // 0 or NFS_ENOCONV (-6)
};

// Krylov-Schur Arnoldi for the nev eigenvalues of Op of largest modulus
// (Op = (M - sigma I)^{-1}: the eigenvalues of M nearest sigma).  V_0 must
// hold a start vector on entry.  Basis size m (nev + 2 <= m < cap); on
// return V_0 .. V_{nev-1} hold unit eigenvectors of the nev values, in the
// order of res.theta (largest modulus first).  When the Krylov space becomes
// invariant (h_{j+1,j} at round-off) the next basis vector is a random one
// orthogonalised against the basis, with zero coupling: the Ritz values so
// far are then exact and the search goes on in the complement.
int krylov_schur(KrylovOps& ops, int nev, int m, double tol, int max_restarts, ArnoldiResult& res);

}  // namespace host
}  // namespace nfs
