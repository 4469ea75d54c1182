"""Section 4 (thm:nfep) and Algorithm 1's second branch: the null space free
eigenvalue problem for any nonsingular B (tier O3 for media outside the
Assumption).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Theorem (thm:nfep): the nonzero eigenvalues of the GEP (eq. discrete_GEP_EH)
are the eigenvalues of the 4n x 4n standard problem (eq. NFSEP_org)

    M y = omega y,   M = diag(Sigma_r^{1/2} Q_r^*, Sigma_r^{1/2} P_r^*) B^{-1}
                         diag(P_r Sigma_r^{1/2}, Q_r Sigma_r^{1/2}),

B = i [[zeta_d, mu_d], [-eps_d, -xi_d]] (eq. mtx_B).  M is not Hermitian in
general (lossy media, Tellegen coupling, Phi not positive definite) and its
eigenvalues are complex; Section 4 names shift-and-invert Arnoldi for it.
Algorithm 1 (else branch) then scales y by diag(Sigma_r^{1/2}, Sigma_r^{1/2})
and recovers x = [E; H] = B^{-1} diag(P_r, Q_r) y.

The vector layout is that of :mod:`oracle.nfgep`: y = [y1a; y1b; y2a; y2b],
the coefficients of P_r = [P_2, P_1] and Q_r = [Q_1, Q_2], each quarter a grid
array (n3, n2, n1) in spectral order; Sigma_r = diag(Lambda_q^{1/2},
Lambda_q^{1/2}) scales each quarter by sqrt(Lambda_q) at its index.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import media as om
from . import yee


class NFSEP:
    def __init__(self, grid, kdota, medium, alpha=yee.DEFAULT_ALPHA, beta=yee.DEFAULT_BETA, a=1.0):
        self.grid = tuple(grid)
        self.kdota = tuple(float(k) for k in kdota)
        self.medium = medium
        self.sym = yee.Symbols(grid, kdota, alpha, beta, a)
        n1, n2, n3 = grid
        self.n = n1 * n2 * n3
        self.shape = (n3, n2, n1)
        eps, mu, xi, zeta = om.tensors(medium)
        # eq. (mtx_B), one 6 x 6 block per voxel index
        B = 1j * np.concatenate([np.concatenate([zeta, mu], axis=1),
                                 np.concatenate([-eps, -xi], axis=1)], axis=0)
        self.Bv = np.moveaxis(B.reshape(6, 6, self.n), -1, 0)   # (n, 6, 6)
        self.sqrt_sigma = np.sqrt(self.sym.sigma)                # Sigma_r^{1/2} per index
        self.nmatvec = 0

    def split(self, y):
        return np.asarray(y, np.complex128).reshape((4,) + self.shape)

    def B_solve(self, p, q):
        """[e; h] = B^{-1} [p; q], voxel by voxel; p, q, e, h are (3, n3, n2, n1)."""
        rhs = np.concatenate([p, q]).reshape(6, self.n).T
        x = np.linalg.solve(self.Bv, rhs[..., None])[..., 0].T.reshape((6,) + self.shape)
        return x[:3], x[3:]

    def fields(self, y):
        """Algorithm 1, else branch: x = [E; H] = B^{-1} diag(P_r, Q_r) diag(Sigma_r^{1/2},
        Sigma_r^{1/2}) y for an NFSEP eigenvector y.  Returns (6, n3, n2, n1)."""
        y = self.split(y)
        s = self.sqrt_sigma
        p = yee.apply_Pr(self.sym, s * y[0], s * y[1])
        q = yee.apply_Qr(self.sym, s * y[2], s * y[3])
        e, h = self.B_solve(p, q)
        return np.concatenate([e, h])

    def apply(self, y):
        """M y (eq. NFSEP_org) with FFT products."""
        self.nmatvec += 1
        x = self.fields(y)
        s = self.sqrt_sigma
        o1a, o1b = yee.apply_QrH(self.sym, x[:3])
        o2a, o2b = yee.apply_PrH(self.sym, x[3:])
        return np.stack([s * o1a, s * o1b, s * o2a, s * o2b]).ravel()

    def dense(self):
        """M as a dense 4n x 4n matrix, column by column (small grids)."""
        N = 4 * self.n
        M = np.empty((N, N), np.complex128)
        for j in range(N):
            e = np.zeros(N, np.complex128)
            e[j] = 1.0
            M[:, j] = self.apply(e)
        return M

    def eigs_near(self, sigma, nev, tol=1e-12, inner_tol=1e-13, seed=0):
        """The nev eigenvalues of M nearest sigma and their eigenvectors, by
        shift-and-invert Arnoldi (ARPACK on (M - sigma I)^{-1}, each inverse
        applied by GMRES).  Returns (omega sorted by distance to sigma, Y)."""
        N = 4 * self.n
        shifted = spla.LinearOperator((N, N), matvec=lambda v: self.apply(v) - sigma * v, dtype=np.complex128)

        def inv(b):
            x, info = spla.gmres(shifted, b, rtol=inner_tol, atol=0.0, restart=200, maxiter=200)
            if info != 0:
                raise RuntimeError(f"oracle GMRES did not converge (info={info})")
            return x
        Minv = spla.LinearOperator((N, N), matvec=inv, dtype=np.complex128)
        Mop = spla.LinearOperator((N, N), matvec=self.apply, dtype=np.complex128)
        rng = np.random.default_rng(seed)
        v0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        w, Y = spla.eigs(Mop, k=nev, sigma=sigma, OPinv=Minv, v0=v0, tol=tol,
                         ncv=min(N - 1, max(2 * nev + 1, 20)))
        order = np.argsort(np.abs(w - sigma))
        return w[order], Y[:, order]
