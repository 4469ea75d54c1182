"""Sections 4.1-4.2: the HHPD null-space-free GEP, applied with FFTs (tier O3).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Theorem (thm:NFSEP_real_ew): under the Assumption the GEP reduces to

    B_r y = omega^{-1} A_r y,   B_r = i [[0, Sigma_r^{-1}], [-Sigma_r^{-1}, 0]],

with A_r of eq. (factor_mtx)

    A_r = diag(P_r^*, Q_r^*) [[mu^{-1} zeta, -I], [I, 0]] diag(Phi^{-1}, mu^{-1})
          [[xi mu^{-1}, I], [-I, 0]] diag(P_r, Q_r),

Hermitian positive definite.  A 4n-vector u = [u1a; u1b; u2a; u2b] holds the
coefficients of the columns of P_r = [P_2, P_1] (u1a, u1b) and of
Q_r = [Q_1, Q_2] (u2a, u2b); each quarter is a grid array (n3, n2, n1) in
spectral order.  Section 4.2 solves A_r u = b by unpreconditioned CG with FFT
products (eq. (spd_LS)) inside invert Lanczos for the largest theta = 1/omega;
here the Lanczos step is ARPACK (the paper used MATLAB eigs, also ARPACK).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import media as om
from . import yee


class NFGEP:
    def __init__(self, grid, kdota, medium, alpha=yee.DEFAULT_ALPHA, beta=yee.DEFAULT_BETA, a=1.0):
        self.grid = tuple(grid)
        self.kdota = tuple(float(k) for k in kdota)
        self.medium = medium
        self.sym = yee.Symbols(grid, kdota, alpha, beta, a)
        eps, mu, xi, zeta = om.tensors(medium)
        self.mu_inv = om.batched_inv(mu)
        self.xi, self.zeta = xi, zeta
        # the fixed per-voxel factors xi mu^{-1} and mu^{-1} zeta of eq.
        # (factor_mtx), formed once per medium rather than in every product
        self.xi_mu_inv = om.tmul(xi, self.mu_inv)
        self.mu_inv_zeta = om.tmul(self.mu_inv, zeta)
        # Phi = eps_d - xi_d mu_d^{-1} zeta_d (Section 4.1)
        self.phi_inv = om.batched_inv(eps - om.tmul(om.tmul(xi, self.mu_inv), zeta))
        n1, n2, n3 = grid
        self.n = n1 * n2 * n3
        self.shape = (n3, n2, n1)
        self.nmatvec = 0

    # -- vectors ------------------------------------------------------------
    def split(self, u):
        return np.asarray(u, np.complex128).reshape((4,) + self.shape)

    # -- eq. (factor_mtx) -----------------------------------------------------
    def middle(self, p, q):
        """Apply the three middle factors of A_r to the real-space pair (p, q);
        returns (f, w), the inputs of P_r^* and Q_r^*."""
        # [[xi mu^{-1}, I], [-I, 0]] [p; q]
        a = om.tapply(self.xi_mu_inv, p) + q
        b = -p
        # diag(Phi^{-1}, mu^{-1})
        c = om.tapply(self.phi_inv, a)
        d = om.tapply(self.mu_inv, b)
        # [[mu^{-1} zeta, -I], [I, 0]]
        f = om.tapply(self.mu_inv_zeta, c) - d
        w = c
        return f, w

    def fields(self, u):
        """(p, q) = (P_r u1, Q_r u2) in real space, each (3, n3, n2, n1)."""
        u = self.split(u)
        return yee.apply_Pr(self.sym, u[0], u[1]), yee.apply_Qr(self.sym, u[2], u[3])

    def Ar(self, u):
        """A_r u via FFT products (Section 4.2)."""
        self.nmatvec += 1
        p, q = self.fields(u)
        f, w = self.middle(p, q)
        o1a, o1b = yee.apply_PrH(self.sym, f)
        o2a, o2b = yee.apply_QrH(self.sym, w)
        return np.stack([o1a, o1b, o2a, o2b]).ravel()

    def Br(self, v):
        """B_r v = i [Sigma_r^{-1} v2; -Sigma_r^{-1} v1], Sigma_r = diag(Lq^{1/2}, Lq^{1/2})."""
        v = self.split(v)
        s = self.sym.sigma
        return (1j * np.stack([v[2] / s, v[3] / s, -v[0] / s, -v[1] / s])).ravel()

    # -- dense forms for small grids (pins) --------------------------------
    def dense_Ar(self):
        Pr, Sr, Qr = yee.dense_svd_factors(self.sym)
        n = self.n
        M = np.zeros((6 * n, 6 * n), np.complex128)
        blk = lambda t: om.block_sparse(t).toarray()   # noqa: E731
        mu_inv, phi_inv = blk(self.mu_inv), blk(self.phi_inv)
        xi, zeta = blk(self.xi), blk(self.zeta)
        I = np.eye(3 * n)
        left = np.block([[mu_inv @ zeta, -I], [I, np.zeros_like(I)]])
        mid = np.block([[phi_inv, np.zeros_like(I)], [np.zeros_like(I), mu_inv]])
        right = np.block([[xi @ mu_inv, I], [-I, np.zeros_like(I)]])
        M = left @ mid @ right
        D = np.block([[Pr, np.zeros_like(Pr)], [np.zeros_like(Qr), Qr]])
        return D.conj().T @ M @ D

    def dense_Br(self):
        n = self.n
        s = np.concatenate([self.sym.sigma.ravel()] * 2)
        Z = np.zeros((2 * n, 2 * n))
        Si = np.diag(1.0 / s)
        return 1j * np.block([[Z, Si], [-Si, Z]])

    # -- solvers ------------------------------------------------------------
    def op_A(self):
        N = 4 * self.n
        return spla.LinearOperator((N, N), matvec=self.Ar, dtype=np.complex128)

    def cg(self, b, tol=1e-12, maxiter=2000, x0=None):
        """Unpreconditioned CG on A_r x = b (eq. (spd_LS)); returns (x, iterations)."""
        it = [0]

        def cb(_):
            it[0] += 1
        x, info = spla.cg(self.op_A(), b, x0=x0, rtol=tol, atol=0.0, maxiter=maxiter, callback=cb)
        if info != 0:
            raise RuntimeError(f"oracle CG did not converge (info={info})")
        return x, it[0]

    def eigs(self, nev, tol=1e-12, cg_tol=1e-13, ncv=None, seed=0):
        """nev smallest positive omega of the NFGEP by invert Lanczos on
        (B_r, A_r): the largest theta = 1/omega of B_r y = theta A_r y (ARPACK
        in mode 2 with the A_r-inverse applied by CG).  Returns (omega ascending,
        Y (4n x nev))."""
        N = 4 * self.n
        B = spla.LinearOperator((N, N), matvec=self.Br, dtype=np.complex128)
        Minv = spla.LinearOperator((N, N), matvec=lambda b: self.cg(b, cg_tol)[0],
                                   dtype=np.complex128)
        rng = np.random.default_rng(seed)
        v0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        if ncv is None:
            ncv = min(N - 1, max(3 * nev, 2 * nev + 1))
        theta, Y = spla.eigs(B, k=nev, M=self.op_A(), Minv=Minv, which="LR", ncv=ncv,
                             tol=tol, v0=v0)
        theta = np.real(theta)
        order = np.argsort(-theta)
        omega = 1.0 / theta[order]
        return omega, Y[:, order]

    # -- Algorithm 1, last step: the fields of the GEP -----------------------
    def eigvec_fields(self, y):
        """x = [E; H] = B^{-1} diag(P_r, Q_r) y (Algorithm 1, final step), with
        B = i [[zeta_d, mu_d], [-eps_d, -xi_d]] of eq. (mtx_B).  B couples only
        the six components of one voxel index, so B x = [P_r y1; Q_r y2] is
        solved as one 6 x 6 system per voxel.  Returns (6, n3, n2, n1):
        E_x, E_y, E_z, H_x, H_y, H_z."""
        p, q = self.fields(y)
        eps, mu, xi, zeta = om.tensors(self.medium)
        B = 1j * np.concatenate([np.concatenate([zeta, mu], axis=1),
                                 np.concatenate([-eps, -xi], axis=1)], axis=0)   # (6, 6, n3, n2, n1)
        Bv = np.moveaxis(B.reshape(6, 6, self.n), -1, 0)                         # (n, 6, 6)
        rhs = np.concatenate([p, q]).reshape(6, self.n).T                       # (n, 6)
        x = np.linalg.solve(Bv, rhs[..., None])[..., 0]
        return x.T.reshape((6,) + self.shape)

    def residual(self, omega, y):
        """||A_r y - omega B_r y|| / ||y||  (scale-free)."""
        return np.linalg.norm(self.Ar(y) - omega * self.Br(y)) / np.linalg.norm(y)
