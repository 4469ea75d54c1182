"""Section 3: the discrete GEP, solved directly (tiers O1 dense, O2 sparse).

TEST INFRASTRUCTURE (see ``oracle/__init__``).

The GEP of eq. (discrete_GEP_EH) is

    diag(C, C^*) [E; H] = omega * i [[zeta_d, mu_d], [-eps_d, -xi_d]] [E; H].

Substituting H' = i H and exchanging the two block rows gives the equivalent
pencil

    [[0, C^*], [C, 0]] [E; H'] = omega [[eps_d, -i xi_d], [i zeta_d, mu_d]] [E; H'],

whose left matrix is Hermitian and whose right matrix is Hermitian exactly
when xi_d^* = zeta_d and positive definite exactly when mu_d > 0 and
Phi = eps_d - xi_d mu_d^{-1} zeta_d > 0 (the Assumption, eq. (assump)).  This
reading is the oracle's choice: it reaches the same eigenvalues as the GEP
(pinned against a non-Hermitian solve of the GEP itself in the tests) while
letting a Hermitian-definite solver return real eigenvalues.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import media as om
from . import yee


def gep_matrices(grid, kdota, medium, a=1.0):
    """(L, B) of eq. (discrete_GEP_EH): L = diag(C, C^*), B = i [[zeta, mu], [-eps, -xi]]."""
    C = yee.curl_matrix(grid, kdota, a)
    eps, mu, xi, zeta = (om.block_sparse(t) for t in om.tensors(medium))
    L = sp.bmat([[C, None], [None, C.conj().T]], format="csr")
    B = 1j * sp.bmat([[zeta, mu], [-eps, -xi]], format="csr")
    return L, B


def gep_residual(grid, kdota, medium, omega, x, a=1.0):
    """Relative residual of an eigenpair (omega, x = [E; H]) of eq.
    (discrete_GEP_EH): ||diag(C, C^*) x - omega B x|| / (|omega| ||B x||), with
    the curl C assembled from its finite-difference blocks (eq. (mtx_C))."""
    L, B = gep_matrices(grid, kdota, medium, a)
    x = np.asarray(x, np.complex128).ravel()
    Bx = B @ x
    return float(np.linalg.norm(L @ x - omega * Bx) / (abs(omega) * np.linalg.norm(Bx)))


def hsep_matrix(grid, kdota, medium, a=1.0):
    """The 6n x 6n Hermitian matrix A of eq. (mtx_A) (Theorem
    lem:skew-symm_A): with mu_d = mu_c mu_c^* and Phi = Phi_c Phi_c^* the
    Cholesky factors (eq. (Phi_12)),

        A = -i [[-Phi_c^{-1}(xi mu^{-1} C - C^* mu^{-1} zeta) Phi_c^{-*}, -Phi_c^{-1} C^* mu_c^{-*}],
                [ mu_c^{-1} C Phi_c^{-*},                                   0                    ]],

    whose eigenvalues are those of the GEP (eq. (discrete_GEP_EH)), zeros
    included.  Dense; for tiny grids only."""
    C = yee.curl_matrix(grid, kdota, a).toarray()
    eps, mu, xi, zeta = (om.block_sparse(t).toarray() for t in om.tensors(medium))
    mu_inv = np.linalg.inv(mu)
    phi = eps - xi @ mu_inv @ zeta
    mu_c = np.linalg.cholesky(mu)
    phi_c = np.linalg.cholesky(phi)
    phi_c_inv = np.linalg.inv(phi_c)
    phi_cH_inv = np.linalg.inv(phi_c.conj().T)
    mu_c_inv = np.linalg.inv(mu_c)
    mu_cH_inv = np.linalg.inv(mu_c.conj().T)
    Ch = C.conj().T
    A11 = -phi_c_inv @ (xi @ mu_inv @ C - Ch @ mu_inv @ zeta) @ phi_cH_inv
    A12 = -phi_c_inv @ Ch @ mu_cH_inv
    A21 = mu_c_inv @ C @ phi_cH_inv
    Z = np.zeros_like(A11)
    return -1j * np.block([[A11, A12], [A21, Z]])


def pencil_matrices(grid, kdota, medium, a=1.0):
    """(K'', B'') of the Hermitian-definite pencil described in the module docstring."""
    C = yee.curl_matrix(grid, kdota, a)
    eps, mu, xi, zeta = (om.block_sparse(t) for t in om.tensors(medium))
    K2 = sp.bmat([[None, C.conj().T], [C, None]], format="csr")
    B2 = sp.bmat([[eps, -1j * xi], [1j * zeta, mu]], format="csr")
    return K2, B2


def smallest_positive(omega, nev, zero_tol):
    pos = np.where(omega > zero_tol)[0]
    order = pos[np.argsort(omega[pos])]
    return order[:nev]


def dense_eigs(grid, kdota, medium, nev=None, a=1.0):
    """Tier O1.  All 6n eigenvalues of the pencil (ascending) and B''-orthonormal
    eigenvectors; plus the indices of the ``nev`` smallest positive ones."""
    K2, B2 = pencil_matrices(grid, kdota, medium, a)
    w, z = sla.eigh(K2.toarray(), B2.toarray())
    scale = np.max(np.abs(w))
    idx = smallest_positive(w, nev if nev is not None else len(w), 1e-8 * scale)
    return w, z, idx


def sparse_eigs(grid, kdota, medium, nev, sigma, a=1.0, tol=1e-13):
    """Tier O2.  The eigenvalues of the pencil nearest ``sigma`` by sparse
    shift-and-invert (ARPACK on (K'' - sigma B'')^{-1} B''); returns the ``nev``
    smallest positive ones and their B''-normalised eigenvectors.

    ``sigma`` must exceed half of the largest wanted eigenvalue so that the
    2n-fold zero eigenvalue lies farther from it than every wanted one."""
    K2, B2 = pencil_matrices(grid, kdota, medium, a)
    k = min(2 * nev + 4, K2.shape[0] - 2)
    w, z = spla.eigsh(K2.tocsc(), k=k, M=B2.tocsc(), sigma=sigma, which="LM", tol=tol)
    w = np.real(w)
    scale = max(np.max(np.abs(w)), 1.0)
    idx = smallest_positive(w, nev, 1e-8 * scale)
    zz = z[:, idx]
    # re-normalise so that z^* B'' z = 1
    nrm = np.sqrt(np.real(np.sum(np.conj(zz) * (B2 @ zz), axis=0)))
    return w[idx], zz / nrm


def pencil_gradient(medium, omega, z):
    """Gradient of omega_j with respect to every per-component eps and gamma
    value, from B''-normalised pencil eigenvectors z (columns) of eigenvalues
    omega (entries).

    K'' does not depend on the material, so for an eigenpair of K'' z = w B'' z
    first-order perturbation gives dw = -w z^* (dB'') z / (z^* B'' z).  dB'' has
    one unit entry at (E_cv, E_cv) for eps_cv; for gamma the entries are those
    of -i xi_d and i zeta_d.  Returns (d_eps (3, n3, n2, n1), d_gamma) summed
    over the columns, with d_gamma shaped like ``medium.gamma``."""
    n1, n2, n3 = medium.grid
    n = n1 * n2 * n3
    d_eps = np.zeros((3, n3, n2, n1))
    d_gam = np.zeros_like(medium.gamma, dtype=float)
    eps, mu, xi, zeta = om.tensors(medium)
    for j in range(z.shape[1]):
        zz = z[:, j]
        w = float(omega[j])
        E = zz[:3 * n].reshape(3, n3, n2, n1)
        Hp = zz[3 * n:].reshape(3, n3, n2, n1)
        # z^* B'' z (1 for normalised vectors, kept explicit)
        bzz = (np.sum(np.conj(E) * om.tapply(eps, E)) + np.sum(np.conj(E) * om.tapply(-1j * xi, Hp))
               + np.sum(np.conj(Hp) * om.tapply(1j * zeta, E)) + np.sum(np.conj(Hp) * om.tapply(mu, Hp)))
        bzz = float(np.real(bzz))
        d_eps += -w * np.abs(E) ** 2 / bzz
        if medium.kind == "chiral":
            # d(-i xi)/d gamma = 1 at (E_c, H'_c); d(i zeta)/d gamma = 1 at (H'_c, E_c)
            d_gam += -w * 2.0 * np.real(np.conj(E) * Hp) / bzz
        else:
            a, b = medium.axes
            d_gam += -w * 2.0 * (np.real(np.conj(E[a]) * Hp[b]) + np.real(np.conj(E[b]) * Hp[a])) / bzz
    return d_eps, d_gam
