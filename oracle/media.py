"""Section 4.3: magnetoelectric tensors of chiral and pseudochiral media.

TEST INFRASTRUCTURE (see ``oracle/__init__``).

Each tensor is an array shaped (3, 3, n3, n2, n1): a 3 x 3 block per voxel,
coupling the components of the same voxel index (the paper's block form of
eqs. (chiral_para_mtx) and (pseudo_chiral_para_mtx)).  The 3n x 3n matrix of
the paper is recovered by :func:`block_sparse` with component-major order
(x block, y block, z block), each block in the grid's linear order.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads.media import BIISOTROPIC, CHIRAL, PSEUDOCHIRAL, Medium


def tensors(medium: Medium):
    """Return (eps_d, mu_d, xi_d, zeta_d), each (3, 3, n3, n2, n1) complex."""
    n1, n2, n3 = medium.grid
    shape = (3, 3, n3, n2, n1)
    eps = np.zeros(shape, np.complex128)
    mu = np.zeros(shape, np.complex128)
    xi = np.zeros(shape, np.complex128)
    zeta = np.zeros(shape, np.complex128)
    for c in range(3):
        eps[c, c] = medium.eps[c]
        mu[c, c] = 1.0 if medium.mu is None else medium.mu[c]
    if medium.kind == CHIRAL:
        # eq. (chiral_para_mtx): xi_d = i gamma I~, zeta_d = -i gamma I~
        for c in range(3):
            xi[c, c] = 1j * medium.gamma[c]
            zeta[c, c] = -1j * medium.gamma[c]
    elif medium.kind == BIISOTROPIC:
        # bi-isotropic constitutive relations written in the GEP's blocks:
        # xi_d = (chi + i gamma) I~, zeta_d = (chi - i gamma) I~ per component;
        # chi = 0 is the chiral medium above.  With complex parameters (loss)
        # or chi^2 + gamma^2 >= eps mu the Assumption fails.
        chi = np.zeros_like(medium.gamma) if medium.chi is None else medium.chi
        for c in range(3):
            xi[c, c] = chi[c] + 1j * medium.gamma[c]
            zeta[c, c] = chi[c] - 1j * medium.gamma[c]
    elif medium.kind == PSEUDOCHIRAL:
        # eq. (pseudo_chiral_para_mtx): i gamma I~_n in the two off-diagonal
        # blocks coupling the chosen axis pair (x-z in the paper).
        a, b = medium.axes
        for (r, s) in ((a, b), (b, a)):
            xi[r, s] = 1j * medium.gamma
            zeta[r, s] = -1j * medium.gamma
    else:
        raise ValueError(medium.kind)
    return eps, mu, xi, zeta


def block_sparse(t):
    """3n x 3n sparse matrix of a per-voxel 3 x 3 tensor field."""
    n = t[0, 0].size
    rows, cols, vals = [], [], []
    idx = np.arange(n)
    for r in range(3):
        for s in range(3):
            v = t[r, s].ravel()
            nz = v != 0
            if np.any(nz):
                rows.append(r * n + idx[nz])
                cols.append(s * n + idx[nz])
                vals.append(v[nz])
    if not rows:
        return sp.csr_matrix((3 * n, 3 * n), dtype=np.complex128)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * n, 3 * n))


def batched_inv(t):
    """Per-voxel inverse of a (3, 3, ...) tensor field."""
    m = np.moveaxis(t.reshape(3, 3, -1), -1, 0)
    inv = np.linalg.inv(m)
    # contiguous copy: the per-voxel products below run much faster on it
    return np.ascontiguousarray(np.moveaxis(inv, 0, -1)).reshape(t.shape)


def tmul(a, b):
    """Per-voxel product of two tensor fields."""
    return np.einsum("rk...,ks...->rs...", a, b)


def tapply(t, v):
    """Per-voxel tensor times a 3-component field (3, n3, n2, n1)."""
    return np.einsum("rs...,s...->r...", t, v)


def assumption_holds(medium: Medium):
    """Assumption (eq. (assump)): mu_d > 0, Phi = eps_d - xi_d mu_d^{-1} zeta_d > 0
    and xi_d^* = zeta_d, checked per voxel block."""
    eps, mu, xi, zeta = tensors(medium)
    if not np.allclose(np.conj(np.swapaxes(xi, 0, 1)), zeta):
        return False
    phi = eps - tmul(tmul(xi, batched_inv(mu)), zeta)
    for t in (mu, phi):
        # "mu_d > 0, Phi > 0" are Hermitian positive definite (eq. (assump))
        m = np.moveaxis(t.reshape(3, 3, -1), -1, 0)
        mh = np.conj(np.swapaxes(m, 1, 2))
        if not np.allclose(m, mh):
            return False
        if np.min(np.linalg.eigvalsh(0.5 * (m + mh))) <= 0:
            return False
    return True
