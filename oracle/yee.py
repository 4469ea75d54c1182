"""Section 2: the discrete single-curl operator and its explicit SVD.

TEST INFRASTRUCTURE (see ``oracle/__init__``).  Dense / sparse FP64, CPU only.

Index convention: a field on the grid is an array shaped (n3, n2, n1); its
flattening (C order) is the paper's linear index (k-1) n1 n2 + (j-1) n1 + i
(appendix, part (b)), x fastest.  A 3n-vector stacks the x, y, z components.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DEFAULT_ALPHA = 2.0
DEFAULT_BETA = 3.0


def mesh_lengths(grid, a=1.0):
    """delta_x, delta_y, delta_z = a / n_l (the paper leaves delta_l unstated)."""
    n1, n2, n3 = grid
    return a / n1, a / n2, a / n3


# ---------------------------------------------------------------------------
# eq. (mtx_K_n1): the quasi-periodic forward-difference matrix K_{a,m}
# ---------------------------------------------------------------------------

def K_matrix(m, kdota):
    """K_{a,m}: -1 on the diagonal, +1 on the super-diagonal and the Bloch
    phase exp(i 2 pi k.a) in the bottom-left corner (eq. (mtx_K_n1))."""
    K = sp.lil_matrix((m, m), dtype=np.complex128)
    for r in range(m):
        K[r, r] = -1.0
        if r + 1 < m:
            K[r, r + 1] = 1.0
    K[m - 1, 0] += np.exp(2j * np.pi * kdota)
    return K.tocsr()


def curl_blocks(grid, kdota, a=1.0):
    """C_1, C_2, C_3 of eq. (mtx_C123) (sparse n x n)."""
    n1, n2, n3 = grid
    dx, dy, dz = mesh_lengths(grid, a)
    I1, I2, I3 = (sp.identity(m, dtype=np.complex128, format="csr") for m in (n1, n2, n3))
    C1 = sp.kron(I3, sp.kron(I2, K_matrix(n1, kdota[0]))) / dx
    C2 = sp.kron(I3, sp.kron(K_matrix(n2, kdota[1]), I1)) / dy
    C3 = sp.kron(K_matrix(n3, kdota[2]), sp.kron(I2, I1)) / dz
    return C1.tocsr(), C2.tocsr(), C3.tocsr()


def curl_matrix(grid, kdota, a=1.0):
    """C of eq. (mtx_C): [[0, -C3, C2], [C3, 0, -C1], [-C2, C1, 0]] (sparse 3n x 3n)."""
    C1, C2, C3 = curl_blocks(grid, kdota, a)
    return sp.bmat([[None, -C3, C2], [C3, None, -C1], [-C2, C1, None]], format="csr")


# ---------------------------------------------------------------------------
# eqs. (mtx_Dm), (mtx_Um), (mtx_T): D_{a,m}, U_m, Lambda_{a,m} and T
# ---------------------------------------------------------------------------

def D_diag(m, kdota):
    """Diagonal of D_{a,m} = diag(1, e^{theta_a}, ..., e^{(m-1) theta_a}),
    theta_{a,m} = i 2 pi k.a / m."""
    return np.exp(2j * np.pi * kdota * np.arange(m) / m)


def U_matrix(m):
    """U_m = [u_{m,0} ... u_{m,m-1}], (u_{m,i})_j = exp(i 2 pi i j / m)."""
    j = np.arange(m)
    return np.exp(2j * np.pi * np.outer(j, j) / m)


def Lambda_1d(m, kdota):
    """Diagonal of Lambda_{a,m}: exp(theta_{m,i} + theta_{a,m}) - 1."""
    return np.exp(2j * np.pi * (np.arange(m) + kdota) / m) - 1.0


def T_dense(grid, kdota):
    """T = n^{-1/2} (D3 x D2 x D1)(U3 x U2 x U1) (eq. (mtx_T)), dense n x n."""
    n1, n2, n3 = grid
    D = np.kron(np.diag(D_diag(n3, kdota[2])),
                np.kron(np.diag(D_diag(n2, kdota[1])), np.diag(D_diag(n1, kdota[0]))))
    U = np.kron(U_matrix(n3), np.kron(U_matrix(n2), U_matrix(n1)))
    return D @ U / np.sqrt(n1 * n2 * n3)


def _D_grid(grid, kdota):
    n1, n2, n3 = grid
    return (D_diag(n3, kdota[2])[:, None, None] * D_diag(n2, kdota[1])[None, :, None]
            * D_diag(n1, kdota[0])[None, None, :])


def apply_T(q, kdota):
    """T q for q shaped (n3, n2, n1): the paper applies T with MATLAB ifftn
    (Section 5, implementation paragraph): T q = sqrt(n) * D * ifftn(q)."""
    n3, n2, n1 = q.shape
    n = n1 * n2 * n3
    return np.sqrt(n) * _D_grid((n1, n2, n3), kdota) * np.fft.ifftn(q)


def apply_Tstar(p, kdota):
    """T^* p = fftn(conj(D) * p) / sqrt(n) (Section 5: fftn applies T^*)."""
    n3, n2, n1 = p.shape
    n = n1 * n2 * n3
    return np.fft.fftn(np.conj(_D_grid((n1, n2, n3), kdota)) * p) / np.sqrt(n)


# ---------------------------------------------------------------------------
# Theorem (thm:SchurDecomp_Ci), the Lemma (eq. (mtx_Lambda_p_q)), Pi_0
# (eq. (mtx_Q0)), Pi_1 (eq. (mtx_Pi_1)), Pi_2 (eq. (mtx_Pi_2))
# ---------------------------------------------------------------------------

class Symbols:
    """Per-voxel diagonal symbols, each an array shaped (n3, n2, n1) in
    spectral index order (i3, i2, i1)."""

    def __init__(self, grid, kdota, alpha=DEFAULT_ALPHA, beta=DEFAULT_BETA, a=1.0):
        n1, n2, n3 = grid
        dx, dy, dz = mesh_lengths(grid, a)
        self.grid = tuple(grid)
        self.kdota = tuple(kdota)
        self.alpha, self.beta = float(alpha), float(beta)
        # thm:SchurDecomp_Ci: Lambda_1 = dx^{-1} (I x I x Lambda_{a1,n1}), etc.
        L1 = (Lambda_1d(n1, kdota[0]) / dx)[None, None, :]
        L2 = (Lambda_1d(n2, kdota[1]) / dy)[None, :, None]
        L3 = (Lambda_1d(n3, kdota[2]) / dz)[:, None, None]
        shape = (n3, n2, n1)
        self.L1 = np.broadcast_to(L1, shape).copy()
        self.L2 = np.broadcast_to(L2, shape).copy()
        self.L3 = np.broadcast_to(L3, shape).copy()
        L1, L2, L3 = self.L1, self.L2, self.L3
        al, be = self.alpha, self.beta
        # eq. (mtx_Lambda_p_q)
        self.Lq = (np.conj(L1) * L1 + np.conj(L2) * L2 + np.conj(L3) * L3).real
        self.Lp = np.stack([be * L3 - L2, L1 - al * L3, al * L2 - be * L1])
        self.Lp2 = np.sum(np.abs(self.Lp) ** 2, axis=0)       # Lambda_p^* Lambda_p
        # eq. (mtx_Q0)
        self.Pi0 = np.stack([L1, L2, L3]) / np.sqrt(self.Lq)
        # eq. (mtx_Pi_1): the printed vector, normalised by (Lambda_q Lambda_p^* Lambda_p)^{-1/2}
        p1, p2, p3 = self.Lp
        v = np.stack([
            p3 * np.conj(L2) - p2 * np.conj(L3),
            p1 * np.conj(L3) - p3 * np.conj(L1),
            p2 * np.conj(L1) - p1 * np.conj(L2),
        ])
        self.Pi1 = v / np.sqrt(self.Lq * self.Lp2)
        # eq. (mtx_Pi_2)
        self.Pi2 = np.conj(self.Lp) / np.sqrt(self.Lp2)
        self.sigma = np.sqrt(self.Lq)                          # Sigma_r diagonal (per block)

    @property
    def n(self):
        n1, n2, n3 = self.grid
        return n1 * n2 * n3


def Pi1_as_printed(sym: Symbols):
    """Pi_1 with the normalisation exactly as printed in the second line of
    eq. (mtx_Pi_1), (Lambda_p^* Lambda_p Lambda_q^{-1})^{-1/2}.  Kept only so a test
    can show that this reading does not give a unitary Q."""
    return sym.Pi1 * np.sqrt(sym.Lq * sym.Lp2) / np.sqrt(sym.Lp2 / sym.Lq)


# ---------------------------------------------------------------------------
# Dense Q, P (eq. (mtx_QdPd)) and the SVD factors (thm:svd_C) -- small grids only
# ---------------------------------------------------------------------------

def _stack_diag(Pi):
    """3n x n matrix with diag(Pi_x), diag(Pi_y), diag(Pi_z) stacked."""
    return np.vstack([np.diag(Pi[c].ravel()) for c in range(3)])


def dense_bases(sym: Symbols):
    """Dense Q = (I3 x T)[Pi1, Pi2, Pi0] and P = (I3 x T)[-conj Pi2, conj Pi1, conj Pi0]."""
    T = T_dense(sym.grid, sym.kdota)
    I3T = np.kron(np.eye(3), T)
    Q = I3T @ np.hstack([_stack_diag(sym.Pi1), _stack_diag(sym.Pi2), _stack_diag(sym.Pi0)])
    P = I3T @ np.hstack([_stack_diag(-np.conj(sym.Pi2)), _stack_diag(np.conj(sym.Pi1)),
                         _stack_diag(np.conj(sym.Pi0))])
    return Q, P


def dense_svd_factors(sym: Symbols):
    """P_r = [P2, P1], Q_r = [Q1, Q2], Sigma_r = diag(Lq^{1/2}, Lq^{1/2})."""
    Q, P = dense_bases(sym)
    n = sym.n
    Qr = Q[:, :2 * n]
    Pr = P[:, :2 * n]
    s = np.sqrt(sym.Lq.ravel())
    Sr = np.concatenate([s, s])
    return Pr, Sr, Qr


# ---------------------------------------------------------------------------
# FFT application of P_r, Q_r and their adjoints (Section 4.2)
# ---------------------------------------------------------------------------

def apply_Pr(sym: Symbols, u1a, u1b):
    """P_r [u1a; u1b] = (I3 x T)(-conj(Pi2) u1a + conj(Pi1) u1b): 3 real-space components."""
    return np.stack([apply_T(-np.conj(sym.Pi2[c]) * u1a + np.conj(sym.Pi1[c]) * u1b, sym.kdota)
                     for c in range(3)])


def apply_Qr(sym: Symbols, u2a, u2b):
    """Q_r [u2a; u2b] = (I3 x T)(Pi1 u2a + Pi2 u2b)."""
    return np.stack([apply_T(sym.Pi1[c] * u2a + sym.Pi2[c] * u2b, sym.kdota) for c in range(3)])


def apply_PrH(sym: Symbols, f):
    """P_r^* f = [(-conj Pi2)^* fhat; (conj Pi1)^* fhat], fhat = (I3 x T^*) f."""
    fh = np.stack([apply_Tstar(f[c], sym.kdota) for c in range(3)])
    return (-np.sum(sym.Pi2 * fh, axis=0), np.sum(sym.Pi1 * fh, axis=0))


def apply_QrH(sym: Symbols, w):
    """Q_r^* w = [Pi1^* what; Pi2^* what]."""
    wh = np.stack([apply_Tstar(w[c], sym.kdota) for c in range(3)])
    return (np.sum(np.conj(sym.Pi1) * wh, axis=0), np.sum(np.conj(sym.Pi2) * wh, axis=0))
