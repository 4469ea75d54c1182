"""Pins of the oracle's Section 2 objects against what the paper and the
mathematics fix: definitions, theorems, closed forms and brute force."""

import numpy as np
import pytest

import workloads as wl
from oracle import yee

GRID = (4, 3, 5)       # ragged, every axis different
K = (0.1, 0.2, 0.3)


@pytest.fixture(scope="module")
def sym():
    return yee.Symbols(GRID, K)


def test_T_unitary_and_fft_form(sym):
    """eq. (mtx_T): T is unitary; the paper applies T q by ifftn and T^* p by
    fftn (Section 5).  Both FFT forms agree with the dense Kronecker product."""
    n = sym.n
    T = yee.T_dense(GRID, K)
    assert np.abs(T.conj().T @ T - np.eye(n)).max() < 1e-13
    q = wl.random_complex((5, 3, 4), 1)
    assert np.abs(yee.apply_T(q, K).ravel() - T @ q.ravel()).max() < 1e-13
    assert np.abs(yee.apply_Tstar(q, K).ravel() - T.conj().T @ q.ravel()).max() < 1e-13


def test_K_eigendecomposition():
    """eq. (eigdecomp_K): K (D U) = (D U) Lambda for a single axis."""
    for m, ka in ((5, 0.3), (6, 0.0), (7, 0.45)):
        K_ = yee.K_matrix(m, ka).toarray()
        DU = np.diag(yee.D_diag(m, ka)) @ yee.U_matrix(m)
        assert np.abs(K_ @ DU - DU @ np.diag(yee.Lambda_1d(m, ka))).max() < 1e-13


def test_theorem_C_l_T(sym):
    """Theorem (thm:SchurDecomp_Ci): C_l T = T Lambda_l for l = 1, 2, 3."""
    T = yee.T_dense(GRID, K)
    for C, L in zip(yee.curl_blocks(GRID, K), (sym.L1, sym.L2, sym.L3)):
        assert np.abs(C @ T - T @ np.diag(L.ravel())).max() < 1e-12


def test_curl_stencil_brute_force():
    """eq. (mtx_C)-(mtx_K_n1) by hand: (C E)_x = dy E_z - dz E_y with
    quasi-periodic forward differences, checked at one voxel of a random field."""
    g = (4, 3, 5)
    n1, n2, n3 = g
    dx, dy, dz = 1 / n1, 1 / n2, 1 / n3
    C = yee.curl_matrix(g, K)
    E = wl.random_complex((3, n3, n2, n1), 7)
    CE = (C @ E.ravel()).reshape(3, n3, n2, n1)

    def fwd(f, axis, ka):
        # f(j+1) - f(j) with f(n) = exp(i 2 pi ka) f(0)
        nxt = np.roll(f, -1, axis=axis)
        sl = [slice(None)] * 3
        sl[axis] = -1
        nxt[tuple(sl)] *= np.exp(2j * np.pi * ka)
        return nxt - f
    d_x = lambda f: fwd(f, 2, K[0]) / dx   # noqa: E731
    d_y = lambda f: fwd(f, 1, K[1]) / dy   # noqa: E731
    d_z = lambda f: fwd(f, 0, K[2]) / dz   # noqa: E731
    ref = np.stack([d_y(E[2]) - d_z(E[1]), d_z(E[0]) - d_x(E[2]), d_x(E[1]) - d_y(E[0])])
    assert np.abs(CE - ref).max() < 1e-12


def test_lemma_positive_and_full_rank(sym):
    """Lemma (lem:nonsingular_full_rank): Lambda_q > 0 and Lambda_p != 0 for
    k != 0 and alpha dx != beta dy, dz != beta dy."""
    assert sym.Lq.min() > 0
    assert sym.Lp2.min() > 1e-6 * sym.Lp2.max()


def test_lemma_conditions_are_needed():
    """The Lemma's hypotheses matter: k = 0 makes Lambda_q singular, and
    alpha dx = beta dy on a cube with k1 = k2 = k3 gives Lambda_p = 0 at the
    diagonal voxels."""
    with np.errstate(divide="ignore", invalid="ignore"):
        s0 = yee.Symbols((4, 4, 4), (0.0, 0.0, 0.0))
        sb = yee.Symbols((4, 4, 4), (0.2, 0.2, 0.2), alpha=1.0, beta=1.0)
    assert s0.Lq.min() < 1e-20
    assert sb.Lp2.min() < 1e-20


def test_null_space(sym):
    """Theorem (Q0, P0): C Q0 = 0, P0^* C = 0; C has rank 2n (the GEP has 2n
    zero eigenvalues, Section 3)."""
    T = yee.T_dense(GRID, K)
    I3T = np.kron(np.eye(3), T)
    stack = lambda Pi: np.vstack([np.diag(Pi[c].ravel()) for c in range(3)])  # noqa: E731
    Q0 = I3T @ stack(sym.Pi0)
    P0 = I3T @ stack(np.conj(sym.Pi0))
    C = yee.curl_matrix(GRID, K).toarray()
    assert np.abs(C @ Q0).max() < 1e-12
    assert np.abs(P0.conj().T @ C).max() < 1e-12
    assert np.linalg.matrix_rank(C, tol=1e-9 * np.abs(C).max()) == 2 * sym.n


def test_Q_P_unitary(sym):
    """Theorem (thm:eigendecomp_A): Q and P are unitary (with the corrected
    Pi_1 normalisation)."""
    Q, P = yee.dense_bases(sym)
    I = np.eye(3 * sym.n)
    assert np.abs(Q.conj().T @ Q - I).max() < 1e-12
    assert np.abs(P.conj().T @ P - I).max() < 1e-12


def test_Pi1_printed_normalisation_is_not_unitary(sym):
    """The second expression of eq. (mtx_Pi_1), taken literally, does not
    normalise Q_1: this is why the oracle divides by sqrt(Lq Lp^* Lp)."""
    Pi1 = yee.Pi1_as_printed(sym)
    norms = np.sum(np.abs(Pi1) ** 2, axis=0)
    assert np.abs(norms - 1).max() > 1.0
    good = np.sum(np.abs(sym.Pi1) ** 2, axis=0)
    assert np.abs(good - 1).max() < 1e-13


def test_Pi1_equals_projection_form(sym):
    """First expression of eq. (mtx_Pi_1): (I - Pi0 Pi0^*) t (Lp^*Lp / Lq)^{-1/2}
    with t = (alpha, beta, 1), computed by projection."""
    t = np.array([sym.alpha, sym.beta, 1.0])[:, None, None, None]
    proj = t - sym.Pi0 * np.sum(np.conj(sym.Pi0) * t, axis=0)
    ref = proj / np.sqrt(sym.Lp2 / sym.Lq)
    assert np.abs(ref - sym.Pi1).max() < 1e-12


def test_svd_reconstruction(sym):
    """SVD theorem (thm:svd_C): C = P_r Sigma_r Q_r^*, and its adjoint
    C^* = Q_r Sigma_r P_r^*."""
    C = yee.curl_matrix(GRID, K).toarray()
    Pr, Sr, Qr = yee.dense_svd_factors(sym)
    assert np.abs(C - Pr @ np.diag(Sr) @ Qr.conj().T).max() < 1e-12 * np.abs(C).max()
    assert np.abs(C.conj().T - Qr @ np.diag(Sr) @ Pr.conj().T).max() < 1e-12 * np.abs(C).max()


def test_singular_values_closed_form(sym):
    """Singular values of C are sqrt(Lambda_q) twice and 0 n times, with
    Lambda_q written out from the discrete plane-wave dispersion
    sum_l 4 sin^2(pi (i_l + k_l) / n_l) / delta_l^2 (independent of the
    oracle's tables)."""
    n1, n2, n3 = GRID
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    lq = (4 * np.sin(np.pi * (i1 + K[0]) / n1) ** 2 * n1 ** 2
          + 4 * np.sin(np.pi * (i2 + K[1]) / n2) ** 2 * n2 ** 2
          + 4 * np.sin(np.pi * (i3 + K[2]) / n3) ** 2 * n3 ** 2).ravel()
    sv = np.linalg.svd(yee.curl_matrix(GRID, K).toarray(), compute_uv=False)
    ref = np.sort(np.concatenate([np.sqrt(lq), np.sqrt(lq), np.zeros(sym.n)]))[::-1]
    assert np.abs(sv - ref).max() < 1e-11
    assert np.abs(sym.Lq.ravel() - lq).max() < 1e-10


def test_cross_product_structure(sym):
    """Lambda_p = t x a with a = (Lambda_1, Lambda_2, Lambda_3) (eq. (mtx_Lambda_p_q));
    C T_1 = -(I3 x T) Lambda_p (proof of the SVD theorem)."""
    T = yee.T_dense(GRID, K)
    I3T = np.kron(np.eye(3), T)
    T1 = np.vstack([sym.alpha * T, sym.beta * T, T])
    C = yee.curl_matrix(GRID, K).toarray()
    stack = lambda Pi: np.vstack([np.diag(Pi[c].ravel()) for c in range(3)])  # noqa: E731
    assert np.abs(C @ T1 + I3T @ stack(sym.Lp)).max() < 1e-10
