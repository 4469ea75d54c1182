"""Pins of the oracle's eigenvector recovery (Algorithm 1, final step) and of
its GEP residual against what the mathematics fixes: recovered fields of exact
NFGEP eigenpairs solve the original GEP (eq. (discrete_GEP_EH)) built from the
finite-difference curl, they are the eigenvectors of the Hermitian pencil, and
the residual of an eigenpair with a perturbed eigenvalue has a closed form."""

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import gep, nfgep

GRID = (4, 3, 5)
K = (0.1, 0.2, 0.3)


def media_cases():
    g = GRID
    with_mu = wl.smoothed_chiral_field(g, seed=7, sigma=0.2)
    rng = np.random.default_rng(8)
    with_mu.mu = 1.0 + rng.random((3,) + with_mu.eps.shape[1:])
    return {
        "chiral_sphere": wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.5),
        "pseudochiral_xz": wl.pseudochiral_cylinders(g, 2, 0.2, 13.0, 1.0, 0.6, (0, 2), seed=3),
        "smoothed_field_mu": with_mu,
    }


@pytest.fixture(scope="module", params=list(media_cases()))
def case(request):
    med = media_cases()[request.param]
    nf = nfgep.NFGEP(GRID, K, med)
    # exact eigenpairs of the HHPD-NFGEP B_r y = theta A_r y, largest theta first
    th, Y = sla.eigh(nf.dense_Br(), nf.dense_Ar())
    order = np.argsort(-th)[:8]
    return request.param, med, nf, 1.0 / th[order], Y[:, order]


def test_fields_solve_the_gep(case):
    """(omega, B^{-1} diag(P_r, Q_r) y) is an eigenpair of the 6n GEP: the FFT
    factors, the Bloch twist of T and the B^{-1} solve are checked against the
    Yee curl C assembled from its difference blocks."""
    _, med, nf, omega, Y = case
    for j in range(omega.size):
        x = nf.eigvec_fields(Y[:, j])
        assert x.shape == (6,) + nf.shape
        assert gep.gep_residual(GRID, K, med, omega[j], x) < 1e-11


def test_fields_are_pencil_eigenvectors(case):
    """For a simple eigenvalue the recovered x = [E; H] is parallel to the
    pencil eigenvector [E; H'] with H' = i H (module docstring of oracle.gep)."""
    _, med, nf, omega, Y = case
    w, z, idx = gep.dense_eigs(GRID, K, med)
    n = nf.n
    wp = w[idx]
    checked = 0
    for j in range(omega.size):
        gaps = np.abs(wp - omega[j])
        m = int(np.argmin(gaps))
        assert gaps[m] < 1e-10 * omega[j]
        if np.sort(gaps)[1] < 1e-6 * omega[j]:
            continue  # degenerate: the eigenvector is not unique
        zz = z[:, idx[m]]
        xp = np.concatenate([zz[:3 * n], -1j * zz[3 * n:]])
        x = nf.eigvec_fields(Y[:, j]).ravel()
        cos = abs(np.vdot(xp, x)) / (np.linalg.norm(xp) * np.linalg.norm(x))
        assert cos > 1 - 1e-10
        checked += 1
    assert checked >= 3


def test_gep_residual_closed_form(case):
    """L x = omega B x gives, for omega' = omega (1 + d), the residual
    ||(omega - omega') B x|| / (|omega'| ||B x||) = d / (1 + d) exactly."""
    _, med, nf, omega, Y = case
    x = nf.eigvec_fields(Y[:, 0])
    assert gep.gep_residual(GRID, K, med, omega[0], x) < 1e-11
    for d in (1e-3, 0.25):
        r = gep.gep_residual(GRID, K, med, omega[0] * (1 + d), x)
        assert abs(r - d / (1 + d)) < 1e-9 * d
    # scale-free in x
    assert abs(gep.gep_residual(GRID, K, med, omega[0] * 1.25, (2 - 3j) * x) - 0.2) < 1e-10


def test_block_factorisation_of_B_inverse(case):
    """Eq. (B_inv): B^{-1} = -i [[I, 0], [-mu^{-1} zeta, I]] [[-Phi^{-1} xi mu^{-1},
    -Phi^{-1}], [mu^{-1}, 0]] (the form the device fields kernel uses through
    B^{-1}[p; q] = [i w; -i f]) equals the inverse of B (eq. mtx_B) computed
    by LAPACK."""
    _, med, nf, _, _ = case
    from oracle import media as om
    eps, mu, xi, zeta = (om.block_sparse(t).toarray() for t in om.tensors(med))
    L, B = gep.gep_matrices(GRID, K, med)
    n3 = eps.shape[0]
    I = np.eye(n3)
    Z = np.zeros_like(I)
    mu_inv = np.linalg.inv(mu)
    phi_inv = np.linalg.inv(eps - xi @ mu_inv @ zeta)
    Binv = -1j * np.block([[I, Z], [-mu_inv @ zeta, I]]) @ np.block([[-phi_inv @ xi @ mu_inv, -phi_inv],
                                                                     [mu_inv, Z]])
    ref = np.linalg.inv(B.toarray())
    assert np.abs(Binv - ref).max() < 1e-12 * np.abs(ref).max()
    # and the fields route: B^{-1}[p; q] = [i w; -i f] with (f, w) the middle factors of A_r
    y = wl.random_complex(4 * nf.n, 9)
    p, q = nf.fields(y)
    f, w = nf.middle(p, q)
    x = nf.eigvec_fields(y)
    assert np.abs(x[:3] - 1j * w).max() < 1e-12 * np.abs(x).max()
    assert np.abs(x[3:] + 1j * f).max() < 1e-12 * np.abs(x).max()
