"""Pins of the oracle's NFSEP (thm:nfep, eq. NFSEP_org) and of Algorithm 1's
second branch against what the paper and the mathematics fix: M has exactly
the nonzero eigenvalues of the GEP (dense non-Hermitian solve of eq.
discrete_GEP_EH) for lossy, Tellegen and strongly coupled bi-isotropic media;
for a medium under the Assumption they are those of the HHPD-NFGEP; vacuum
gives the closed form +-sqrt(Lambda_q); recovered fields solve the GEP; the
shift-and-invert Arnoldi returns the eigenvalues nearest its shift."""

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import linear_sum_assignment

import workloads as wl
from oracle import gep, media as om, nfgep, nfsep

GRID = (4, 3, 5)
K = (0.1, 0.2, 0.3)


def cases():
    g = GRID
    return {
        # loss: complex eps inside
        "lossy": wl.biisotropic_sphere(g, 0.3, 13.0 + 2.0j, 1.0, 0.5, 0.0),
        # Tellegen coupling with chirality: xi^* = zeta holds for real chi and
        # Phi = eps - (chi^2 + gamma^2) / mu > 0, so this one is Hermitian
        "tellegen": wl.biisotropic_sphere(g, 0.3, 6.0, 1.0, 0.8, 0.9, mu_in=1.5),
        # chi^2 + gamma^2 > eps mu: Phi indefinite, outside the Assumption
        "strong": wl.biisotropic_sphere(g, 0.3, 2.0, 1.0, 1.2, 1.1),
        # complex Tellegen parameter: xi^* != zeta
        "nonreciprocal": wl.biisotropic_sphere(g, 0.3, 9.0, 1.0, 0.3, 0.4 + 0.3j),
    }


def match(a, b):
    """Largest distance of the best one-to-one pairing of two multisets."""
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


@pytest.fixture(scope="module", params=list(cases()))
def case(request):
    med = cases()[request.param]
    nf = nfsep.NFSEP(GRID, K, med)
    M = nf.dense()
    w, V = np.linalg.eig(M)
    return request.param, med, nf, w, V


def test_which_cases_leave_the_assumption(case):
    name, med, *_ = case
    assert om.assumption_holds(med) == (name == "tellegen"), name


def test_nfsep_has_the_nonzero_gep_eigenvalues(case):
    """Theorem (thm:nfep): M and the GEP share their 4n nonzero eigenvalues;
    the GEP's other 2n are zero (Theorem thm:svd_C)."""
    _, med, nf, w, _ = case
    L, B = gep.gep_matrices(GRID, K, med)
    ev = sla.eigvals(L.toarray(), B.toarray())
    scale = np.abs(ev[np.isfinite(ev)]).max()
    nz = np.abs(ev) > 1e-8 * scale
    assert np.sum(~nz) == 2 * nf.n
    assert w.size == 4 * nf.n
    assert match(w, ev[nz]) < 1e-9 * scale


def test_recovered_fields_solve_the_gep(case):
    """Algorithm 1 (else branch): x = B^{-1} diag(P_r, Q_r) Sigma^{1/2} y is an
    eigenvector of the GEP for the same omega."""
    _, med, nf, w, V = case
    order = np.argsort(np.abs(w))[:6]
    for j in order:
        x = nf.fields(V[:, j])
        assert gep.gep_residual(GRID, K, med, w[j], x) < 1e-10


def test_shift_invert_arnoldi_nearest(case):
    _, med, nf, w, _ = case
    sigma = 0.6 * np.sort(np.abs(w))[8] * (1 + 0.1j)
    om_, Y = nf.eigs_near(sigma, 4)
    ref = w[np.argsort(np.abs(w - sigma))[:4]]
    assert match(om_, ref) < 1e-9 * np.abs(ref).max()
    for j in range(4):
        r = nf.apply(Y[:, j]) - om_[j] * Y[:, j]
        assert np.linalg.norm(r) < 1e-9 * abs(om_[j]) * np.linalg.norm(Y[:, j])


def test_hermitian_medium_reduces_to_hhpd_nfgep():
    """Under the Assumption (chiral medium) M's eigenvalues are real and are
    those of B_r y = omega^{-1} A_r y (thm:NFSEP_real_ew)."""
    med = wl.chiral_sphere(GRID, 0.3, 13.0, 1.0, 0.5)
    w = np.linalg.eigvals(nfsep.NFSEP(GRID, K, med).dense())
    nh = nfgep.NFGEP(GRID, K, med)
    th = sla.eigh(nh.dense_Br(), nh.dense_Ar(), eigvals_only=True)
    assert np.abs(w.imag).max() < 1e-9 * np.abs(w).max()
    assert np.abs(np.sort(w.real) - np.sort(1.0 / th)).max() < 1e-9 * np.abs(w).max()


def test_vacuum_closed_form():
    """eps = mu = 1, no coupling: omega = +-sqrt(Lambda_q), each twice (the two
    transverse polarisations), written out from the plane-wave dispersion."""
    g = (4, 3, 5)
    med = wl.biisotropic_sphere(g, 0.3, 1.0, 1.0, 0.0, 0.0)
    w = np.linalg.eigvals(nfsep.NFSEP(g, K, med).dense())
    n1, n2, n3 = g
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    disp = np.sqrt(4 * np.sin(np.pi * (i1 + K[0]) / n1) ** 2 * n1 ** 2
                   + 4 * np.sin(np.pi * (i2 + K[1]) / n2) ** 2 * n2 ** 2
                   + 4 * np.sin(np.pi * (i3 + K[2]) / n3) ** 2 * n3 ** 2).ravel()
    ref = np.concatenate([disp, disp, -disp, -disp])
    assert match(w, ref) < 1e-10 * disp.max()


def test_both_branches_of_algorithm_1_give_the_same_fields():
    """Inside the Assumption both branches of Algorithm 1 apply: the fields
    B^{-1} diag(P_r, Q_r) y_r of an HHPD-NFGEP eigenvector and B^{-1}
    diag(P_r, Q_r) Sigma^{1/2} y of the NFSEP eigenvector of the same simple
    eigenvalue are parallel."""
    med = wl.chiral_sphere(GRID, 0.3, 13.0, 1.0, 0.5)
    nh = nfgep.NFGEP(GRID, K, med)
    th, Yr = sla.eigh(nh.dense_Br(), nh.dense_Ar())
    ns = nfsep.NFSEP(GRID, K, med)
    w, V = np.linalg.eig(ns.dense())
    om = 1.0 / th
    checked = 0
    for j in np.argsort(np.abs(om))[:10]:
        gaps = np.abs(om - om[j])
        if np.sort(gaps)[1] < 1e-6 * abs(om[j]):
            continue  # degenerate: no unique direction
        i = int(np.argmin(np.abs(w - om[j])))
        assert abs(w[i] - om[j]) < 1e-9 * abs(om[j])
        x1 = nh.eigvec_fields(Yr[:, j]).ravel()
        x2 = ns.fields(V[:, i]).ravel()
        cos = abs(np.vdot(x1, x2)) / (np.linalg.norm(x1) * np.linalg.norm(x2))
        assert cos > 1 - 1e-9
        checked += 1
    assert checked >= 4


def test_invariant_subspace_identity(case):
    """Theorem (thm:nonzero_invariant_subsp), eq. (pf_invariant_1): with
    W = B^{-1} diag(P_r Sigma^{1/2}, Q_r Sigma^{1/2}) (6n x 4n, the NFSEP's
    field map applied to the unit vectors), diag(C, C^*) W = B W M: the span
    of W is invariant under the GEP and M is the GEP restricted to it."""
    _, med, nf, _, _ = case
    N = 4 * nf.n
    W = np.stack([nf.fields(np.eye(N)[:, j]).ravel() for j in range(N)], axis=1)
    L, B = gep.gep_matrices(GRID, K, med)
    M = nf.dense()
    lhs = L @ W
    rhs = B @ (W @ M)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()


def test_tellegen_coupling_breaks_reciprocity():
    """A Tellegen parameter (chi != 0) makes the medium non-reciprocal: the
    spectra at k and -k differ; with chi = 0 (the chiral medium) they agree,
    as the reciprocity pin of the Hermitian branch requires."""
    kneg = tuple(-x for x in K)
    tel = wl.biisotropic_sphere(GRID, 0.3, 6.0, 1.0, 0.8, 0.9, mu_in=1.5)
    chi0 = wl.biisotropic_sphere(GRID, 0.3, 6.0, 1.0, 0.8, 0.0)

    def spectrum(k, med):
        return np.sort(np.linalg.eigvals(nfsep.NFSEP(GRID, k, med).dense()).real)
    assert np.abs(spectrum(K, tel) - spectrum(kneg, tel)).max() > 1e-2
    assert np.abs(spectrum(K, chi0) - spectrum(kneg, chi0)).max() < 1e-10 * np.abs(spectrum(K, chi0)).max()
