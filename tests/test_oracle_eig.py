"""Pins of the oracle's eigenproblem tiers (Sections 3-5) against what the
paper and the mathematics fix."""

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import gep, media as om, nfgep, yee

GRID = (4, 3, 5)
K = (0.1, 0.2, 0.3)


def media_cases():
    g = GRID
    return {
        "chiral_sphere": wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.5),
        "pseudochiral_xz": wl.pseudochiral_cylinders(g, 2, 0.2, 13.0, 1.0, 0.6, (0, 2), seed=3),
        "smoothed_field": wl.smoothed_chiral_field(g, seed=5, sigma=0.2),
    }


@pytest.fixture(scope="module", params=list(media_cases()))
def case(request):
    med = media_cases()[request.param]
    w, z, idx = gep.dense_eigs(GRID, K, med)
    return request.param, med, w, z, idx


def test_assumption_holds(case):
    """Assumption (eq. (assump)) holds for chiral / pseudochiral media with
    gamma^2 < eps (Section 4.3)."""
    _, med, *_ = case
    assert om.assumption_holds(med)


def test_gep_has_2n_zeros_and_matches_pencil(case):
    """Section 3: the GEP (eq. (discrete_GEP_EH)) has 2n zero eigenvalues; the
    nonzero ones are real under the Assumption (thm:skew-symm_A) and equal
    those of the Hermitian pencil the oracle solves."""
    _, med, w, _, idx = case
    n = np.prod(GRID)
    L, B = gep.gep_matrices(GRID, K, med)
    ev = sla.eigvals(L.toarray(), B.toarray())
    assert np.all(np.isfinite(ev))
    scale = np.abs(ev).max()
    nz = np.abs(ev) > 1e-9 * scale
    assert np.sum(~nz) == 2 * n
    assert np.abs(ev[nz].imag).max() < 1e-9 * scale
    assert np.sum(np.abs(w) < 1e-9 * np.abs(w).max()) == 2 * n
    gep_sorted = np.sort(ev[nz].real)
    pen_sorted = np.sort(w[np.abs(w) > 1e-9 * np.abs(w).max()])
    assert np.abs(gep_sorted - pen_sorted).max() < 1e-9 * scale


def test_nfgep_dense_matches_pencil(case):
    """Theorems (thm:nfep), (thm:NFSEP_real_ew): the 4n x 4n HHPD-NFGEP has
    exactly the 4n nonzero GEP eigenvalues; A_r is Hermitian positive definite
    and B_r Hermitian."""
    _, med, w, _, _ = case
    nf = nfgep.NFGEP(GRID, K, med)
    A = nf.dense_Ar()
    B = nf.dense_Br()
    assert np.abs(A - A.conj().T).max() < 1e-12 * np.abs(A).max()
    assert np.abs(B - B.conj().T).max() == 0
    assert np.linalg.eigvalsh(A).min() > 0
    th = sla.eigh(B, A, eigvals_only=True)
    om_ = np.sort(1.0 / th)
    nz = np.sort(w[np.abs(w) > 1e-9 * np.abs(w).max()])
    assert om_.size == nz.size
    assert np.abs(om_ - nz).max() < 1e-10 * np.abs(nz).max()


def test_fft_matvec_equals_dense(case):
    """Section 4.2: A_r applied with FFTs equals the dense eq. (factor_mtx)."""
    _, med, *_ = case
    nf = nfgep.NFGEP(GRID, K, med)
    u = wl.random_complex(4 * nf.n, 11)
    Au = nf.dense_Ar() @ u
    assert np.abs(nf.Ar(u) - Au).max() < 1e-13 * np.abs(Au).max()
    assert np.abs(nf.Br(u) - nf.dense_Br() @ u).max() < 1e-14 * np.abs(u).max() * 10


def test_arpack_invert_lanczos_equals_dense(case):
    """Tier O3 (CG inside ARPACK invert Lanczos) reaches the brute-force
    eigenvalues; residual ||A_r y - omega B_r y|| / ||y|| is tiny."""
    _, med, w, _, idx = case
    nf = nfgep.NFGEP(GRID, K, med)
    omega, Y = nf.eigs(6)
    assert np.abs(omega - w[idx[:6]]).max() < 1e-10 * w[idx[5]]
    for j in range(6):
        assert nf.residual(omega[j], Y[:, j]) < 1e-9 * omega[j]


def test_cg_solves(case):
    _, med, *_ = case
    nf = nfgep.NFGEP(GRID, K, med)
    b = wl.random_complex(4 * nf.n, 2)
    x, it = nf.cg(b, tol=1e-12)
    assert np.linalg.norm(nf.Ar(x) - b) <= 1e-11 * np.linalg.norm(b)
    assert 0 < it < 4 * nf.n


def test_homogeneous_closed_form():
    """Section 5.1 (second validation): for (eps_i, eps_o, gamma) = (1, 1, 0)
    the eigenvalues are sqrt(Lambda_q), each twice; with eps = 4 they halve.
    The reference values are the discrete plane-wave dispersion written out."""
    g = (6, 4, 5)
    k = (0.25, 0.1, 0.4)
    n1, n2, n3 = g
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    disp = np.sqrt(4 * np.sin(np.pi * (i1 + k[0]) / n1) ** 2 * n1 ** 2
                   + 4 * np.sin(np.pi * (i2 + k[1]) / n2) ** 2 * n2 ** 2
                   + 4 * np.sin(np.pi * (i3 + k[2]) / n3) ** 2 * n3 ** 2).ravel()
    ref = np.sort(np.concatenate([disp, disp]))
    for eps, scale in ((1.0, 1.0), (4.0, 0.5)):
        w, _, idx = gep.dense_eigs(g, k, wl.homogeneous(g, eps=eps))
        pos = np.sort(w[idx])
        assert pos.size == ref.size
        assert np.abs(pos - scale * ref).max() < 1e-12 * ref.max()
        nf = nfgep.NFGEP(g, k, wl.homogeneous(g, eps=eps))
        omega, _ = nf.eigs(8)
        assert np.abs(omega - scale * ref[:8]).max() / (scale * ref[:8]).min() < 1e-11


def test_gamma_zero_is_photonic_crystal():
    """Section 5.1 (first validation): with gamma = 0 and mu = 1 the GEP and
    A E = omega^2 eps_d E (A = C^* C) have the same band structure."""
    g = GRID
    med = wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.0)
    w, _, idx = gep.dense_eigs(g, K, med)
    C = yee.curl_matrix(g, K).toarray()
    eps = np.diag(med.eps.reshape(-1))
    lam = sla.eigh(C.conj().T @ C, eps, eigvals_only=True)
    lam = np.sort(lam[lam > 1e-9 * lam.max()])
    assert lam.size == idx.size
    assert np.abs(np.sqrt(lam) - np.sort(w[idx])).max() < 1e-10 * np.sqrt(lam.max())


def test_alpha_beta_invariance():
    """Section 2, closing remark: P and Q are not unique; the eigenvalues do
    not depend on the free parameters alpha, beta."""
    med = wl.chiral_sphere(GRID, 0.3, 13.0, 1.0, 0.5)
    th1 = sla.eigh(nfgep.NFGEP(GRID, K, med).dense_Br(), nfgep.NFGEP(GRID, K, med).dense_Ar(),
                   eigvals_only=True)
    nf2 = nfgep.NFGEP(GRID, K, med, alpha=-1.5, beta=0.7)
    th2 = sla.eigh(nf2.dense_Br(), nf2.dense_Ar(), eigvals_only=True)
    assert np.abs(np.sort(th1) - np.sort(th2)).max() < 1e-12 * np.abs(th1).max()


def test_sparse_shift_invert_equals_dense():
    """Tier O2 (sparse shift-invert on the pencil) reaches the dense eigenvalues."""
    med = wl.smoothed_chiral_field((6, 6, 6), seed=2, sigma=0.15)
    w, _, idx = gep.dense_eigs((6, 6, 6), K, med)
    wanted = w[idx[:6]]
    om2, _ = gep.sparse_eigs((6, 6, 6), K, med, 6, sigma=0.6 * wanted[-1])
    assert np.abs(om2 - wanted).max() < 1e-10 * wanted[-1]


def test_pencil_gradient_matches_finite_differences():
    """First-order perturbation of the pencil eigenvalue against central
    differences of brute-force eigenvalues (a random field keeps every
    eigenvalue simple)."""
    g = GRID
    med = wl.smoothed_chiral_field(g, seed=9, sigma=0.2)
    w, z, idx = gep.dense_eigs(g, K, med)
    j = idx[0]
    d_eps, d_gam = gep.pencil_gradient(med, w[[j]], z[:, [j]])
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(4):
        c, v3, v2, v1 = rng.integers(0, 3), rng.integers(0, 5), rng.integers(0, 3), rng.integers(0, 4)
        for which in ("eps", "gamma"):
            vals = []
            for s in (+1, -1):
                m = wl.Medium(med.grid, med.kind, med.eps.copy(), med.gamma.copy())
                arr = m.eps if which == "eps" else m.gamma
                arr[c, v3, v2, v1] += s * h
                ww, _, ii = gep.dense_eigs(g, K, m)
                vals.append(ww[ii[0]])
            fd = (vals[0] - vals[1]) / (2 * h)
            an = (d_eps if which == "eps" else d_gam)[c, v3, v2, v1]
            assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3), (which, fd, an)


def test_bz_path_avoids_gamma():
    ks = wl.bz_path_midpoints(48)
    assert ks.shape == (48, 3)
    assert np.all(np.any(np.abs(ks - np.round(ks)) > 1e-6, axis=1))


def test_hsep_matrix_is_hermitian_with_the_gep_spectrum(case):
    """Theorem (lem:skew-symm_A): under the Assumption the Cholesky-scaled A
    of eq. (mtx_A) is Hermitian and has all 6n eigenvalues of the GEP (the 2n
    zeros included), so the GEP's eigenvalues are real."""
    _, med, w, _, _ = case
    A = gep.hsep_matrix(GRID, K, med)
    assert np.abs(A - A.conj().T).max() < 1e-12 * np.abs(A).max()
    lam = np.linalg.eigvalsh(A)
    assert np.abs(np.sort(lam) - np.sort(w)).max() < 1e-9 * np.abs(w).max()


def test_hsep_matrix_with_mu():
    g = GRID
    med = wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.5)
    rng = np.random.default_rng(11)
    med = wl.Medium(g, med.kind, med.eps, med.gamma, 1.0 + rng.random(med.eps.shape), med.axes)
    A = gep.hsep_matrix(g, K, med)
    assert np.abs(A - A.conj().T).max() < 1e-12 * np.abs(A).max()
    w, _, _ = gep.dense_eigs(g, K, med)
    assert np.abs(np.sort(np.linalg.eigvalsh(A)) - np.sort(w)).max() < 1e-9 * np.abs(w).max()


def test_gamma_sweep_conditioning():
    """Section 5.3 (the gamma sweep): as gamma grows towards sqrt(eps_i) the
    material factor Phi = eps - gamma^2 approaches singularity, so the
    condition number of A_r and the CG iterations per solve grow (the paper's
    pcg counts rise from 39 to 90 at 128^3 for gamma 0.25 -> 3); here both
    grow monotonically at 4 x 3 x 5."""
    conds, its = [], []
    for gam in (0.25, 1.0, 2.0, 3.0, 3.5):
        med = wl.chiral_sphere(GRID, 0.3, 13.0, 1.0, gam)
        nf = nfgep.NFGEP(GRID, (0.5, 0.1, 0.2), med)
        ev = np.linalg.eigvalsh(nf.dense_Ar())
        conds.append(ev.max() / ev.min())
        its.append(nf.cg(wl.random_complex(4 * nf.n, 5), tol=1e-10)[1])
    assert all(b > a for a, b in zip(conds, conds[1:])), conds
    assert all(b > a for a, b in zip(its, its[1:])), its
    assert conds[-1] > 10 * conds[0]


def test_bloch_periodicity_and_reciprocity(case):
    """Bloch periodicity: the phase exp(i 2 pi k.a_l) (eq. quasi_periodic)
    depends on k.a_l modulo 1, so shifting one component by an integer leaves
    the spectrum unchanged.  Reciprocity: chiral and pseudochiral media with
    xi^* = zeta and real parameters are reciprocal and lossless, so the
    spectrum at -k equals the one at k."""
    _, med, w, _, _ = case
    scale = np.abs(w).max()
    for shift in ((1.0, 0.0, 0.0), (0.0, -2.0, 1.0)):
        ks = tuple(a + b for a, b in zip(K, shift))
        w2, _, _ = gep.dense_eigs(GRID, ks, med)
        assert np.abs(np.sort(w2) - np.sort(w)).max() < 1e-10 * scale
    wneg, _, _ = gep.dense_eigs(GRID, tuple(-a for a in K), med)
    assert np.abs(np.sort(wneg) - np.sort(w)).max() < 1e-10 * scale
