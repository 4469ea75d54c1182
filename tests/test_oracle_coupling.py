"""Pins of the oracle's magnetoelectric coupling (Section 4.3) that depend on
the size and sign of gamma, not only on eps.

1. Homogeneous chiral and pseudochiral media: the twisted DFT basis T
   diagonalises every difference block (C_l T = T Lambda_l,
   thm:SchurDecomp_Ci) and a homogeneous material commutes with I_3 (x) T, so
   the 6n x 6n pencil of the GEP splits into one 6 x 6 pencil per spectral
   index (l1, l2, l3): curl [[0, -L3, L2], [L3, 0, -L1], [-L2, L1, 0]] with
   L_l = (exp(i 2 pi (l_l + k.a_l) / n_l) - 1) / delta_l, and the material
   written here by hand from eqs. chiral_para_mtx / pseudo_chiral_para_mtx.
   The union of those small spectra must equal the oracle's dense spectrum;
   a wrong coupling (2 i gamma, a sign, a transposed pair) changes it.
2. The Assumption (eq. assump) flips exactly where Phi = eps - xi mu^-1 zeta
   stops being positive: chiral at gamma^2 = eps mu, pseudochiral on the pair
   (a, b) at gamma^2 = min(eps_a mu_b, eps_b mu_a); and NFGEP's 1/Phi equals
   the hand formula 1 / (eps_a - gamma^2 / mu_b) there.
"""

import numpy as np
import scipy.linalg as sla

import workloads as wl
from oracle import gep, media, nfgep

GRID = (4, 3, 5)
K = (0.1, 0.2, 0.3)


def per_index_spectrum(grid, kdota, eps, mu, xi, zeta):
    """All 6n eigenvalues from 6 x 6 pencils per spectral index; eps, mu, xi,
    zeta are the 3 x 3 per-voxel tensors of a homogeneous medium."""
    n1, n2, n3 = grid
    out = []
    for l3 in range(n3):
        for l2 in range(n2):
            for l1 in range(n1):
                L = [(np.exp(2j * np.pi * (l + k) / m) - 1.0) * m for l, k, m in zip((l1, l2, l3), kdota, grid)]
                Ck = np.array([[0, -L[2], L[1]], [L[2], 0, -L[0]], [-L[1], L[0], 0]], dtype=np.complex128)
                Kk = np.block([[np.zeros((3, 3)), Ck.conj().T], [Ck, np.zeros((3, 3))]])
                Bk = np.block([[eps, -1j * xi], [1j * zeta, mu]])
                out.append(sla.eigh(Kk, Bk, eigvals_only=True))
    return np.sort(np.concatenate(out))


def test_homogeneous_chiral_spectrum_by_spectral_index():
    e, m, g = 4.0, 1.5, 0.7
    n1, n2, n3 = GRID
    shape = (3, n3, n2, n1)
    med = wl.Medium(GRID, "chiral", np.full(shape, e), np.full(shape, g), np.full(shape, m))
    w, _, _ = gep.dense_eigs(GRID, K, med)
    I = np.eye(3)
    # eq. chiral_para_mtx: xi = i gamma I, zeta = -i gamma I
    ref = per_index_spectrum(GRID, K, e * I, m * I, 1j * g * I, -1j * g * I)
    scale = np.abs(ref).max()
    assert np.abs(np.sort(w) - ref).max() < 1e-11 * scale
    # and the coupling matters: twice the coupling is a different spectrum
    twice = per_index_spectrum(GRID, K, e * I, m * I, 2j * g * I, -2j * g * I)
    assert np.abs(twice - ref).max() > 1e-3 * scale


def test_homogeneous_pseudochiral_spectrum_by_spectral_index():
    n1, n2, n3 = GRID
    epsv, muv, g, (a, b) = (4.0, 9.0, 2.0), (1.0, 2.0, 1.5), 0.9, (0, 2)
    eps = np.stack([np.full((n3, n2, n1), v) for v in epsv])
    mu = np.stack([np.full((n3, n2, n1), v) for v in muv])
    med = wl.Medium(GRID, "pseudochiral", eps, np.full((n3, n2, n1), g), mu, (a, b))
    w, _, _ = gep.dense_eigs(GRID, K, med)
    # eq. pseudo_chiral_para_mtx: i gamma in the two off-diagonal places of the pair
    xi = np.zeros((3, 3), np.complex128)
    xi[a, b] = xi[b, a] = 1j * g
    ref = per_index_spectrum(GRID, K, np.diag(epsv), np.diag(muv), xi, xi.conj())
    scale = np.abs(ref).max()
    assert np.abs(np.sort(w) - ref).max() < 1e-11 * scale
    # the other pair gives another spectrum (the pair is not ignored)
    xo = np.zeros((3, 3), np.complex128)
    xo[0, 1] = xo[1, 0] = 1j * g
    other = per_index_spectrum(GRID, K, np.diag(epsv), np.diag(muv), xo, xo.conj())
    assert np.abs(other - ref).max() > 1e-4 * scale


def _chiral(e, m, g):
    n1, n2, n3 = GRID
    shape = (3, n3, n2, n1)
    return wl.Medium(GRID, "chiral", np.full(shape, e), np.full(shape, g), np.full(shape, m))


def test_assumption_flips_at_gamma_squared_eps_mu_chiral():
    e, m = 4.0, 2.25            # eps mu = 9: the boundary is gamma = 3
    for f, holds in ((1 - 1e-6, True), (1 + 1e-6, False)):
        assert media.assumption_holds(_chiral(e, m, 3.0 * f)) is holds
    for g in (1.3, 3.0 * (1 - 1e-6)):
        ph = nfgep.NFGEP(GRID, K, _chiral(e, m, g)).phi_inv
        hand = 1.0 / (e - g * g / m)
        for c in range(3):
            assert np.allclose(ph[c, c], hand, rtol=1e-9, atol=0)


def test_assumption_flips_at_the_pseudochiral_pair_boundary():
    n1, n2, n3 = GRID
    epsv, muv, (a, b) = (4.0, 9.0, 2.0), (1.0, 2.0, 1.5), (0, 1)
    # Phi_a = eps_a - gamma^2 / mu_b = 4 - gamma^2 / 2, Phi_b = 9 - gamma^2 / 1:
    # the first reaches zero first, at gamma^2 = 8
    gb = np.sqrt(8.0)
    eps = np.stack([np.full((n3, n2, n1), v) for v in epsv])
    mu = np.stack([np.full((n3, n2, n1), v) for v in muv])

    def med(g):
        return wl.Medium(GRID, "pseudochiral", eps, np.full((n3, n2, n1), g), mu, (a, b))

    for f, holds in ((1 - 1e-6, True), (1 + 1e-6, False)):
        assert media.assumption_holds(med(gb * f)) is holds
    g = 1.7
    ph = nfgep.NFGEP(GRID, K, med(g)).phi_inv
    hand = {a: 1.0 / (epsv[a] - g * g / muv[b]), b: 1.0 / (epsv[b] - g * g / muv[a]), 2: 1.0 / epsv[2]}
    for c in range(3):
        assert np.allclose(ph[c, c], hand[c], rtol=1e-12, atol=0)
        for d in range(3):
            if d != c:
                assert np.abs(ph[c, d]).max() == 0.0
