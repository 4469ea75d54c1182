"""GPU eigensolver and gradient parity against the oracle.

Eigenvalues: FP64 path within 1e-10 relative of the oracle, mixed path
within 1e-8 and residual ||A_r y - omega B_r y|| / ||y|| <= 1e-8 (the
tolerances the eigensolver is specified to).  Expected values come from
tests/golden (written by tests/golden/make_golden.py from the oracle) or
from the oracle at run time."""

import os

import numpy as np
import pytest

import workloads as wl
from oracle import gep, nfgep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
K = (0.1, 0.2, 0.3)


def golden(name):
    return np.loadtxt(os.path.join(HERE, "golden", name))


@pytest.fixture(scope="module")
def nfs(lib):
    return lib


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_sphere8_eigs_vs_golden(nfs, precision, tol):
    w = wl.workload("sphere8")
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision=precision)
    omega, Y, info = ctx.eigs(10)
    ref = golden("sphere8_omega.txt")
    assert np.abs(omega - ref).max() / ref.min() < tol
    res = nfs.residuals(ctx, omega, Y)
    assert max(res) / omega.max() < 1e-8
    assert info.nconv == 10
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_pseudo8_eigs_vs_golden(nfs, precision, tol):
    g = (8, 8, 8)
    med = wl.pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), seed=0)
    ctx = nfs.Context(g, K, med, precision=precision)
    omega, _, _ = ctx.eigs(10)
    ref = golden("pseudo8_omega.txt")
    assert np.abs(omega - ref).max() / ref.min() < tol
    ctx.close()


def test_eigs_vs_oracle_ragged(nfs):
    """12 x 12 x 16 grid, random smooth field, vs the oracle's ARPACK solve."""
    g = (12, 12, 16)
    med = wl.smoothed_chiral_field(g, seed=3, sigma=0.15)
    ctx = nfs.Context(g, K, med)
    omega, Y, _ = ctx.eigs(6)
    ref, _ = nfgep.NFGEP(g, K, med).eigs(6)
    assert np.abs(omega - ref).max() / ref.min() < 1e-10
    ctx.close()


def test_homogeneous_closed_form(nfs):
    """Section 5.1: (1, 1, 0) eigenvalues are sqrt(Lambda_q), each twice."""
    g = (16, 16, 16)
    k = (0.25, 0.1, 0.4)
    ctx = nfs.Context(g, k, wl.homogeneous(g))
    omega, _, _ = ctx.eigs(8)
    n1 = 16
    i = np.arange(n1)
    s1 = 4 * np.sin(np.pi * (i + k[0]) / n1) ** 2 * n1 ** 2
    s2 = 4 * np.sin(np.pi * (i + k[1]) / n1) ** 2 * n1 ** 2
    s3 = 4 * np.sin(np.pi * (i + k[2]) / n1) ** 2 * n1 ** 2
    disp = np.sqrt(s3[:, None, None] + s2[None, :, None] + s1[None, None, :]).ravel()
    ref = np.sort(np.concatenate([disp, disp]))[:8]
    assert np.abs(omega - ref).max() / ref.min() < 1e-10
    ctx.close()


def test_homogeneous_closed_form_128_mixed(nfs):
    """Section 5.1 closed form at 128^3 on the mixed path (its refinement
    products run the five-pass complex128 product of planes that do not fit
    in shared memory)."""
    g = (128, 128, 128)
    k = (0.25, 0.1, 0.4)
    ctx = nfs.Context(g, k, wl.homogeneous(g), precision="mixed")
    omega, _, _ = ctx.eigs(6, vectors=False)
    n1 = 128
    i = np.arange(n1)
    s = [4 * np.sin(np.pi * (i + kk) / n1) ** 2 * n1 ** 2 for kk in k]
    disp = np.sqrt(s[2][:, None, None] + s[1][None, :, None] + s[0][None, None, :]).ravel()
    ref = np.sort(np.concatenate([disp, disp]))[:6]
    assert np.abs((omega - ref) / ref).max() < 1e-8
    ctx.close()


def test_eig_gradient_vs_oracle(nfs):
    """Adjoint gradient of omega_1 + 2 omega_2 w.r.t. per-component eps and
    gamma against the oracle's pencil perturbation formula (8^3, random
    field so the eigenvalues are simple)."""
    g = (8, 8, 8)
    med = wl.smoothed_chiral_field(g, seed=11, sigma=0.15)
    ctx = nfs.Context(g, K, med)
    omega, Y, _ = ctx.eigs(3)
    weights = np.array([1.0, 2.0])
    d_eps, d_gam = ctx.eig_grad(Y[:2].contiguous(), weights)
    w, z, idx = gep.dense_eigs(g, K, med)
    assert np.abs(w[idx[:3]] - omega).max() / omega.min() < 1e-10
    re = np.zeros((3,) + med.eps.shape[1:])
    rg = np.zeros_like(re)
    for j, wt in enumerate(weights):
        a, b = gep.pencil_gradient(med, w[[idx[j]]], z[:, [idx[j]]])
        re += wt * a
        rg += wt * b
    de = d_eps.cpu().numpy()
    dg = d_gam.cpu().numpy()
    assert np.abs(de - re).max() / np.abs(re).max() < 1e-6
    assert np.abs(dg - rg).max() / np.abs(rg).max() < 1e-6
    ctx.close()


def test_eig_gradient_pseudochiral(nfs):
    g = (8, 8, 8)
    med = wl.pseudochiral_cylinders(g, 2, 0.2, 9.0, 1.0, 0.5, (0, 2), seed=4)
    # perturb eps with a smooth field so that no eigenvalue is degenerate
    med.eps = med.eps * (1.0 + 0.3 * wl.media.smoothed_field(g, 8, 0.2))[None]
    ctx = nfs.Context(g, K, med)
    omega, Y, _ = ctx.eigs(2)
    d_eps, d_gam = ctx.eig_grad(Y[:1].contiguous(), [1.0])
    w, z, idx = gep.dense_eigs(g, K, med)
    re, rg = gep.pencil_gradient(med, w[[idx[0]]], z[:, [idx[0]]])
    assert np.abs(d_eps.cpu().numpy() - re).max() / np.abs(re).max() < 1e-6
    assert np.abs(d_gam.cpu().numpy() - rg).max() / np.abs(rg).max() < 1e-6
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deflation_checks_find_degenerate_copies(nfs, precision):
    """At k.a = (0.45, 0.05, 0) the z-invariant cylinders keep the mirror
    symmetry z -> -z and this medium has a double eigenvalue at positions 7
    and 8 (oracle).  With deflation checks the solver returns both copies;
    every check it ran is reported."""
    g = (8, 8, 8)
    k = (0.45, 0.05, 0.0)
    med = wl.pseudochiral_cylinders(g, 2, 0.2, 13.0, 1.0, 0.5, (0, 2), 4)
    w, _, idx = gep.dense_eigs(g, k, med)
    ref = w[idx[:8]]
    assert abs(ref[7] - ref[6]) < 1e-10 * ref[7]  # the degenerate pair
    ctx = nfs.Context(g, k, med, precision=precision, deflation_checks=3)
    omega, Y, info = ctx.eigs(8)
    assert np.abs(omega - ref).max() < 1e-9 * ref.max()
    assert 1 <= info.deflation_checks <= 3
    # the returned vectors are A_r-orthonormal eigenvectors, the pair included
    res = nfs.residuals(ctx, omega, Y)
    assert max(res) < 1e-8
    ctx.close()


def test_residuals_call_matches_oracle(nfs):
    # nfs_residuals against the oracle's ||A_r y - omega B_r y|| / ||y|| for
    # eigenpairs whose omega is perturbed by a known amount (so the residual
    # is far above rounding): same definition, two independent evaluations
    w = wl.workload("sphere8")
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision="fp64")
    omega, Y, _ = ctx.eigs(4)
    om_p = omega * (1.0 + 1e-3 * np.arange(1, 5))
    got = nfs.residuals(ctx, om_p, Y)
    O = nfgep.NFGEP(w["grid"], w["kdota"], w["medium"])
    Yh = Y.cpu().numpy()
    ref = [O.residual(om_p[j], Yh[j]) for j in range(4)]
    assert np.allclose(got, ref, rtol=1e-9, atol=0), (got, ref)
    ctx.close()


def test_reserve_then_eigs_allocates_nothing(nfs):
    w = wl.workload("sphere8")
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision="mixed")
    ctx.reserve(6)
    before = ctx.device_bytes
    ctx.eigs(6)
    assert ctx.device_bytes == before
    ctx.close()
    # an explicit basis size: the basis is taken by nfs_setup itself
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision="mixed", ncv=18)
    before = ctx.device_bytes
    ctx.eigs(6)
    assert ctx.device_bytes == before
    ctx.close()
