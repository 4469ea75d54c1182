"""The differentiable eigenvalue function (autograd over nfs_eig_grad) against
central finite differences of the GPU eigenvalues and against the oracle.

A per-voxel difference with step 1e-6 is below the eigenvalue accuracy
(d omega / d eps_v ~ omega / n), so the finite-difference checks are
directional: grad . d against [f(p + h d) - f(p - h d)] / 2h with a dense
random direction d, plus a per-voxel check with a larger step.  The
directional step is h = 1e-4: with |grad . d| ~ 1e-2 a step of 1e-6 would need
the eigenvalue sums to ~1e-15 absolute, below what an iterative solve at
tolerance 1e-13 reproduces between runs, while h = 1e-4 keeps the O(h^2)
truncation near 1e-8 relative."""

import numpy as np
import pytest

import workloads as wl
from oracle import gep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = (0.1, 0.2, 0.3)


@pytest.fixture(scope="module")
def ag(lib):
    from paper_1402_6297_gb300 import autograd
    return autograd


def f_sum(ag, eps, gam, g, nev=5):
    return float(ag.chiral_eigenvalues(eps, gam, g, K, nev=6, eig_tol=1e-12, cg_tol=1e-13)[:nev].sum())


def test_directional_derivative_matches_central_difference(ag):
    g = (16, 16, 16)
    med = wl.smoothed_chiral_field(g, seed=2, sigma=0.1)
    eps = torch.tensor(med.eps[0], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor(med.gamma[0], dtype=torch.float64, requires_grad=True)
    om = ag.chiral_eigenvalues(eps, gam, g, K, nev=6, eig_tol=1e-12, cg_tol=1e-13)
    assert om[4] < om[5] * (1 - 1e-6)  # the summed cluster is complete
    om[:5].sum().backward()
    rng = np.random.default_rng(0)
    for which in ("eps", "gamma"):
        d = torch.tensor(rng.standard_normal(eps.shape))
        h = 1e-4
        base_e, base_g = eps.detach(), gam.detach()
        if which == "eps":
            fp = f_sum(ag, base_e + h * d, base_g, g)
            fm = f_sum(ag, base_e - h * d, base_g, g)
            an = float((eps.grad * d).sum())
        else:
            fp = f_sum(ag, base_e, base_g + h * d, g)
            fm = f_sum(ag, base_e, base_g - h * d, g)
            an = float((gam.grad * d).sum())
        fd = (fp - fm) / (2 * h)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9, (which, fd, an)


def test_per_voxel_gradient_large_step(ag):
    g = (8, 8, 8)
    med = wl.smoothed_chiral_field(g, seed=7, sigma=0.15)
    eps = torch.tensor(med.eps[0], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor(med.gamma[0], dtype=torch.float64, requires_grad=True)
    om = ag.chiral_eigenvalues(eps, gam, g, K, nev=3, eig_tol=1e-12, cg_tol=1e-13)
    om[0].backward()
    # oracle: pencil perturbation formula, summed over the three components
    w, z, idx = gep.dense_eigs(g, K, med)
    re, rg = gep.pencil_gradient(med, w[[idx[0]]], z[:, [idx[0]]])
    assert np.abs(eps.grad.numpy() - re.sum(0)).max() < 1e-6 * np.abs(re.sum(0)).max()
    assert np.abs(gam.grad.numpy() - rg.sum(0)).max() < 1e-6 * np.abs(rg.sum(0)).max()
    # per-voxel central differences with h = 1e-3 (second-order error ~ h^2)
    rng = np.random.default_rng(1)
    for _ in range(4):
        v = tuple(int(x) for x in rng.integers(0, 8, size=3))
        h = 1e-3
        e2 = eps.detach().clone()
        e2[v] += h
        fp = float(ag.chiral_eigenvalues(e2, gam.detach(), g, K, nev=3, eig_tol=1e-12, cg_tol=1e-13)[0])
        e2[v] -= 2 * h
        fm = float(ag.chiral_eigenvalues(e2, gam.detach(), g, K, nev=3, eig_tol=1e-12, cg_tol=1e-13)[0])
        fd = (fp - fm) / (2 * h)
        an = float(eps.grad[v])
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-10, (v, fd, an)


def test_uniform_direction_derivative_128(lib):
    """At 128^3 (five-pass complex128 pass 1 inside the gradient): the sum of
    d(omega_1 + ... + omega_5)/d eps over every voxel and component against a
    central difference of eigensolves with all of eps shifted by +-h.  A
    per-voxel step would move omega by less than the solver's accuracy; the
    uniform direction moves the sum by ~1e-4 at h = 1e-4."""
    nfs = lib
    w = wl.workload("field128")
    g, k, med = w["grid"], w["kdota"], w["medium"]
    opts = dict(precision="mixed", cg_tol=1e-11, eig_tol=1e-11)
    ctx = nfs.Context(g, k, med, **opts)
    omega, Y, _ = ctx.eigs(6)
    assert omega[4] < omega[5] * (1 - 1e-6)
    d_eps, _ = ctx.eig_grad(Y[:5].contiguous(), np.ones(5))
    an = float(d_eps.sum())
    ctx.close()
    h = 1e-4
    f = []
    for sgn in (1, -1):
        m2 = wl.Medium(med.grid, med.kind, med.eps + sgn * h, med.gamma, med.mu, med.axes)
        c2 = nfs.Context(g, k, m2, **opts)
        om2, _, _ = c2.eigs(6, vectors=False)
        f.append(float(om2[:5].sum()))
        c2.close()
    fd = (f[0] - f[1]) / (2 * h)
    assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)


def test_library_context_released_without_backward(ag, lib):
    # inference (no_grad) keeps nothing; a forward whose output is dropped
    # before backward releases its context with the graph
    import gc
    g = (8, 8, 8)
    med = wl.chiral_sphere(g)
    eps = torch.tensor(med.eps[0], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor(med.gamma[0], dtype=torch.float64, requires_grad=True)
    gc.collect()
    before = lib.live_contexts()
    with torch.no_grad():
        om = ag.chiral_eigenvalues(eps, gam, g, K, nev=3)
    assert lib.live_contexts() == before
    om = ag.chiral_eigenvalues(eps, gam, g, K, nev=3)
    assert lib.live_contexts() == before + 1
    del om
    gc.collect()
    assert lib.live_contexts() == before
    om = ag.chiral_eigenvalues(eps, gam, g, K, nev=3)
    om.sum().backward()
    assert lib.live_contexts() == before


def test_oracle_pencil_gradient_16(lib):
    """Config 5's oracle check at 16^3: d(omega_1 + ... + omega_5) / d(every
    per-component eps and gamma) from the GPU's NFGEP adjoint against the
    oracle's first-order perturbation of the Hermitian pencil K'' z = omega B'' z
    (independent formulas), with the oracle's own eigenvectors: tier O3
    (FFT NFGEP, ARPACK) y -> fields [E; H] of Algorithm 1's last step ->
    z = [E; i H]."""
    from oracle import nfgep
    w = wl.workload("field16")
    g, k, med = w["grid"], w["kdota"], w["medium"]
    O = nfgep.NFGEP(g, k, med)
    om_o, Y_o = O.eigs(6, tol=1e-12, cg_tol=1e-13)
    assert om_o[4] < om_o[5] * (1 - 1e-6)  # the summed cluster is complete
    n = O.n
    Z = []
    for j in range(5):
        x = O.eigvec_fields(Y_o[:, j]).reshape(6, n)
        Z.append(np.concatenate([x[:3].ravel(), 1j * x[3:].ravel()]))
    re, rg = gep.pencil_gradient(med, om_o[:5], np.stack(Z, axis=1))
    ctx = lib.Context(g, k, med, precision="fp64", eig_tol=1e-12, cg_tol=1e-13)
    omega, Y, _ = ctx.eigs(6)
    assert np.abs(omega[:5] - om_o[:5]).max() < 1e-10 * om_o[4]
    d_eps, d_gam = ctx.eig_grad(Y[:5].contiguous(), np.ones(5))
    ctx.close()
    d_eps, d_gam = d_eps.cpu().numpy(), d_gam.cpu().numpy()
    assert np.abs(d_eps - re).max() < 1e-6 * np.abs(re).max()
    assert np.abs(d_gam - rg).max() < 1e-6 * np.abs(rg).max()


def test_per_voxel_central_differences_64(lib):
    """Config 5 at 64^3: the gradient of omega_1 + ... + omega_5 with respect to
    the per-voxel eps (all three components of a voxel move together) on 32
    random voxels against central differences with step h = 0.05 (the
    readings' larger per-voxel step: d omega / d eps_v ~ omega / n, so a step
    of 1e-6 would move omega below the eigensolver's accuracy; the O(h^2)
    truncation of a single-voxel change scales with 1/n^2)."""
    w = wl.workload("field64")
    g, k, med = w["grid"], w["kdota"], w["medium"]
    opts = dict(precision="mixed", cg_tol=1e-12, eig_tol=1e-12)
    ctx = lib.Context(g, k, med, **opts)
    omega, Y, _ = ctx.eigs(6)
    assert omega[4] < omega[5] * (1 - 1e-6)
    d_eps, _ = ctx.eig_grad(Y[:5].contiguous(), np.ones(5))
    ctx.close()
    grad_v = d_eps.sum(0).cpu().numpy()  # per voxel: the three components together
    rng = np.random.default_rng(64)
    h = 0.05
    errs = []
    for _ in range(32):
        v = tuple(int(x) for x in rng.integers(0, 64, size=3))
        f = []
        for sgn in (1, -1):
            e2 = med.eps.copy()
            e2[(slice(None),) + v] += sgn * h
            m2 = wl.Medium(med.grid, med.kind, e2, med.gamma, med.mu, med.axes)
            c2 = lib.Context(g, k, m2, **opts)
            om2, _, _ = c2.eigs(6, vectors=False)
            c2.close()
            f.append(float(om2[:5].sum()))
        fd = (f[0] - f[1]) / (2 * h)
        errs.append(abs(fd - grad_v[v]) / abs(grad_v[v]))
    assert max(errs) < 1e-4, max(errs)


def test_random_direction_derivative_128(lib):
    """At 128^3: grad . d of omega_1 + ... + omega_5 for a dense random
    direction d (uniform in [0.5, 1.5] at every voxel and component of eps)
    against a central difference of eigensolves at eps +- h d, to 1e-6
    relative.  Signed normal entries would cancel the gradient down to ~1e-6
    (measured), below what solves accurate to ~1e-12 can difference at any
    admissible step; with positive entries grad . d ~ 0.5 and h = 1e-4 puts
    both the solvers' noise (~1e-11 / 2h) and the O(h^2) truncation near
    1e-7 relative."""
    w = wl.workload("field128")
    g, k, med = w["grid"], w["kdota"], w["medium"]
    opts = dict(precision="mixed", cg_tol=1e-12, eig_tol=1e-12)
    ctx = lib.Context(g, k, med, **opts)
    omega, Y, _ = ctx.eigs(6)
    assert omega[4] < omega[5] * (1 - 1e-6)
    d_eps, _ = ctx.eig_grad(Y[:5].contiguous(), np.ones(5))
    ctx.close()
    d = np.random.default_rng(128).uniform(0.5, 1.5, size=med.eps.shape)
    an = float((d_eps.cpu().numpy() * d).sum())
    h = 1e-4
    f = []
    for sgn in (1, -1):
        m2 = wl.Medium(med.grid, med.kind, med.eps + sgn * h * d, med.gamma, med.mu, med.axes)
        c2 = lib.Context(g, k, m2, **opts)
        om2, _, _ = c2.eigs(6, vectors=False)
        c2.close()
        f.append(float(om2[:5].sum()))
    fd = (f[0] - f[1]) / (2 * h)
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
