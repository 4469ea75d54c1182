"""GPU parity of the eigenvector fields x = [E; H] = B^{-1} diag(P_r, Q_r) y
(Algorithm 1, final step) and of the GEP residual against the CPU oracle,
element by element on seeded inputs, and the end-to-end property that the
fields of computed eigenpairs solve the GEP of eq. (discrete_GEP_EH).

The fields are one complex128 product's first half (pass 1 and the z DFT,
O(log n) ulps), the pointwise material step and the Bloch twist: 1e-12
relative to the largest entry, as for the complex128 product.  The residual
is a norm ratio of stencil sums in FP64: 1e-10 relative (it cancels nothing
for a random x, where it is O(1))."""

import numpy as np
import pytest

import workloads as wl
from oracle import gep, nfgep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = (0.1, 0.2, 0.3)
K_FAR = (1.3, -0.45, 2.2)  # k.a_l outside [0, 1): the twist uses k.a_l itself


def with_mu(med, seed=3):
    rng = np.random.default_rng(seed)
    mu = 1.0 + 0.5 * rng.random(med.eps.shape)
    return wl.Medium(med.grid, med.kind, med.eps, med.gamma, mu, med.axes)


CASES = [
    ("sphere8", (8, 8, 8), K, lambda g: wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)),
    ("sphere12x16_kfar", (12, 12, 16), K_FAR, lambda g: wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.7)),
    ("pseudo_xy_16x24", (16, 16, 24), K, lambda g: wl.pseudochiral_cylinders(g, 4, 0.15, 13.0, 1.0, 0.4, (0, 1), 1)),
    ("pseudo_xz_24x12_mu", (24, 24, 12), K,
     lambda g: with_mu(wl.pseudochiral_cylinders(g, 3, 0.2, 9.0, 1.5, 0.6, (0, 2), 2))),
    ("field32x48_mu", (32, 32, 48), K_FAR, lambda g: with_mu(wl.smoothed_chiral_field(g, seed=4, sigma=0.1))),
    # complex128 planes of 128 x 128 take the five-pass form of the product
    ("split128x16", (128, 128, 16), K, lambda g: wl.smoothed_chiral_field(g, seed=9, sigma=0.1)),
]


def rel_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,grid,k,make", CASES, ids=[c[0] for c in CASES])
def test_fields_parity(lib, name, grid, k, make):
    med = make(grid)
    orc = nfgep.NFGEP(grid, k, med)
    for precision in ("fp64", "mixed"):
        ctx = lib.Context(grid, k, med, precision=precision)
        Y = np.stack([wl.random_complex(4 * ctx.n, 31), wl.random_complex(4 * ctx.n, 32)])
        X = ctx.eig_fields(torch.from_numpy(Y).cuda()).cpu().numpy()
        assert X.shape == (2, 6) + orc.shape
        for j in range(2):
            assert rel_err(X[j], orc.eigvec_fields(Y[j])) < 1e-12
        ctx.close()


@pytest.mark.parametrize("name,grid,k,make", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_gep_residual_parity(lib, name, grid, k, make):
    """The residual of arbitrary fields at an arbitrary omega equals the
    oracle's sparse-matrix value."""
    med = make(grid)
    ctx = lib.Context(grid, k, med)
    X = np.stack([wl.random_complex(6 * ctx.n, 41), wl.random_complex(6 * ctx.n, 42)])
    omega = np.array([3.7, -0.25])
    got = ctx.gep_residual(omega, torch.from_numpy(X).cuda())
    for j in range(2):
        ref = gep.gep_residual(grid, k, med, omega[j], X[j])
        assert abs(got[j] - ref) < 1e-10 * ref
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eigenpair_fields_solve_the_gep(lib, precision):
    """Fields of the GPU eigenpairs solve the 6n GEP: the device residual and
    the oracle's sparse residual of the same fields agree and are small."""
    g = (12, 12, 16)
    med = wl.pseudochiral_cylinders(g, 2, 0.2, 13.0, 1.0, 0.5, (0, 2), 7)
    ctx = lib.Context(g, K, med, precision=precision, eig_tol=1e-12, cg_tol=1e-13)
    omega, Y, _ = ctx.eigs(6)
    X = ctx.eig_fields(Y)
    res = ctx.gep_residual(omega, X)
    Xh = X.cpu().numpy()
    for j in range(6):
        ref = gep.gep_residual(g, K, med, omega[j], Xh[j])
        assert ref < 1e-9
        assert abs(res[j] - ref) < 1e-6 * ref + 1e-15
    ctx.close()


def test_headline_grid_fields(lib):
    """96^3 pseudochiral cylinders, mixed precision: the fields of the four
    lowest eigenpairs solve the GEP, and those of the first equal the oracle's
    recovery of the same eigenvector element by element."""
    w = wl.workload("pseudo96", 0)
    g, k, med = w["grid"], w["kdota"], w["medium"]
    ctx = lib.Context(g, k, med, precision="mixed")
    omega, Y, _ = ctx.eigs(4)
    X = ctx.eig_fields(Y)
    res = ctx.gep_residual(omega, X)
    assert np.all(res < 1e-9), res
    ref = nfgep.NFGEP(g, k, med).eigvec_fields(Y[0].cpu().numpy())
    assert rel_err(X[0].cpu().numpy(), ref) < 1e-12
    ctx.close()
