"""GPU parity of the null space free standard problem for media outside the
Assumption (thm:nfep, eq. NFSEP_org; Algorithm 1's second branch) against the
CPU oracle: the product M y element by element, the fields of the second
branch, the eigenvalues nearest a shift (shift-and-invert Arnoldi with GMRES)
against the oracle's stored ones, and the GEP residual of the computed
eigenpairs through the oracle's finite-difference curl.  complex128
throughout: 1e-12 relative for the products and fields (as the complex128
A_r product), 1e-9 for eigenvalues (Ritz tolerance 1e-10)."""

import os

import numpy as np
import pytest

import workloads as wl
from oracle import gep, nfsep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = (0.1, 0.2, 0.3)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "nfsep8_omega.txt")

CASES = [
    ("lossy8", (8, 8, 8), lambda g: wl.biisotropic_sphere(g, 0.25, 13.0 + 2.0j, 1.0, 0.5, 0.2)),
    ("tellegen_mu_12x16", (12, 12, 16), lambda g: wl.biisotropic_sphere(g, 0.3, 6.0, 1.0, 0.8, 0.9, mu_in=1.5)),
    ("nonreciprocal_16x24", (16, 16, 24), lambda g: wl.biisotropic_sphere(g, 0.3, 9.0, 1.0, 0.3, 0.4 + 0.3j)),
    ("strong_24x12", (24, 24, 12), lambda g: wl.biisotropic_sphere(g, 0.3, 2.0, 1.0, 1.2, 1.1)),
]


def rel_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,grid,make", CASES, ids=[c[0] for c in CASES])
def test_nfsep_matvec_and_fields_parity(lib, name, grid, make):
    med = make(grid)
    orc = nfsep.NFSEP(grid, K, med)
    ctx = lib.NFSEPContext(grid, K, med)
    y = wl.random_complex(ctx.N, 51)
    got = ctx.matvec(torch.from_numpy(y).cuda()).cpu().numpy()
    assert rel_err(got, orc.apply(y)) < 1e-12
    X = ctx.fields(torch.from_numpy(y).cuda()).cpu().numpy()[0]
    assert rel_err(X, orc.fields(y)) < 1e-12
    ctx.close()


def test_ar_calls_refuse_a_biisotropic_context(lib):
    import ctypes
    g = (8, 8, 8)
    ctx = lib.NFSEPContext(g, K, CASES[0][2](g))
    u = torch.zeros(ctx.N, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(u)
    rc = lib.lib().nfs_matvec(ctx.h, lib.C128, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    assert rc == lib.NFS_EUNSUPPORTED
    ctx.close()


def test_nfsep_eigs_nearest_shift(lib):
    """The four eigenvalues nearest 2 + 0.1i of the lossy sphere equal the
    oracle's; their fields solve the GEP (eq. discrete_GEP_EH)."""
    g = (8, 8, 8)
    med = CASES[0][2](g)
    ref = np.loadtxt(GOLDEN)
    ref = ref[:, 0] + 1j * ref[:, 1]
    ctx = lib.NFSEPContext(g, K, med, eig_tol=1e-10, cg_tol=1e-12, cg_maxit=4000)
    om, Y, info = ctx.eigs(4, 2.0 + 0.1j)
    assert info.nconv == 4
    assert np.abs(om - ref).max() < 1e-9 * np.abs(ref).max(), (om, ref)
    X = ctx.fields(Y).cpu().numpy()
    for j in range(4):
        assert gep.gep_residual(g, K, med, om[j], X[j]) < 1e-8
    ctx.close()


def test_nfsep_eigs_16_vs_oracle(lib):
    """The same sphere on 16^3 (the bench's second NFSEP size): the four
    eigenvalues nearest 2 + 0.1i against the oracle's stored ones."""
    g = (16, 16, 16)
    ref = np.loadtxt(os.path.join(os.path.dirname(GOLDEN), "nfsep16_omega.txt"))
    ref = ref[:, 0] + 1j * ref[:, 1]
    ctx = lib.NFSEPContext(g, K, CASES[0][2](g), eig_tol=1e-10, cg_tol=1e-12, cg_maxit=20000, max_restarts=20)
    om, _, info = ctx.eigs(4, 2.0 + 0.1j, vectors=False)
    ctx.close()
    assert info.nconv == 4
    assert rel_err(om, ref) < 1e-9, (om, ref)


def test_nfsep_reserve_then_eigs_allocates_nothing(lib):
    """nfs_reserve on a bi-isotropic context takes the Arnoldi and GMRES bases
    up front; the eigensolve then allocates no device memory."""
    g = (8, 8, 8)
    ctx = lib.NFSEPContext(g, K, CASES[0][2](g), eig_tol=1e-10, cg_tol=1e-12, cg_maxit=4000)
    ctx.reserve(4)
    before = ctx.device_bytes
    om, _, info = ctx.eigs(4, 2.0 + 0.1j, vectors=False)
    assert ctx.device_bytes == before
    assert info.nconv == 4
    ctx.close()
