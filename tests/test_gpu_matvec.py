"""GPU parity of the A_r product, B_r and CG against the CPU oracle
(element by element, seeded inputs).  Tolerances: complex128 path 1e-12
relative to the largest output entry (FFT round-off of O(log n) ulps with a
1e4 margin); complex64 path 2e-5 (single-precision FFT and basis round-off,
log2(n) ~ 20 butterfly levels of ~6e-8)."""

import numpy as np
import pytest

import workloads as wl
from oracle import nfgep

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = (0.1, 0.2, 0.3)

CASES = [
    ("sphere8", (8, 8, 8), lambda g: wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)),
    ("sphere12x16", (12, 12, 16), lambda g: wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.7)),
    ("pseudo_xy_16x24", (16, 16, 24), lambda g: wl.pseudochiral_cylinders(g, 4, 0.15, 13.0, 1.0, 0.4, (0, 1), 1)),
    ("pseudo_xz_24x12", (24, 24, 12), lambda g: wl.pseudochiral_cylinders(g, 3, 0.2, 9.0, 1.5, 0.6, (0, 2), 2)),
    ("field32x48", (32, 32, 48), lambda g: wl.smoothed_chiral_field(g, seed=4, sigma=0.1)),
    ("field48x32", (48, 48, 32), lambda g: wl.smoothed_chiral_field(g, seed=6, sigma=0.1)),
]


def with_mu(med):
    rng = np.random.default_rng(3)
    mu = 1.0 + 0.5 * rng.random(med.eps.shape)
    m = wl.Medium(med.grid, med.kind, med.eps, med.gamma, mu, med.axes)
    return m


@pytest.fixture(scope="module")
def nfs(lib):
    return lib


def rel_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,grid,make", CASES, ids=[c[0] for c in CASES])
def test_matvec_parity(nfs, name, grid, make):
    med = make(grid)
    ctx = nfs.Context(grid, K, med, precision="mixed")
    orc = nfgep.NFGEP(grid, K, med)
    u = wl.random_complex(4 * ctx.n, 17)
    ref = orc.Ar(u)
    got64 = ctx.matvec(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(got64, ref) < 1e-12
    got32 = ctx.matvec(torch.from_numpy(u.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel_err(got32, ref) < 2e-5
    ctx.close()


@pytest.mark.parametrize("kind", ["chiral", "pseudochiral"])
def test_matvec_with_mu(nfs, kind):
    g = (16, 16, 12)
    base = (wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.5) if kind == "chiral"
            else wl.pseudochiral_cylinders(g, 2, 0.2, 13.0, 1.0, 0.5, (1, 2), 5))
    med = with_mu(base)
    ctx = nfs.Context(g, K, med)
    u = wl.random_complex(4 * ctx.n, 23)
    ref = nfgep.NFGEP(g, K, med).Ar(u)
    got = ctx.matvec(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(got, ref) < 1e-12
    ctx.close()


def test_matvec_hermitian_positive(nfs):
    """A_r is Hermitian positive definite (thm:NFSEP_real_ew): <v, A u> =
    conj(<u, A v>) and <u, A u> > 0 on the device path."""
    g = (24, 24, 24)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    ctx = nfs.Context(g, K, med)
    u = torch.from_numpy(wl.random_complex(4 * ctx.n, 1)).cuda()
    v = torch.from_numpy(wl.random_complex(4 * ctx.n, 2)).cuda()
    Au, Av = ctx.matvec(u), ctx.matvec(v)
    lhs = torch.vdot(v, Au).item()
    rhs = torch.vdot(u, Av).item().conjugate()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert torch.vdot(u, Au).real.item() > 0
    ctx.close()


def test_apply_Br(nfs):
    g = (12, 12, 8)
    med = wl.chiral_sphere(g)
    ctx = nfs.Context(g, K, med)
    v = wl.random_complex(4 * ctx.n, 5)
    got = ctx.apply_Br(torch.from_numpy(v).cuda()).cpu().numpy()
    ref = nfgep.NFGEP(g, K, med).Br(v)
    assert rel_err(got, ref) < 1e-14
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_solve(nfs, precision):
    g = (16, 16, 16)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    ctx = nfs.Context(g, K, med, precision=precision, cg_tol=1e-11)
    orc = nfgep.NFGEP(g, K, med)
    b = wl.random_complex(4 * ctx.n, 9)
    x, info = ctx.cg_solve(torch.from_numpy(b).cuda())
    assert info.status == 0
    x = x.cpu().numpy()
    res = np.linalg.norm(orc.Ar(x) - b) / np.linalg.norm(b)
    assert res < 1e-10
    xo, _ = orc.cg(b, tol=1e-13)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-9
    if precision == "mixed":
        assert info.refinements >= 1
    ctx.close()


def test_mixed_refinement_reports_true_residual(nfs):
    """Mixed refinement switches to the complex64 product of the correction
    once the residual is small; the residual it then reports (a recursive one)
    must stay within a few percent of the tolerance of the true residual."""
    g = (48, 48, 48)
    med = wl.pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), seed=1)
    tol = 1e-10
    ctx = nfs.Context(g, K, med, precision="mixed", cg_tol=tol)
    orc = nfgep.NFGEP(g, K, med)
    b = wl.random_complex(4 * ctx.n, 12)
    x, info = ctx.cg_solve(torch.from_numpy(b).cuda())
    assert info.status == 0 and info.refinements >= 2
    res = np.linalg.norm(orc.Ar(x.cpu().numpy()) - b) / np.linalg.norm(b)
    assert res <= 1.05 * tol, res
    assert abs(res - info.rel_residual) <= 0.05 * tol, (res, info.rel_residual)
    ctx.close()


def test_cg_nonzero_initial_guess_and_maxit(nfs):
    g = (12, 12, 12)
    med = wl.chiral_sphere(g)
    ctx = nfs.Context(g, K, med, cg_maxit=3)
    b = torch.from_numpy(wl.random_complex(4 * ctx.n, 10)).cuda()
    x, info = ctx.cg_solve(b, x0=torch.ones_like(b))
    assert info.status == nfs.NFS_ENOCONV and info.iterations == 3
    ctx.close()


def test_matvec_full_size_96(nfs):
    """Full-size parity at 96^3 (pseudochiral cylinders, the headline
    workload) for both element types, in the bench's launch configuration."""
    w = wl.workload("pseudo96")
    grid, med = w["grid"], w["medium"]
    ctx = nfs.Context(grid, w["kdota"], med, precision="mixed")
    orc = nfgep.NFGEP(grid, w["kdota"], med)
    u = wl.random_complex(4 * ctx.n, 31)
    ref = orc.Ar(u)
    got64 = ctx.matvec(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(got64, ref) < 1e-12
    got32 = ctx.matvec(torch.from_numpy(u.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel_err(got32, ref) < 2e-5
    ctx.close()


def test_matvec_full_size_128(nfs):
    """Full-size parity at 128^3 (smoothed chiral field): the complex128
    product runs the five-pass form (a 128 x 128 complex128 plane does not fit
    in shared memory), the complex64 one the three-pass form."""
    w = wl.workload("field128")
    grid, med = w["grid"], w["medium"]
    ctx = nfs.Context(grid, w["kdota"], med, precision="mixed")
    orc = nfgep.NFGEP(grid, w["kdota"], med)
    u = wl.random_complex(4 * ctx.n, 33)
    ref = orc.Ar(u)
    got64 = ctx.matvec(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(got64, ref) < 1e-12
    got32 = ctx.matvec(torch.from_numpy(u.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel_err(got32, ref) < 2e-5
    ctx.close()


@pytest.mark.parametrize("grid", [(8, 8, 8), (12, 12, 16), (96, 96, 96), (128, 128, 128)])
def test_matvec_double_single(nfs, grid):
    """The double-single product (float pairs on the FP32 units) that the mixed
    path uses for its refinement residuals: within 1e-12 of the oracle, like
    the complex128 product, at three-pass and five-pass sizes."""
    med = wl.smoothed_chiral_field(grid, seed=5, sigma=0.1)
    ctx = nfs.Context(grid, K, med, precision="mixed")
    orc = nfgep.NFGEP(grid, K, med)
    u = wl.random_complex(4 * ctx.n, 41)
    ref = orc.Ar(u)
    got = ctx.matvec_ds(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_err(got, ref) < 1e-12
    ctx.close()
    ctx64 = nfs.Context(grid, K, med, precision="fp64")
    with pytest.raises(nfs.NFSError):
        ctx64.matvec_ds(torch.from_numpy(u).cuda())
    ctx64.close()
