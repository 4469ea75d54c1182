"""The allocation-free product nfs_matvec_noalloc agrees with nfs_matvec.

nfs_matvec_noalloc exists for callers that cannot let the library allocate
device memory: a host framework that already reserved the GPU through its own
caching allocator, or a service with a fixed device-memory budget.  It runs in
one fixed workspace inside the library.  Here it is called through the C ABI
several times in a row (different inputs, then a different problem, so the
shared workspace is reused with stale contents) and each result is compared
with the ordinary context-based product at the complex128 tolerance the other
parity tests use (1e-12 relative).  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = (0.1, 0.2, 0.3)


def _device(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_context_product_on_consecutive_calls(lib):
    cases = [
        ((16, 16, 24), wl.chiral_sphere((16, 16, 24), 0.3, 13.0, 1.0, 0.6), 1),
        ((16, 16, 24), wl.chiral_sphere((16, 16, 24), 0.3, 13.0, 1.0, 0.6), 2),
        ((32, 32, 16), wl.pseudochiral_cylinders((32, 32, 16), 3, 0.15, 13.0, 1.0, 0.4, (0, 1), 3), 3),
    ]
    for grid, med, seed in cases:
        ctx = lib.Context(grid, K, med)
        u = _device(wl.random_complex(4 * ctx.n, seed))
        ref = ctx.matvec(u)
        out = torch.full_like(u, complex(float("nan"), 0.0))
        lib.matvec_noalloc(grid, K, med.kind, med.axes, _device(med.eps), _device(med.gamma), u, out)
        err = ((out - ref).abs().max() / ref.abs().max()).item()
        assert err < 1e-12, (grid, seed, err)
        ctx.close()


def test_noalloc_rejects_grids_beyond_its_workspace(lib):
    g = (64, 64, 64)  # 262144 voxels > NFS_NOALLOC_MAX_VOXELS
    med = wl.chiral_sphere(g)
    u = torch.zeros(4 * 64 ** 3, dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.NFSError) as exc:
        lib.matvec_noalloc(g, K, "chiral", (0, 1), _device(med.eps), _device(med.gamma), u, torch.empty_like(u))
    assert exc.value.code == lib.NFS_EUNSUPPORTED


def test_noalloc_status_word_is_cleared_between_calls(lib):
    # Phi = eps - gamma^2 < 0 at one voxel: NFS_ENOTHPD.  The next valid call
    # must start from a cleared status word and match the context product.
    g = (16, 16, 24)
    med = wl.chiral_sphere(g, 0.3, 13.0, 1.0, 0.6)
    u = _device(wl.random_complex(4 * 16 * 16 * 24, 4))
    out = torch.empty_like(u)
    bad_eps = med.eps.copy()
    assert med.gamma[1, 12, 8, 8] == 0.6  # inside the sphere
    bad_eps[1, 12, 8, 8] = 0.5 * med.gamma[1, 12, 8, 8] ** 2
    with pytest.raises(lib.NFSError) as exc:
        lib.matvec_noalloc(g, K, "chiral", (0, 1), _device(bad_eps), _device(med.gamma), u, out)
    assert exc.value.code == lib.NFS_ENOTHPD
    # a non-finite permittivity is a bad argument, as for nfs_setup
    inf_eps = med.eps.copy()
    inf_eps[0, 0, 0, 0] = np.inf
    with pytest.raises(lib.NFSError) as exc:
        lib.matvec_noalloc(g, K, "chiral", (0, 1), _device(inf_eps), _device(med.gamma), u, out)
    assert exc.value.code == lib.NFS_EINVAL
    ctx = lib.Context(g, K, med)
    ref = ctx.matvec(u)
    ctx.close()
    lib.matvec_noalloc(g, K, "chiral", (0, 1), _device(med.eps), _device(med.gamma), u, out)
    err = ((out - ref).abs().max() / ref.abs().max()).item()
    assert err < 1e-12, err


def test_noalloc_rejects_the_gamma_point(lib):
    # k.a_l all integers: Lambda_q vanishes at one voxel (the Lemma)
    g = (16, 16, 16)
    med = wl.chiral_sphere(g)
    u = torch.zeros(4 * 16 ** 3, dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.NFSError) as exc:
        lib.matvec_noalloc(g, (0.0, 0.0, 0.0), "chiral", (0, 1), _device(med.eps), _device(med.gamma), u,
                           torch.empty_like(u))
    assert exc.value.code == lib.NFS_EKPOINT
