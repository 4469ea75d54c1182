"""The C-ABI library builds, loads and exports every symbol include/nfs.h
declares; struct layouts agree with the binding; host-side validation returns
the documented error codes (these checks run before any CUDA call, so they
need no GPU)."""

import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nfs.h")


@pytest.fixture(scope="module")
def nfs():
    from paper_1402_6297_gb300 import build, nfs as binding
    build.build()
    binding.lib()
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfs_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(nfs):
    names = declared_functions()
    assert len(names) >= 12
    L = nfs.lib()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(nfs.EXPORTED) | (set(names) - set(nfs.EXPORTED))
    for name in nfs.EXPORTED:
        assert name in names


def test_struct_layouts_match_header(nfs):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "nfs.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(nfs_options), sizeof(nfs_material), sizeof(nfs_solve_info), sizeof(nfs_eigs_info));
  printf("%zu %zu %zu\n", offsetof(nfs_options, seed), offsetof(nfs_options, stream), offsetof(nfs_eigs_info, max_ritz_residual));
  printf("%zu %zu %zu\n", sizeof(nfs_problem), offsetof(nfs_problem, k), offsetof(nfs_problem, mat));
  printf("%zu %zu %zu %zu\n", sizeof(nfs_biiso_material), sizeof(nfs_nfsep_info),
         offsetof(nfs_nfsep_info, max_ritz_residual), offsetof(nfs_nfsep_info, kernel_launches));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = list(map(int, out))
    assert sizes[0] == ctypes.sizeof(nfs.Options)
    assert sizes[1] == ctypes.sizeof(nfs.Material)
    assert sizes[2] == ctypes.sizeof(nfs.SolveInfo)
    assert sizes[3] == ctypes.sizeof(nfs.EigsInfo)
    assert sizes[4] == nfs.Options.seed.offset
    assert sizes[5] == nfs.Options.stream.offset
    assert sizes[6] == nfs.EigsInfo.max_ritz_residual.offset
    assert sizes[7] == ctypes.sizeof(nfs.Problem)
    assert sizes[8] == nfs.Problem.k.offset
    assert sizes[9] == nfs.Problem.mat.offset
    assert sizes[10] == ctypes.sizeof(nfs.BiisoMaterial)
    assert sizes[11] == ctypes.sizeof(nfs.NfsepInfo)
    assert sizes[12] == nfs.NfsepInfo.max_ritz_residual.offset
    assert sizes[13] == nfs.NfsepInfo.kernel_launches.offset


def test_default_options(nfs):
    o = nfs.default_options()
    assert o.precision == nfs.PREC_FP64
    assert (o.alpha, o.beta) == (2.0, 3.0)
    assert o.cg_tol == 1e-12 and o.eig_tol == 1e-10
    assert o.cg_maxit == 2000 and o.max_restarts == 200 and o.orth_tol == 1e-10
    assert o.deflation_checks == 0 and o.seed == 1 and o.ncv == 0
    assert nfs.lib().nfs_strerror(nfs.NFS_EKPOINT).decode().startswith("k.a_l")


def _setup(nfs, grid, k, med, **opt):
    L = nfs.lib()
    o = nfs.default_options()
    for key, v in opt.items():
        setattr(o, key, v)
    m = nfs.Material()
    m.kind = 0 if med.kind == "chiral" else 1
    m.axis_a, m.axis_b = med.axes
    eps = np.ascontiguousarray(med.eps)
    gam = np.ascontiguousarray(med.gamma)
    m.eps = eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.gamma = gam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.mu = ctypes.POINTER(ctypes.c_double)()
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    kk = np.asarray(k, dtype=np.float64)
    code = L.nfs_setup(ctypes.byref(h), g, None, kk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       ctypes.byref(m), ctypes.byref(o))
    assert not h.value  # these cases never create a context
    return code


def test_validation_errors_without_gpu(nfs):
    g = (8, 8, 8)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    # Lemma: k = 0 (all k.a_l integer) makes Lambda_q singular
    assert _setup(nfs, g, (0.0, 0.0, 0.0), med) == nfs.NFS_EKPOINT
    assert _setup(nfs, g, (1.0, 0.0, 2.0), med) == nfs.NFS_EKPOINT
    # Lemma: alpha dx = beta dy with k1 = k2 = k3 gives Lambda_p = 0 somewhere
    assert _setup(nfs, g, (0.2, 0.2, 0.2), med, alpha=1.0, beta=1.0) == nfs.NFS_EBASIS
    assert _setup(nfs, g, (0.1, 0.2, 0.3), med, alpha=0.0) == nfs.NFS_EBASIS
    # Assumption: Phi = eps - gamma^2 must stay positive
    bad = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 3.7)
    assert _setup(nfs, g, (0.1, 0.2, 0.3), bad) == nfs.NFS_ENOTHPD
    neg = wl.homogeneous(g, eps=-1.0)
    assert _setup(nfs, g, (0.1, 0.2, 0.3), neg) == nfs.NFS_ENOTHPD
    # unsupported sizes and shapes
    assert _setup(nfs, (10, 10, 10), (0.1, 0.2, 0.3), wl.homogeneous((10, 10, 10))) == nfs.NFS_EUNSUPPORTED
    assert _setup(nfs, (8, 16, 8), (0.1, 0.2, 0.3), wl.homogeneous((8, 16, 8))) == nfs.NFS_EUNSUPPORTED
    # bad options
    assert _setup(nfs, g, (0.1, 0.2, 0.3), med, precision=7) == nfs.NFS_EINVAL
    assert _setup(nfs, g, (0.1, 0.2, 0.3), med, cg_tol=0.0) == nfs.NFS_EINVAL
    pc = wl.pseudochiral_cylinders(g, axes=(1, 1))
    assert _setup(nfs, g, (0.1, 0.2, 0.3), pc) == nfs.NFS_EINVAL


def test_null_handles_rejected(nfs):
    L = nfs.lib()
    assert L.nfs_matvec(None, 0, None, None) == nfs.NFS_EINVAL
    assert L.nfs_cg_solve(None, None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_eigs(None, 3, None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_eig_grad(None, 1, None, None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_reserve(None, 3) == nfs.NFS_EINVAL
    assert L.nfs_residuals(None, 1, None, None, None) == nfs.NFS_EINVAL
    L.nfs_destroy(None)


def _batch_code(nfs, problems, **opt):
    """nfs_setup_batch over (grid, k, medium) tuples; returns the code."""
    L = nfs.lib()
    arr = (nfs.Problem * len(problems))()
    keep = []
    for i, (grid, k, med) in enumerate(problems):
        m, kp = nfs._material(med)
        keep.append(kp)
        arr[i].grid[:] = list(grid)
        arr[i].k[:] = list(k)
        arr[i].mat = m
    o = nfs.default_options()
    for key, v in opt.items():
        setattr(o, key, v)
    h = ctypes.c_void_p()
    code = L.nfs_setup_batch(ctypes.byref(h), len(problems), arr, ctypes.byref(o))
    assert not h.value
    return code


def test_batch_validation_errors_without_gpu(nfs):
    """A batch is validated problem by problem on the host before any device
    memory is taken: one bad problem anywhere fails the whole batch."""
    L = nfs.lib()
    g = (8, 8, 8)
    good = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    g16 = (16, 16, 16)
    good16 = wl.chiral_sphere(g16, 0.25, 13.0, 1.0, 0.5)
    ok = [(g, (0.1, 0.2, 0.3), good), (g16, (0.2, 0.1, 0.3), good16)]
    assert _batch_code(nfs, ok + [(g, (0.0, 0.0, 0.0), good)]) == nfs.NFS_EKPOINT
    bad = wl.chiral_sphere(g16, 0.25, 13.0, 1.0, 3.7)
    assert _batch_code(nfs, ok + [(g16, (0.1, 0.2, 0.3), bad)]) == nfs.NFS_ENOTHPD
    assert _batch_code(nfs, ok + [((10, 10, 10), (0.1, 0.2, 0.3), wl.homogeneous((10, 10, 10)))]) \
        == nfs.NFS_EUNSUPPORTED
    assert _batch_code(nfs, ok, cg_tol=-1.0) == nfs.NFS_EINVAL
    h = ctypes.c_void_p()
    assert L.nfs_setup_batch(ctypes.byref(h), 0, None, None) == nfs.NFS_EINVAL
    assert L.nfs_eigs_batch(None, 3, None, None) == nfs.NFS_EINVAL
    assert L.nfs_batch_num_classes(None) == 0
    L.nfs_destroy_batch(None)


def test_kpath_samples_segment_midpoints():
    """The band path of Section 5.3 (G-X-M-R-G, ten samples per segment):
    midpoints of equal subintervals, never a corner (Gamma is singular)."""
    from paper_1402_6297_gb300 import nfs
    ks, arc = nfs.kpath()
    assert ks.shape == (40, 3)
    assert np.all(np.diff(arc) > 0)
    assert np.allclose(ks[0], (0.025, 0.0, 0.0)) and np.allclose(ks[9], (0.475, 0.0, 0.0))
    assert np.allclose(ks[10], (0.5, 0.025, 0.0))
    assert np.allclose(ks[-1], (0.025, 0.025, 0.025))
    corners = np.array(list(nfs.SC_POINTS.values()))
    assert np.min(np.linalg.norm(ks[:, None, :] - corners[None], axis=2)) > 0.02
    ks2, _ = nfs.kpath(("X", (0.5, 0.5, 0.5)), per_segment=4)
    assert np.allclose(ks2[:, 0], 0.5) and np.allclose(ks2[:, 1], ks2[:, 2])


def test_new_entry_points_validate_on_the_host(nfs):
    """Field recovery, GEP residual, band structure and the NFSEP calls reject
    bad arguments before any CUDA call; a singular B (mu eps = zeta xi in some
    voxel, eq. mtx_B) is refused by nfs_setup_biiso."""
    L = nfs.lib()
    assert L.nfs_eig_fields(None, 1, None, None) == nfs.NFS_EINVAL
    assert L.nfs_gep_residual(None, 1, None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_nfsep_matvec(None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_nfsep_eigs(None, 2, None, None, None, None) == nfs.NFS_EINVAL
    assert L.nfs_nfsep_fields(None, 1, None, None) == nfs.NFS_EINVAL
    g = (8, 8, 8)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    m, keep = nfs._material(med)
    gi = (ctypes.c_int * 3)(*g)
    k = np.array([[0.1, 0.2, 0.3]])
    om = np.zeros(4)
    assert L.nfs_band_structure(gi, ctypes.byref(m), 0, nfs._dptr(k), None, 4, 0, nfs._dptr(om), None, None) \
        == nfs.NFS_EINVAL
    assert L.nfs_band_structure(gi, ctypes.byref(m), 1, nfs._dptr(k), None, 0, 0, nfs._dptr(om), None, None) \
        == nfs.NFS_EINVAL
    o = nfs.default_options()
    o.deflation_checks = -1
    assert L.nfs_band_structure(gi, ctypes.byref(m), 1, nfs._dptr(k), ctypes.byref(o), 4, 0, nfs._dptr(om),
                                None, None) == nfs.NFS_EINVAL
    # singular B: chi = 1 with eps = mu = 1, gamma = 0 gives zeta xi = mu eps
    sing = wl.biisotropic_sphere(g, 0.25, 1.0, 1.0, 0.0, 1.0)
    arrs = [np.ascontiguousarray(a, dtype=np.complex128) for a in (sing.eps, sing.mu, sing.gamma, sing.chi)]
    bm = nfs.BiisoMaterial()
    for name, a in zip(("eps", "mu", "gamma", "chi"), arrs):
        setattr(bm, name, a.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    h = ctypes.c_void_p()
    kv = np.array([0.1, 0.2, 0.3])
    assert L.nfs_setup_biiso(ctypes.byref(h), gi, None, nfs._dptr(kv), ctypes.byref(bm), None) == nfs.NFS_EINVAL
    assert not h.value
    # the binding refuses media the library does not solve
    with pytest.raises(ValueError):
        nfs._material(wl.biisotropic_sphere(g, 0.25, 13.0 + 1j, 1.0, 0.5, 0.0))
    with pytest.raises(ValueError):
        nfs.NFSEPContext(g, (0.1, 0.2, 0.3), med)


def test_non_finite_inputs_are_refused(nfs):
    """Fault injection on the host: NaN or infinite material values and Bloch
    vectors are rejected by the set-up before any device memory is taken."""
    g = (8, 8, 8)
    med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
    for field, value, code in (("eps", np.nan, nfs.NFS_ENOTHPD), ("eps", np.inf, nfs.NFS_ENOTHPD),
                               ("gamma", np.nan, nfs.NFS_EINVAL), ("gamma", np.inf, nfs.NFS_EINVAL)):
        bad = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
        getattr(bad, field)[1, 2, 3, 4] = value
        assert _setup(nfs, g, (0.1, 0.2, 0.3), bad) == code, (field, value)
    assert _setup(nfs, g, (0.1, np.nan, 0.3), med) == nfs.NFS_EINVAL
    assert _setup(nfs, g, (np.inf, 0.2, 0.3), med) == nfs.NFS_EINVAL
    # bi-isotropic: a NaN anywhere makes B's determinant non-finite
    L = nfs.lib()
    sph = wl.biisotropic_sphere(g, 0.25, 13.0 + 2.0j, 1.0, 0.5, 0.2)
    sph.eps[0, 0, 0, 0] = complex(np.nan, 0.0)
    arrs = [np.ascontiguousarray(a, dtype=np.complex128) for a in (sph.eps, sph.mu, sph.gamma, sph.chi)]
    bm = nfs.BiisoMaterial()
    for name, a in zip(("eps", "mu", "gamma", "chi"), arrs):
        setattr(bm, name, a.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    h = ctypes.c_void_p()
    gi = (ctypes.c_int * 3)(*g)
    kv = np.array([0.1, 0.2, 0.3])
    assert L.nfs_setup_biiso(ctypes.byref(h), gi, None, nfs._dptr(kv), ctypes.byref(bm), None) == nfs.NFS_EINVAL
