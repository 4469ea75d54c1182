"""Batched eigensolves (nfs_setup_batch / nfs_eigs_batch) against the oracle
and against one-problem contexts.

A batch groups problems by grid, medium kind, axis pair and mu-ness; each
group runs in lock-step through single kernel launches, and the groups run
concurrently.  The eigenvalues of every problem must not depend on which
batch it was solved in: within 1e-10 relative of the oracle on the FP64 path
and 1e-8 on the mixed path, and within the same bounds of a one-problem
context."""

import numpy as np
import pytest

import workloads as wl
from oracle import gep, nfgep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nfs(lib):
    return lib


def _sphere(g, gamma, radius=0.25):
    return wl.chiral_sphere(g, radius, 13.0, 1.0, gamma)


def test_batch_same_grid_vs_dense_oracle(nfs):
    """Four 8^3 chiral spheres at four k-points of G-X-M-R-G: FP64 batch vs
    the dense pencil eigensolve (oracle tier O1)."""
    g = (8, 8, 8)
    ks = wl.bz_path_midpoints(4)
    gams = [0.3, 0.5, 0.7, 0.2]
    probs = [(g, tuple(k), _sphere(g, gm)) for k, gm in zip(ks, gams)]
    nev = 8
    with nfs.Batch(probs, precision="fp64") as b:
        assert b.num_classes == 1
        omega, infos = b.eigs(nev)
    for i, (_, k, med) in enumerate(probs):
        w, _, idx = gep.dense_eigs(g, k, med, nev)
        ref = w[idx]
        assert np.abs(omega[i] - ref).max() / ref.min() < 1e-10, i
        assert infos[i].nconv == nev and infos[i].status == nfs.NFS_OK


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_batch_mixed_classes_equal_single_contexts(nfs, precision, tol):
    """Three classes (16^3 chiral, 8^3 pseudochiral, 12x12x16 chiral) with
    uneven class sizes; each problem vs the same problem in its own context."""
    ks = wl.bz_path_midpoints(7)
    probs = []
    for j in range(3):
        g = (16, 16, 16)
        probs.append((g, tuple(ks[j]), _sphere(g, 0.3 + 0.2 * j)))
    for j in range(2):
        g = (8, 8, 8)
        probs.append((g, tuple(ks[3 + j]), wl.pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), seed=j)))
    g = (12, 12, 16)
    probs.append((g, tuple(ks[5]), wl.smoothed_chiral_field(g, seed=4, sigma=0.15)))
    # interleave the classes in the input order
    order = [0, 3, 1, 5, 4, 2]
    probs = [probs[i] for i in order]
    nev = 6
    with nfs.Batch(probs, precision=precision) as b:
        assert b.num_classes == 3
        omega, infos = b.eigs(nev)
    for i, (g, k, med) in enumerate(probs):
        ctx = nfs.Context(g, k, med, precision=precision)
        ref, Y, _ = ctx.eigs(nev)
        ctx.close()
        assert np.abs(omega[i] - ref).max() / ref.min() < tol, (i, omega[i], ref)
        assert infos[i].nconv == nev


def test_batch_mixed_residuals_through_single_context(nfs):
    """The mixed batch's eigenvalues are those of each problem's FP64 pencil:
    16^3 spheres at 5 k-points vs the oracle's NSF eigensolve (tier O3)."""
    g = (16, 16, 16)
    ks = wl.bz_path_midpoints(5)
    probs = [(g, tuple(k), _sphere(g, 0.5)) for k in ks]
    nev = 5
    with nfs.Batch(probs, precision="mixed") as b:
        omega, infos = b.eigs(nev)
    for i in (0, 2, 4):
        _, k, med = probs[i]
        ref, _ = nfgep.NFGEP(g, k, med).eigs(nev)
        assert np.abs(omega[i] - ref).max() / ref.min() < 1e-8, i
    assert all(inf.max_ritz_residual >= 0 for inf in infos)


def test_batch_of_one_equals_context(nfs):
    w = wl.workload("sphere8")
    with nfs.Batch([(w["grid"], w["kdota"], w["medium"])], precision="fp64") as b:
        omega, _ = b.eigs(10)
    ctx = nfs.Context(w["grid"], w["kdota"], w["medium"], precision="fp64")
    ref, _, _ = ctx.eigs(10, vectors=False)
    ctx.close()
    assert np.abs(omega[0] - ref).max() / ref.min() < 1e-12


def test_batch_with_restarts_equals_single_contexts(nfs):
    """A small basis (ncv 30 for nev 10) forces thick restarts; problems that
    restart in lock-step inside a batch must give what each gives alone with
    the same basis size."""
    g = (16, 16, 16)
    ks = wl.bz_path_midpoints(9)
    probs = [(g, tuple(ks[j]), _sphere(g, 0.3 + 0.1 * j)) for j in (1, 4, 7)]
    nev = 10
    with nfs.Batch(probs, precision="mixed", ncv=30) as b:
        omega, infos = b.eigs(nev)
    assert max(i.restarts for i in infos) > 0
    for i, (gg, k, med) in enumerate(probs):
        ctx = nfs.Context(gg, k, med, precision="mixed", ncv=30)
        ref, _, info = ctx.eigs(nev, vectors=False)
        ctx.close()
        assert info.restarts == infos[i].restarts
        assert np.abs((omega[i] - ref) / ref).max() < 1e-12, (i, omega[i], ref)
