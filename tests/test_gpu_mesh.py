"""Mesh convergence (Section 5.1, third validation; Fig. diff_mesh): the three
smallest eigenvalues of the chiral sphere (eps_i, eps_o, gamma) = (13, 1, 0.5)
at k = (0.5, 0, 0) on n^3 grids.  The GPU values equal the oracle's stored
ones (tests/golden/mesh_sphere_omega.txt) at every stored n, and the
differences between successive grids shrink as n grows."""

import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = (0.5, 0.0, 0.0)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mesh_sphere_omega.txt")


def test_mesh_convergence(lib):
    rows = np.loadtxt(GOLDEN)
    golden = {int(r[0]): r[1:] for r in rows}
    vals = {}
    for n in (8, 16, 24, 32, 64):
        g = (n, n, n)
        med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
        ctx = lib.Context(g, K, med, precision="mixed")
        om, _, _ = ctx.eigs(3, vectors=False)
        ctx.close()
        vals[n] = om
        if n in golden:
            assert np.abs(om - golden[n]).max() < 1e-8 * golden[n].max(), (n, om, golden[n])
    d_coarse = np.abs(vals[16] - vals[8]).max()
    d_fine = np.abs(vals[64] - vals[32]).max()
    assert d_fine < d_coarse
