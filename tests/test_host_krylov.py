"""The host Krylov drivers of the non-Hermitian null space free problem
(restarted GMRES, Krylov-Schur Arnoldi, shift-and-invert Arnoldi), run on
host vectors through a test shim, against LAPACK through numpy, and on the
oracle's dense NFSEP operator of a lossy bi-isotropic medium (eq.
NFSEP_org)."""

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import workloads as wl
from oracle import nfsep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kl():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "kshim.so")
    csrc = os.path.join(ROOT, "paper_1402_6297_gb300", "csrc")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           os.path.join(ROOT, "tests", "shim", "krylov_shim.cpp"),
                           os.path.join(csrc, "krylov.cpp"), os.path.join(csrc, "host_zeig.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    P = ctypes.POINTER(ctypes.c_double)
    IP = ctypes.POINTER(ctypes.c_int)
    d_, i_ = ctypes.c_double, ctypes.c_int
    L.shim_gmres.argtypes = [i_, P, d_, d_, P, P, i_, d_, i_, IP, P]
    L.shim_krylov_schur.argtypes = [i_, P, i_, i_, d_, i_, ctypes.c_uint, P, P, IP, IP]
    L.shim_shift_invert.argtypes = [i_, P, d_, d_, i_, i_, d_, i_, d_, ctypes.c_uint, P, IP, IP]
    L.shim_krylov_schur_from.argtypes = [i_, P, P, i_, i_, d_, i_, P, IP, IP]
    return L


def cp(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def match(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


def test_gmres(kl):
    rng = np.random.default_rng(1)
    N = 150
    A = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N) + 3 * np.eye(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    sigma = 0.5 - 0.25j
    Ac, Ap = cp(A)
    bc, bp = cp(b)
    x = np.zeros(N, complex)
    xc, xp = cp(x)
    its, rel = ctypes.c_int(), ctypes.c_double()
    for m in (10, 40):  # restarted and not
        rc = kl.shim_gmres(N, Ap, sigma.real, sigma.imag, bp, xp, m, 1e-12, 5000, ctypes.byref(its),
                           ctypes.byref(rel))
        assert rc == 0
        ref = np.linalg.solve(A - sigma * np.eye(N), b)
        assert np.linalg.norm(xc - ref) < 1e-10 * np.linalg.norm(ref)
        assert rel.value <= 1e-12


def test_krylov_schur_largest_modulus(kl):
    rng = np.random.default_rng(2)
    N = 200
    A = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N)
    A[np.arange(6), np.arange(6)] += np.array([4, 3.5j, -3.2, 2.9 + 1j, -2.7j, 2.5])
    Ac, Ap = cp(A)
    nev = 6
    th = np.zeros(nev, complex)
    thc, thp = cp(th)
    Y = np.zeros((nev, N), complex)
    Yc, Yp = cp(Y)
    steps, rst = ctypes.c_int(), ctypes.c_int()
    rc = kl.shim_krylov_schur(N, Ap, nev, 20, 1e-12, 200, 7, thp, Yp, ctypes.byref(steps), ctypes.byref(rst))
    assert rc == 0
    assert rst.value >= 1  # the basis of 20 had to restart
    ev = np.linalg.eigvals(A)
    ref = ev[np.argsort(-np.abs(ev))[:nev]]
    assert match(thc, ref) < 1e-10
    assert np.all(np.diff(np.abs(thc)) <= 1e-12)
    for e in range(nev):
        assert np.linalg.norm(A @ Yc[e] - thc[e] * Yc[e]) < 1e-9
        assert abs(np.linalg.norm(Yc[e]) - 1) < 1e-12


def test_shift_invert_on_the_oracle_nfsep(kl):
    """Shift-and-invert Arnoldi (Section 4) with GMRES inner solves on M of
    eq. NFSEP_org for a lossy bi-isotropic sphere: the eigenvalues nearest
    the shift equal the dense ones."""
    g, k = (4, 3, 5), (0.1, 0.2, 0.3)
    med = wl.biisotropic_sphere(g, 0.3, 13.0 + 2.0j, 1.0, 0.5, 0.2)
    M = nfsep.NFSEP(g, k, med).dense()
    N = M.shape[0]
    w = np.linalg.eigvals(M)
    sigma = 0.6 * np.sort(np.abs(w))[8] * (1 + 0.1j)
    Mc, Mp = cp(M)
    nev = 5
    lam = np.zeros(nev, complex)
    lc, lp = cp(lam)
    steps, inner = ctypes.c_int(), ctypes.c_int()
    rc = kl.shim_shift_invert(N, Mp, sigma.real, sigma.imag, nev, 16, 1e-11, 60, 1e-13, 3, lp,
                              ctypes.byref(steps), ctypes.byref(inner))
    assert rc == 0
    ref = w[np.argsort(np.abs(w - sigma))[:nev]]
    assert match(lc, ref) < 1e-9 * np.abs(ref).max()
    assert inner.value > steps.value


def test_krylov_schur_leaves_an_invariant_subspace(kl):
    """A start vector inside an invariant subspace (the first block of a
    block-diagonal matrix) makes h_{j+1,j} vanish after a few steps; the
    driver continues from a random direction and still finds the eigenvalues
    of largest modulus, which all lie in the other block."""
    rng = np.random.default_rng(4)
    k, N = 6, 120
    A = np.zeros((N, N), complex)
    A[:k, :k] = 0.3 * (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    B = (rng.standard_normal((N - k, N - k)) + 1j * rng.standard_normal((N - k, N - k))) / np.sqrt(N)
    B[np.arange(4), np.arange(4)] += np.array([5.0, -4.5, 4.0j, 3.5])
    A[k:, k:] = B
    v0 = np.zeros(N, complex)
    v0[:k] = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    Ac, Ap = cp(A)
    vc, vp = cp(v0)
    nev = 4
    th = np.zeros(nev, complex)
    thc, thp = cp(th)
    steps, inj = ctypes.c_int(), ctypes.c_int()
    rc = kl.shim_krylov_schur_from(N, Ap, vp, nev, 24, 1e-12, 100, thp, ctypes.byref(steps), ctypes.byref(inj))
    assert rc == 0
    assert inj.value >= 1
    ev = np.linalg.eigvals(A)
    ref = ev[np.argsort(-np.abs(ev))[:nev]]
    assert match(thc, ref) < 1e-10


def test_gmres_reports_non_convergence(kl):
    """A product cap below what the system needs ends GMRES with NFS_ENOCONV
    (-6) and the residual reached so far."""
    rng = np.random.default_rng(6)
    N = 120
    A = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N) + 1.5 * np.eye(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Ac, Ap = cp(A)
    bc, bp = cp(b)
    x = np.zeros(N, complex)
    xc, xp = cp(x)
    its, rel = ctypes.c_int(), ctypes.c_double()
    rc = kl.shim_gmres(N, Ap, 0.0, 0.0, bp, xp, 5, 1e-14, 10, ctypes.byref(its), ctypes.byref(rel))
    assert rc == -6
    assert its.value == 10
    assert 1e-14 < rel.value < 1.0
    assert abs(np.linalg.norm(b - A @ xc) / np.linalg.norm(b) - rel.value) < 1e-12
