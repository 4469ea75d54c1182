"""The Lanczos driver's host eigensolver (Householder + implicit QR) against
LAPACK on the matrix shapes it meets: tridiagonal, tridiagonal with an arrow
(after a thick restart), dense random, and clusters of equal eigenvalues."""

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sym_eig():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "shim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           os.path.join(ROOT, "tests", "shim", "host_eig_shim.cpp"),
                           os.path.join(ROOT, "paper_1402_6297_gb300", "csrc", "host_eig.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    P = ctypes.POINTER(ctypes.c_double)
    L.shim_sym_eig.argtypes = [ctypes.c_int, P, P, P]
    L.shim_sym_eig_last_row.argtypes = [ctypes.c_int, P, P, P]

    def run(A):
        m = A.shape[0]
        A = np.ascontiguousarray(A, dtype=np.float64)
        w = np.zeros(m)
        Z = np.zeros((m, m))
        rc = L.shim_sym_eig(m, A.ctypes.data_as(P), w.ctypes.data_as(P), Z.ctypes.data_as(P))
        assert rc == 0
        w2 = np.zeros(m)
        zl = np.zeros(m)
        rc = L.shim_sym_eig_last_row(m, A.ctypes.data_as(P), w2.ctypes.data_as(P), zl.ctypes.data_as(P))
        assert rc == 0
        # the last-row mode gives the same eigenvalues and the last row of Z
        assert np.array_equal(w2, w)
        assert np.abs(zl - Z[-1]).max() < 1e-13
        return w, Z
    return run


def check(sym_eig, A):
    w, Z = sym_eig(A)
    ref = np.linalg.eigvalsh(A)
    scale = max(np.abs(ref).max(), 1.0)
    assert np.abs(w - ref).max() < 1e-12 * scale
    assert np.abs(Z.T @ Z - np.eye(len(w))).max() < 1e-12
    assert np.abs(A @ Z - Z * w).max() < 1e-11 * scale


def test_tridiagonal(sym_eig):
    rng = np.random.default_rng(0)
    for m in (1, 2, 3, 10, 61, 160):
        a, b = rng.standard_normal(m), rng.standard_normal(m - 1)
        check(sym_eig, np.diag(a) + np.diag(b, 1) + np.diag(b, -1))


def test_arrow_plus_tridiagonal(sym_eig):
    rng = np.random.default_rng(1)
    m, k = 60, 35
    A = np.zeros((m, m))
    A[np.arange(k), np.arange(k)] = np.sort(rng.standard_normal(k))
    A[k, :k] = A[:k, k] = 1e-3 * rng.standard_normal(k)
    t = rng.standard_normal(m - k)
    A[np.arange(k, m), np.arange(k, m)] = t
    s = rng.standard_normal(m - k - 1)
    A[np.arange(k, m - 1), np.arange(k + 1, m)] = s
    A[np.arange(k + 1, m), np.arange(k, m - 1)] = s
    check(sym_eig, A)


def test_dense_and_clustered(sym_eig):
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 40))
    check(sym_eig, M + M.T)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.repeat([1.0, 2.0, 2.0 + 1e-13, 5.0, -3.0], 6)
    check(sym_eig, Q @ np.diag(lam) @ Q.T)
    check(sym_eig, np.zeros((5, 5)))


def test_locked_block_with_coinciding_tridiagonal(sym_eig):
    """The projected matrix of a deflation check: the locked Ritz values on
    the diagonal (repeated, as in a degenerate cluster), decoupled from a
    Lanczos tridiagonal whose eigenvalues include the locked ones (the copies
    the check is looking for)."""
    rng = np.random.default_rng(3)
    lam = np.concatenate([[0.7767] * 3, [0.6957] * 3, 0.4 * rng.random(200)])
    n = lam.size
    for steps in (5, 20, 60):
        v = rng.standard_normal(n)
        V = [v / np.linalg.norm(v)]
        a, b = [], []
        for j in range(steps):
            w = lam * V[-1]
            for _ in range(2):
                for u in V:
                    w -= (u @ w) * u
            a.append(V[-1] @ (lam * V[-1]))
            if j < steps - 1:
                b.append(np.linalg.norm(w))
                V.append(w / b[-1])
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        k = 8
        A = np.zeros((k + steps, k + steps))
        A[np.arange(k), np.arange(k)] = [0.7767] * 4 + [0.6957] * 4
        A[k:, k:] = T
        check(sym_eig, A)
