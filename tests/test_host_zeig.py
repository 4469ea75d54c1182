"""The host complex Schur routines (for the Arnoldi projected matrices of the
non-Hermitian null space free problem) against LAPACK through numpy: the
decomposition A = Q T Q^*, unitarity, triangularity and the eigenvalues on
random, Hessenberg, real (conjugate pairs), normal-with-repeated-eigenvalue
and graded matrices; the reordering; the eigenvectors."""

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zl():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "zshim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                           os.path.join(ROOT, "tests", "shim", "host_zeig_shim.cpp"),
                           os.path.join(ROOT, "paper_1402_6297_gb300", "csrc", "host_zeig.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    P = ctypes.POINTER(ctypes.c_double)
    IP = ctypes.POINTER(ctypes.c_int)
    L.shim_complex_schur.argtypes = [ctypes.c_int, P, P, P]
    L.shim_schur_reorder.argtypes = [ctypes.c_int, P, P, IP]
    L.shim_triangular_eigvecs.argtypes = [ctypes.c_int, P, P]

    def ptr(a):
        return a.ctypes.data_as(P)

    def schur(A):
        m = A.shape[0]
        a = np.ascontiguousarray(A, dtype=np.complex128)
        T = np.zeros_like(a)
        Q = np.zeros_like(a)
        rc = L.shim_complex_schur(m, ptr(a.view(np.float64)), ptr(T.view(np.float64)), ptr(Q.view(np.float64)))
        assert rc == 0
        return T, Q

    def reorder(T, Q, sel):
        T = np.ascontiguousarray(T.copy())
        Q = np.ascontiguousarray(Q.copy())
        s = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
        L.shim_schur_reorder(T.shape[0], ptr(T.view(np.float64)), ptr(Q.view(np.float64)), s.ctypes.data_as(IP))
        return T, Q

    def eigvecs(T):
        T = np.ascontiguousarray(T, dtype=np.complex128)
        V = np.zeros_like(T)
        L.shim_triangular_eigvecs(T.shape[0], ptr(T.view(np.float64)), ptr(V.view(np.float64)))
        return V

    return schur, reorder, eigvecs


def match(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


def matrices():
    rng = np.random.default_rng(5)
    out = []
    for m in (1, 2, 3, 7, 20, 61, 150):
        out.append(("random", rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))))
    for m in (5, 40):
        out.append(("real", rng.standard_normal((m, m))))
        H = np.triu(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)), -1)
        out.append(("hessenberg", H))
        U, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
        lam = rng.standard_normal(m // 4 + 1) + 1j * rng.standard_normal(m // 4 + 1)
        out.append(("normal_repeated", U @ np.diag(np.resize(lam, m)) @ U.conj().T))
        out.append(("graded", (rng.standard_normal((m, m)) + 0j) * np.logspace(0, -8, m)[None, :]))
    out.append(("diagonal", np.diag(np.arange(6, dtype=complex))))
    out.append(("zero", np.zeros((4, 4), complex)))
    return out


@pytest.mark.parametrize("name,A", matrices(), ids=[f"{n}{a.shape[0]}" for n, a in matrices()])
def test_schur(zl, name, A):
    schur, _, _ = zl
    T, Q = schur(A)
    m = A.shape[0]
    nrm = max(np.abs(A).max(), 1e-300)
    assert np.abs(np.tril(T, -1)).max(initial=0.0) == 0.0
    assert np.abs(Q.conj().T @ Q - np.eye(m)).max() < 1e-13 * m
    assert np.abs(Q @ T @ Q.conj().T - A).max() < 1e-13 * m * nrm
    assert match(np.diag(T), np.linalg.eigvals(A)) < 1e-9 * max(nrm, 1.0) * m


def test_reorder_and_eigenvectors(zl):
    schur, reorder, eigvecs = zl
    rng = np.random.default_rng(9)
    m = 30
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    T, Q = schur(A)
    lam = np.diag(T).copy()
    sel = (np.abs(lam) > np.median(np.abs(lam))).astype(int)
    T2, Q2 = reorder(T, Q, sel)
    k = int(sel.sum())
    assert np.abs(np.tril(T2, -1)).max() == 0.0
    assert np.abs(Q2.conj().T @ Q2 - np.eye(m)).max() < 1e-13 * m
    assert np.abs(Q2 @ T2 @ Q2.conj().T - A).max() < 1e-12 * m * np.abs(A).max()
    assert match(np.diag(T2)[:k], lam[sel == 1]) < 1e-10 * np.abs(lam).max()
    # the selected ones keep their order
    assert np.abs(np.diag(T2)[:k] - lam[sel == 1]).max() < 1e-9 * np.abs(lam).max()
    V = eigvecs(T2)
    X = Q2 @ V
    for j in range(m):
        r = A @ X[:, j] - T2[j, j] * X[:, j]
        assert np.linalg.norm(r) < 1e-10 * np.abs(A).max() * m
        assert abs(np.linalg.norm(X[:, j]) - 1) < 1e-12
