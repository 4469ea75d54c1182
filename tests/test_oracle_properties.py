"""Property checks of the oracle over random tiny problems (grid, Bloch
vector, medium drawn by hypothesis): the identities the paper fixes hold for
every draw, not only for the hand-picked cases of the other pin files.

* C = P_r Sigma_r Q_r^* (thm:svd_C) and Q, P unitary;
* A_r Hermitian positive definite under the Assumption (thm:NFSEP_real_ew)
  and its FFT form equal to the dense eq. (factor_mtx);
* the HHPD-NFGEP and the NFSEP (thm:nfep) have exactly the GEP's nonzero
  eigenvalues."""

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import linear_sum_assignment

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import workloads as wl  # noqa: E402
from oracle import gep, nfgep, nfsep, yee  # noqa: E402


def match(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


@st.composite
def problems(draw):
    n12 = draw(st.integers(2, 4))
    n3 = draw(st.integers(2, 4))
    g = (n12, n12, n3)
    # k.a_l in (0, 1) away from the integers (Gamma excluded by the Lemma)
    k = tuple(draw(st.floats(0.05, 0.95)) for _ in range(3))
    seed = draw(st.integers(0, 10_000))
    rng = np.random.default_rng(seed)
    shape = (3, n3, n12, n12)
    eps = 1.0 + 12.0 * rng.random(shape)
    kind = draw(st.sampled_from(["chiral", "pseudochiral"]))
    if kind == "chiral":
        gam = 0.8 * np.sqrt(eps.min()) * (rng.random(shape) - 0.5)
        med = wl.Medium(g, wl.media.CHIRAL, eps, gam)
    else:
        gam = 0.8 * (rng.random((n3, n12, n12)) - 0.5)
        axes = draw(st.sampled_from([(0, 1), (0, 2), (1, 2)]))
        med = wl.Medium(g, wl.media.PSEUDOCHIRAL, eps, gam, None, axes)
    return g, k, med


@settings(max_examples=25, deadline=None)
@given(problems())
def test_svd_of_the_curl(p):
    g, k, _ = p
    sym = yee.Symbols(g, k)
    Pr, Sr, Qr = yee.dense_svd_factors(sym)
    C = yee.curl_matrix(g, k).toarray()
    assert np.abs(Pr @ np.diag(Sr) @ Qr.conj().T - C).max() < 1e-10 * np.abs(C).max()
    assert np.abs(Pr.conj().T @ Pr - np.eye(Pr.shape[1])).max() < 1e-10
    assert np.abs(Qr.conj().T @ Qr - np.eye(Qr.shape[1])).max() < 1e-10


@settings(max_examples=25, deadline=None)
@given(problems())
def test_ar_hpd_and_fft_form(p):
    g, k, med = p
    nf = nfgep.NFGEP(g, k, med)
    A = nf.dense_Ar()
    assert np.abs(A - A.conj().T).max() < 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    u = wl.random_complex(4 * nf.n, 3)
    assert np.abs(nf.Ar(u) - A @ u).max() < 1e-12 * np.abs(A @ u).max()


@settings(max_examples=20, deadline=None)
@given(problems())
def test_both_null_space_free_problems_have_the_gep_spectrum(p):
    g, k, med = p
    L, B = gep.gep_matrices(g, k, med)
    ev = sla.eigvals(L.toarray(), B.toarray())
    scale = np.abs(ev[np.isfinite(ev)]).max()
    nz = ev[np.abs(ev) > 1e-8 * scale]
    nf = nfgep.NFGEP(g, k, med)
    th = sla.eigh(nf.dense_Br(), nf.dense_Ar(), eigvals_only=True)
    assert nz.size == th.size
    assert match(1.0 / th + 0j, nz) < 1e-8 * scale
    w = np.linalg.eigvals(nfsep.NFSEP(g, k, med).dense())
    assert match(w, nz) < 1e-8 * scale
