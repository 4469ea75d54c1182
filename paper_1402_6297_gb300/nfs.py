"""ctypes binding of libnfs (include/nfs.h): argument marshalling only.

Every numerical step runs in the CUDA library.  PyTorch supplies device
memory and the stream; tensors crossing the boundary are CUDA tensors of
dtype complex128 (NFS_C128) or complex64 (NFS_C64), 4n elements, laid out
[u1a | u1b | u2a | u2b] in spectral order (see the header).

If the library has not been built the first call raises ``NFSLibraryMissing``;
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libnfs.so")

NFS_OK = 0
NFS_EINVAL = -1
NFS_EUNSUPPORTED = -2
NFS_EKPOINT = -3
NFS_EBASIS = -4
NFS_ENOTHPD = -5
NFS_ENOCONV = -6
NFS_EBREAKDOWN = -7
NFS_ETIMEOUT = -8
NFS_ECUDA = -9
NFS_ENOMEM = -10

MEDIUM_CHIRAL = 0
MEDIUM_PSEUDOCHIRAL = 1
PREC_FP64 = 0
PREC_MIXED = 1
C128 = 0
C64 = 1
C128_DS = 2

EXPORTED = (
    "nfs_default_options", "nfs_setup", "nfs_matvec", "nfs_matvec_passes", "nfs_apply_Br", "nfs_cg_solve",
    "nfs_eigs", "nfs_eig_grad", "nfs_num_voxels", "nfs_device_bytes", "nfs_set_stream",
    "nfs_destroy", "nfs_strerror", "nfs_matvec_noalloc",
    "nfs_setup_batch", "nfs_eigs_batch", "nfs_batch_num_classes", "nfs_destroy_batch",
    "nfs_eig_fields", "nfs_gep_residual", "nfs_band_structure",
    "nfs_setup_biiso", "nfs_nfsep_matvec", "nfs_nfsep_eigs", "nfs_nfsep_fields",
    "nfs_residuals", "nfs_reserve",
)
NOALLOC_MAX_VOXELS = 32768


class NFSLibraryMissing(RuntimeError):
    pass


class NFSError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {_strerror(code)} (code {code})")


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("cg_tol", ctypes.c_double),
        ("cg_maxit", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("max_refine", ctypes.c_int),
        ("eig_tol", ctypes.c_double),
        ("ncv", ctypes.c_int),
        ("max_restarts", ctypes.c_int),
        ("orth_tol", ctypes.c_double),
        ("deflation_checks", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("stream", ctypes.c_void_p),
    ]


class Material(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("axis_a", ctypes.c_int),
        ("axis_b", ctypes.c_int),
        ("eps", ctypes.POINTER(ctypes.c_double)),
        ("mu", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.POINTER(ctypes.c_double)),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("refinements", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("status", ctypes.c_int),
    ]


class EigsInfo(ctypes.Structure):
    _fields_ = [
        ("lanczos_steps", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("cg_iterations", ctypes.c_longlong),
        ("matvecs_c64", ctypes.c_longlong),
        ("matvecs_c128", ctypes.c_longlong),
        ("nconv", ctypes.c_int),
        ("max_ritz_residual", ctypes.c_double),
        ("status", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong),
        ("seconds_total", ctypes.c_double),
        ("seconds_cg", ctypes.c_double),
        ("seconds_refine", ctypes.c_double),
        ("seconds_ritz", ctypes.c_double),
        ("seconds_recurrence", ctypes.c_double),
        ("seconds_orth", ctypes.c_double),
        ("seconds_vectors", ctypes.c_double),
        ("reorthogonalisations", ctypes.c_int),
        ("deflation_checks", ctypes.c_int),
    ]


class BiisoMaterial(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.POINTER(ctypes.c_double)),
        ("mu", ctypes.POINTER(ctypes.c_double)),
        ("gamma", ctypes.POINTER(ctypes.c_double)),
        ("chi", ctypes.POINTER(ctypes.c_double)),
    ]


class NfsepInfo(ctypes.Structure):
    _fields_ = [
        ("arnoldi_steps", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("gmres_iterations", ctypes.c_longlong),
        ("nconv", ctypes.c_int),
        ("max_ritz_residual", ctypes.c_double),
        ("status", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong),
    ]


class Problem(ctypes.Structure):
    _fields_ = [
        ("grid", ctypes.c_int * 3),
        ("k", ctypes.c_double * 3),
        ("mat", Material),
    ]


_lib = None


def lib():
    """Load libnfs.so (once).  Raises NFSLibraryMissing if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise NFSLibraryMissing(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.nfs_default_options.argtypes = [ctypes.POINTER(Options)]
    L.nfs_default_options.restype = None
    L.nfs_setup.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Material), ctypes.POINTER(Options)]
    L.nfs_setup.restype = ip
    L.nfs_matvec.argtypes = [vp, ip, vp, vp]
    L.nfs_matvec.restype = ip
    L.nfs_matvec_passes.argtypes = [vp, ip, ip, vp, vp]
    L.nfs_matvec_passes.restype = ip
    L.nfs_apply_Br.argtypes = [vp, vp, vp]
    L.nfs_apply_Br.restype = ip
    L.nfs_cg_solve.argtypes = [vp, vp, vp, ctypes.POINTER(SolveInfo)]
    L.nfs_cg_solve.restype = ip
    L.nfs_eigs.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), vp, ctypes.POINTER(EigsInfo)]
    L.nfs_eigs.restype = ip
    L.nfs_reserve.argtypes = [vp, ip]
    L.nfs_reserve.restype = ip
    L.nfs_residuals.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), vp, ctypes.POINTER(ctypes.c_double)]
    L.nfs_residuals.restype = ip
    L.nfs_eig_grad.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), vp, vp, vp]
    L.nfs_eig_grad.restype = ip
    L.nfs_eig_fields.argtypes = [vp, ip, vp, vp]
    L.nfs_eig_fields.restype = ip
    L.nfs_gep_residual.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), vp, ctypes.POINTER(ctypes.c_double)]
    L.nfs_gep_residual.restype = ip
    L.nfs_setup_biiso.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(BiisoMaterial),
                                  ctypes.POINTER(Options)]
    L.nfs_setup_biiso.restype = ip
    L.nfs_nfsep_matvec.argtypes = [vp, vp, vp]
    L.nfs_nfsep_matvec.restype = ip
    L.nfs_nfsep_eigs.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp,
                                 ctypes.POINTER(NfsepInfo)]
    L.nfs_nfsep_eigs.restype = ip
    L.nfs_nfsep_fields.argtypes = [vp, ip, vp, vp]
    L.nfs_nfsep_fields.restype = ip
    L.nfs_num_voxels.argtypes = [vp]
    L.nfs_num_voxels.restype = ctypes.c_longlong
    L.nfs_device_bytes.argtypes = [vp]
    L.nfs_device_bytes.restype = ctypes.c_longlong
    L.nfs_set_stream.argtypes = [vp, vp]
    L.nfs_set_stream.restype = ip
    L.nfs_destroy.argtypes = [vp]
    L.nfs_destroy.restype = None
    L.nfs_matvec_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ip, ip, ip,
                                      vp, vp, dp, dp, vp, vp, vp]
    L.nfs_matvec_noalloc.restype = ip
    L.nfs_setup_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(Problem), ctypes.POINTER(Options)]
    L.nfs_setup_batch.restype = ip
    L.nfs_eigs_batch.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(EigsInfo)]
    L.nfs_eigs_batch.restype = ip
    L.nfs_band_structure.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Material), ip,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Options), ip, ip,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(EigsInfo),
                                     ctypes.POINTER(ctypes.c_int)]
    L.nfs_band_structure.restype = ip
    L.nfs_batch_num_classes.argtypes = [vp]
    L.nfs_batch_num_classes.restype = ip
    L.nfs_destroy_batch.argtypes = [vp]
    L.nfs_destroy_batch.restype = None
    L.nfs_strerror.argtypes = [ip]
    L.nfs_strerror.restype = ctypes.c_char_p
    _ = dp
    _lib = L
    return L


def _strerror(code):
    try:
        return lib().nfs_strerror(int(code)).decode()
    except NFSLibraryMissing:
        return "libnfs missing"


def _check(code, where):
    if code != NFS_OK:
        raise NFSError(code, where)


def default_options() -> Options:
    o = Options()
    lib().nfs_default_options(ctypes.byref(o))
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _material(medium):
    """nfs_material over host copies of the medium (returned to keep alive)."""
    if medium.kind not in ("chiral", "pseudochiral"):
        raise ValueError(f"the CUDA library solves chiral and pseudochiral media, not {medium.kind!r}")
    eps = np.ascontiguousarray(medium.eps, dtype=np.float64)
    gam = np.ascontiguousarray(medium.gamma, dtype=np.float64)
    mu = None if medium.mu is None else np.ascontiguousarray(medium.mu, dtype=np.float64)
    m = Material()
    m.kind = MEDIUM_CHIRAL if medium.kind == "chiral" else MEDIUM_PSEUDOCHIRAL
    m.axis_a, m.axis_b = (int(medium.axes[0]), int(medium.axes[1]))
    m.eps = _dptr(eps)
    m.gamma = _dptr(gam)
    m.mu = _dptr(mu) if mu is not None else ctypes.POINTER(ctypes.c_double)()
    return m, (eps, gam, mu)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


_live_contexts = 0  # Context objects whose library context is open


def live_contexts():
    """How many Context objects currently hold an open library context."""
    return _live_contexts


class Context:
    """One Bloch problem on the GPU: grid, k, medium, options (nfs_setup)."""

    def __init__(self, grid, kdota, medium, precision="fp64", stream=None, **opts):
        import torch  # device memory and streams
        L = lib()
        self.grid = tuple(int(g) for g in grid)
        n1, n2, n3 = self.grid
        self.n = n1 * n2 * n3
        self.N = 4 * self.n
        self.medium = medium
        o = default_options()
        o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        for key, val in opts.items():
            setattr(o, key, val)
        self.stream_handle = stream if stream is not None else _current_stream()
        o.stream = self.stream_handle
        self.options = o
        self.precision = precision
        m, self._keep = _material(medium)
        a = float(getattr(medium, "a", 1.0))
        lattice = np.diag([a, a, a]).astype(np.float64).ravel()
        # kdota = (k.a_1, k.a_2, k.a_3); for a lattice a_l = a e_l, k = kdota / a
        kvec = np.asarray(kdota, dtype=np.float64) / a
        g = (ctypes.c_int * 3)(*self.grid)
        h = ctypes.c_void_p()
        _check(L.nfs_setup(ctypes.byref(h), g, _dptr(lattice), _dptr(kvec), ctypes.byref(m), ctypes.byref(o)),
               "nfs_setup")
        self.h = h
        self._torch = torch
        global _live_contexts
        _live_contexts += 1

    # -- helpers --------------------------------------------------------------
    def _vec(self, t, dtype):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
                and t.numel() == self.N):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of {self.N} elements")
        return ctypes.c_void_p(t.data_ptr())

    def close(self):
        if getattr(self, "h", None):
            lib().nfs_destroy(self.h)
            self.h = None
            global _live_contexts
            _live_contexts -= 1

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def device_bytes(self):
        return int(lib().nfs_device_bytes(self.h))

    # -- operations -----------------------------------------------------------
    def matvec(self, u, out=None):
        """A_r u (complex128 or complex64 CUDA tensor)."""
        torch = self._torch
        dt = u.dtype
        code = C128 if dt == torch.complex128 else C64
        if out is None:
            out = torch.empty_like(u)
        _check(lib().nfs_matvec(self.h, code, self._vec(u, dt), self._vec(out, dt)), "nfs_matvec")
        return out

    def matvec_ds(self, u, out=None):
        """A_r u for a complex128 tensor, computed in double-single arithmetic
        (mixed contexts; the product their refinement residuals use)."""
        torch = self._torch
        if out is None:
            out = torch.empty_like(u)
        _check(lib().nfs_matvec(self.h, C128_DS, self._vec(u, torch.complex128), self._vec(out, torch.complex128)),
               "nfs_matvec")
        return out

    def matvec_passes(self, mask, u, out):
        """Only the selected passes of the product (timing aid; see nfs.h)."""
        torch = self._torch
        dt = u.dtype
        code = C128 if dt == torch.complex128 else C64
        _check(lib().nfs_matvec_passes(self.h, code, int(mask), self._vec(u, dt), self._vec(out, dt)),
               "nfs_matvec_passes")
        return out

    def apply_Br(self, v, out=None):
        torch = self._torch
        if out is None:
            out = torch.empty_like(v)
        _check(lib().nfs_apply_Br(self.h, self._vec(v, torch.complex128), self._vec(out, torch.complex128)),
               "nfs_apply_Br")
        return out

    def cg_solve(self, b, x0=None):
        torch = self._torch
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        info = SolveInfo()
        code = lib().nfs_cg_solve(self.h, self._vec(b, torch.complex128), self._vec(x, torch.complex128),
                                  ctypes.byref(info))
        if code not in (NFS_OK, NFS_ENOCONV):
            raise NFSError(code, "nfs_cg_solve")
        return x, info

    def reserve(self, nev):
        """Allocate now what an eigensolve for nev pairs uses (nfs_reserve)."""
        _check(lib().nfs_reserve(self.h, int(nev)), "nfs_reserve")

    def eigs(self, nev, vectors=True, allow_noconv=False):
        torch = self._torch
        omega = np.zeros(nev, dtype=np.float64)
        Y = torch.empty((nev, self.N), dtype=torch.complex128, device="cuda") if vectors else None
        info = EigsInfo()
        code = lib().nfs_eigs(self.h, int(nev), _dptr(omega), ctypes.c_void_p(Y.data_ptr()) if vectors else None,
                              ctypes.byref(info))
        if code != NFS_OK and not (allow_noconv and code == NFS_ENOCONV):
            raise NFSError(code, "nfs_eigs")
        return omega, Y, info

    def eig_grad(self, Y, weights):
        """d(sum_j w_j omega_j) / d(per-component eps, gamma) from eigenvectors Y."""
        torch = self._torch
        m = int(Y.shape[0])
        if not (Y.is_cuda and Y.dtype == torch.complex128 and Y.is_contiguous() and Y.shape[1] == self.N):
            raise ValueError("Y must be a contiguous CUDA complex128 tensor (m, 4n)")
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(m))
        n1, n2, n3 = self.grid
        d_eps = torch.empty((3, n3, n2, n1), dtype=torch.float64, device="cuda")
        gshape = (3, n3, n2, n1) if self.medium.kind == "chiral" else (n3, n2, n1)
        d_gam = torch.empty(gshape, dtype=torch.float64, device="cuda")
        _check(lib().nfs_eig_grad(self.h, m, _dptr(w), ctypes.c_void_p(Y.data_ptr()),
                                  ctypes.c_void_p(d_eps.data_ptr()), ctypes.c_void_p(d_gam.data_ptr())),
               "nfs_eig_grad")
        return d_eps, d_gam

    def eig_fields(self, Y):
        """Fields [E; H] = B^{-1} diag(P_r, Q_r) y of eigenvectors Y (m, 4n):
        a CUDA complex128 tensor (m, 6, n3, n2, n1), components E_x, E_y, E_z,
        H_x, H_y, H_z (nfs_eig_fields)."""
        torch = self._torch
        Y = Y.reshape(-1, self.N)
        if not (Y.is_cuda and Y.dtype == torch.complex128 and Y.is_contiguous()):
            raise ValueError("Y must be a contiguous CUDA complex128 tensor (m, 4n)")
        m = int(Y.shape[0])
        n1, n2, n3 = self.grid
        X = torch.empty((m, 6, n3, n2, n1), dtype=torch.complex128, device="cuda")
        _check(lib().nfs_eig_fields(self.h, m, ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(X.data_ptr())),
               "nfs_eig_fields")
        return X

    def gep_residual(self, omega, X):
        """||diag(C, C^*) x - omega B x|| / (|omega| ||B x||) per eigenpair of
        the GEP, from fields X (m, 6n) (nfs_gep_residual)."""
        torch = self._torch
        X = X.reshape(-1, 6 * self.n)
        if not (X.is_cuda and X.dtype == torch.complex128 and X.is_contiguous()):
            raise ValueError("X must be a contiguous CUDA complex128 tensor (m, 6n)")
        m = int(X.shape[0])
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(m))
        res = np.zeros(m, dtype=np.float64)
        _check(lib().nfs_gep_residual(self.h, m, _dptr(om), ctypes.c_void_p(X.data_ptr()), _dptr(res)),
               "nfs_gep_residual")
        return res


class NFSEPContext:
    """A bi-isotropic medium outside the Assumption (nfs_setup_biiso): the
    null space free standard problem M y = omega y of eq. NFSEP_org, its
    shift-and-invert Arnoldi eigensolve and Algorithm 1's second branch."""

    def __init__(self, grid, kdota, medium, stream=None, **opts):
        import torch
        L = lib()
        if medium.kind != "biisotropic":
            raise ValueError("NFSEPContext takes a biisotropic medium")
        self.grid = tuple(int(g) for g in grid)
        n1, n2, n3 = self.grid
        self.n = n1 * n2 * n3
        self.N = 4 * self.n

        def carr(a):
            return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
        self._keep = [carr(medium.eps), carr(medium.mu), carr(medium.gamma), carr(getattr(medium, "chi", None))]
        m = BiisoMaterial()
        null = ctypes.POINTER(ctypes.c_double)()
        for name, arr in zip(("eps", "mu", "gamma", "chi"), self._keep):
            setattr(m, name, arr.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                    if arr is not None else null)
        o = default_options()
        for key, val in opts.items():
            setattr(o, key, val)
        o.stream = stream if stream is not None else _current_stream()
        a = float(getattr(medium, "a", 1.0))
        lattice = np.diag([a, a, a]).astype(np.float64).ravel()
        kvec = np.asarray(kdota, dtype=np.float64) / a
        g = (ctypes.c_int * 3)(*self.grid)
        h = ctypes.c_void_p()
        _check(L.nfs_setup_biiso(ctypes.byref(h), g, _dptr(lattice), _dptr(kvec), ctypes.byref(m), ctypes.byref(o)),
               "nfs_setup_biiso")
        self.h = h
        self._torch = torch

    def _vec(self, t):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
                and t.numel() == self.N):
            raise ValueError(f"expected a contiguous CUDA complex128 tensor of {self.N} elements")
        return ctypes.c_void_p(t.data_ptr())

    def reserve(self, nev):
        """Allocate now what nfs_nfsep_eigs for nev values uses (nfs_reserve)."""
        _check(lib().nfs_reserve(self.h, int(nev)), "nfs_reserve")

    @property
    def device_bytes(self):
        return int(lib().nfs_device_bytes(self.h))

    def matvec(self, y, out=None):
        """M y (eq. NFSEP_org)."""
        if out is None:
            out = self._torch.empty_like(y)
        _check(lib().nfs_nfsep_matvec(self.h, self._vec(y), self._vec(out)), "nfs_nfsep_matvec")
        return out

    def eigs(self, nev, sigma, vectors=True, allow_noconv=False):
        """The nev eigenvalues of M nearest the complex shift sigma: (omega
        complex (nev,), Y (nev, 4n) or None, NfsepInfo).  With allow_noconv an
        NFS_ENOCONV return is passed through: omega holds the results if the
        restart cap was hit, zeros if an inner GMRES solve did not converge
        (info.nconv = 0 then)."""
        torch = self._torch
        sg = np.array([complex(sigma).real, complex(sigma).imag], dtype=np.float64)
        om = np.zeros(2 * nev, dtype=np.float64)
        Y = torch.empty((nev, self.N), dtype=torch.complex128, device="cuda") if vectors else None
        info = NfsepInfo()
        code = lib().nfs_nfsep_eigs(self.h, int(nev), _dptr(sg), _dptr(om),
                                    ctypes.c_void_p(Y.data_ptr()) if vectors else None, ctypes.byref(info))
        if code != NFS_OK and not (allow_noconv and code == NFS_ENOCONV):
            raise NFSError(code, "nfs_nfsep_eigs")
        return om[0::2] + 1j * om[1::2], Y, info

    def fields(self, Y):
        """[E; H] of NFSEP eigenvectors Y (m, 4n): (m, 6, n3, n2, n1)."""
        torch = self._torch
        Y = Y.reshape(-1, self.N)
        if not (Y.is_cuda and Y.dtype == torch.complex128 and Y.is_contiguous()):
            raise ValueError("Y must be a contiguous CUDA complex128 tensor (m, 4n)")
        m = int(Y.shape[0])
        n1, n2, n3 = self.grid
        X = torch.empty((m, 6, n3, n2, n1), dtype=torch.complex128, device="cuda")
        _check(lib().nfs_nfsep_fields(self.h, m, ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(X.data_ptr())),
               "nfs_nfsep_fields")
        return X

    def close(self):
        if getattr(self, "h", None):
            lib().nfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent Bloch problems solved together (nfs_setup_batch).

    problems: sequence of (grid, kdota, medium) on the unit cube lattice.
    Problems sharing a grid, medium kind, pseudochiral axes and mu-ness are
    solved in lock-step through single kernel launches; distinct classes run
    concurrently."""

    def __init__(self, problems, precision="mixed", stream=None, **opts):
        import torch  # noqa: F401  (device and stream owner)
        L = lib()
        self.nprob = len(problems)
        arr = (Problem * max(1, self.nprob))()
        keep = []
        for i, (grid, kdota, medium) in enumerate(problems):
            if float(getattr(medium, "a", 1.0)) != 1.0:
                raise ValueError("batched problems use the unit cube lattice")
            m, kp = _material(medium)
            keep.append(kp)
            arr[i].grid[:] = [int(x) for x in grid]
            arr[i].k[:] = [float(x) for x in kdota]
            arr[i].mat = m
        o = default_options()
        o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
        for key, val in opts.items():
            setattr(o, key, val)
        o.stream = stream if stream is not None else _current_stream()
        h = ctypes.c_void_p()
        _check(L.nfs_setup_batch(ctypes.byref(h), int(self.nprob), arr, ctypes.byref(o)), "nfs_setup_batch")
        self.h = h

    @property
    def num_classes(self):
        return int(lib().nfs_batch_num_classes(self.h))

    def eigs(self, nev, allow_noconv=False):
        """(omega [nprob, nev], list of EigsInfo)."""
        omega = np.zeros((self.nprob, nev), dtype=np.float64)
        infos = (EigsInfo * max(1, self.nprob))()
        code = lib().nfs_eigs_batch(self.h, int(nev), _dptr(omega), infos)
        if code != NFS_OK and not (allow_noconv and code == NFS_ENOCONV):
            raise NFSError(code, "nfs_eigs_batch")
        return omega, [infos[i] for i in range(self.nprob)]

    def close(self):
        if getattr(self, "h", None):
            lib().nfs_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# High-symmetry points of the simple cubic Brillouin zone, Bloch vector / 2 pi
# on the unit cube lattice.
SC_POINTS = {"G": (0.0, 0.0, 0.0), "X": (0.5, 0.0, 0.0), "M": (0.5, 0.5, 0.0), "R": (0.5, 0.5, 0.5)}


def kpath(corners=("G", "X", "M", "R", "G"), per_segment=10):
    """Bloch vectors along the polyline through ``corners`` (names of
    SC_POINTS or triples): ``per_segment`` uniformly spaced samples per
    segment at the midpoints of its equal subintervals, which never land on a
    corner, so Gamma (where Lambda_q is singular) is never sampled.  Returns
    (k (m, 3), arc length at each k (m,))."""
    pts = [np.asarray(SC_POINTS[c] if isinstance(c, str) else c, dtype=np.float64) for c in corners]
    ks, arc, s0 = [], [], 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        seg = float(np.linalg.norm(b - a))
        for i in range(per_segment):
            t = (i + 0.5) / per_segment
            ks.append(a + t * (b - a))
            arc.append(s0 + t * seg)
        s0 += seg
    return np.array(ks), np.array(arc)


def band_structure(grid, medium, kpoints, nev, precision="mixed", max_chunk=0, stream=None, deflation_checks=2,
                   **opts):
    """The nev smallest positive omega at every Bloch vector of ``kpoints``
    (m, 3) for one grid and medium (nfs_band_structure: chunks of k-points
    solved as batches sized to the device memory).  Paths through
    high-symmetry points meet degenerate eigenvalues, so by default every
    solve runs two deflation checks (nfs_options.deflation_checks).  Returns
    (omega (m, nev), list of EigsInfo, number of chunks)."""
    opts["deflation_checks"] = deflation_checks
    L = lib()
    if float(getattr(medium, "a", 1.0)) != 1.0:
        raise ValueError("band_structure uses the unit cube lattice")
    k = np.ascontiguousarray(np.asarray(kpoints, dtype=np.float64).reshape(-1, 3))
    nk = int(k.shape[0])
    m, keep = _material(medium)
    o = default_options()
    o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
    for key, val in opts.items():
        setattr(o, key, val)
    o.stream = stream if stream is not None else _current_stream()
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    omega = np.zeros((nk, nev), dtype=np.float64)
    infos = (EigsInfo * nk)()
    chunks = ctypes.c_int(0)
    code = L.nfs_band_structure(g, ctypes.byref(m), nk, _dptr(k), ctypes.byref(o), int(nev), int(max_chunk),
                                _dptr(omega), infos, ctypes.byref(chunks))
    del keep
    if code != NFS_OK:
        raise NFSError(code, "nfs_band_structure")
    return omega, [infos[i] for i in range(nk)], int(chunks.value)


def matvec_noalloc(grid, kdota, kind, axes, eps, gamma, u, out, alpha=2.0, beta=3.0, stream=None):
    """A_r u through nfs_matvec_noalloc: no device allocation by the library.

    For callers that cannot let the library allocate device memory (their
    framework already reserved the GPU, or their budget is fixed).  eps and
    gamma are CUDA float64 tensors in the medium layout; u and out CUDA
    complex128 tensors of 4n elements.  Grids up to NOALLOC_MAX_VOXELS voxels,
    unit cube, mu = 1.  Calls share one workspace inside the library, so they
    must not overlap on the GPU."""
    import torch
    for t, dt in ((eps, torch.float64), (gamma, torch.float64), (u, torch.complex128), (out, torch.complex128)):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError("eps, gamma: contiguous CUDA float64; u, out: contiguous CUDA complex128")
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    k = (ctypes.c_double * 3)(*[float(x) for x in kdota])
    kd = MEDIUM_CHIRAL if kind == "chiral" else MEDIUM_PSEUDOCHIRAL
    st = stream if stream is not None else _current_stream()
    code = lib().nfs_matvec_noalloc(g, k, kd, int(axes[0]), int(axes[1]), ctypes.c_void_p(eps.data_ptr()),
                                    ctypes.c_void_p(gamma.data_ptr()), float(alpha), float(beta),
                                    ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()), st)
    _check(code, "nfs_matvec_noalloc")
    return out


def residuals(ctx: Context, omega, Y):
    """||A_r y - omega B_r y|| / ||y|| per eigenpair (nfs_residuals: FP64 on
    the device)."""
    torch = ctx._torch
    m = len(omega)
    if m == 0:
        return []
    Yc = Y.contiguous()
    if not (Yc.is_cuda and Yc.dtype == torch.complex128 and Yc.numel() == m * 4 * ctx.n):
        raise ValueError("Y: CUDA complex128 tensor of m x 4n")
    om = (ctypes.c_double * m)(*[float(w) for w in omega])
    res = (ctypes.c_double * m)()
    _check(lib().nfs_residuals(ctx.h, m, om, ctypes.c_void_p(Yc.data_ptr()), res), "nfs_residuals")
    return [float(x) for x in res]
