"""torch.autograd wrapper: eigenvalues as a differentiable function of the
per-voxel permittivity and chirality.

Forward runs nfs_setup + nfs_eigs; backward calls nfs_eig_grad with the
incoming gradient as the weights, i.e. the adjoint d(sum_j g_j omega_j) /
d(eps, gamma) = sum_j g_j y_j^* (dA_r) y_j / (y_j^* B_r y_j) evaluated by the
hand-written CUDA kernel.  Both steps run in libnfs; this module only moves
tensors.  The gradient of a single eigenvalue inside a degenerate cluster is
not defined; the gradient of a sum over a complete cluster is.

Device memory: when no gradient is wanted (torch.no_grad, or neither input
requires one) the forward releases its library context before returning.
Otherwise the context and the eigenvectors stay with the autograd graph until
backward runs, or until the graph is freed (the output and everything derived
from it are gone), whichever comes first.
"""

from __future__ import annotations

import numpy as np
import torch

import workloads as wl

from . import nfs


def _as_components(t, shape3):
    a = t.detach().to("cpu", torch.float64).numpy()
    if a.shape == shape3[1:]:
        return np.broadcast_to(a, shape3).copy(), True
    if a.shape == shape3:
        return np.ascontiguousarray(a), False
    raise ValueError(f"expected a per-voxel {shape3[1:]} or per-component {shape3} array, got {a.shape}")


class NSFEigenvalues(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eps, gamma, grid, kdota, nev, precision, options):
        n1, n2, n3 = grid
        shape3 = (3, n3, n2, n1)
        e, eps_voxel = _as_components(eps, shape3)
        g, gam_voxel = _as_components(gamma, shape3)
        medium = wl.Medium(tuple(grid), "chiral", e, g)
        ctx = nfs.Context(grid, kdota, medium, precision=precision, **options)
        try:
            omega, Y, _ = ctx.eigs(nev, vectors=True)
        except Exception:
            ctx.close()
            raise
        fctx.nfs_ctx = ctx
        fctx.Y = Y
        fctx.flags = (eps_voxel, gam_voxel, eps.dtype, eps.device, gamma.dtype, gamma.device)
        return torch.as_tensor(omega, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(fctx, grad_omega):
        eps_voxel, gam_voxel, edt, edev, gdt, gdev = fctx.flags
        w = grad_omega.detach().to("cpu", torch.float64).numpy()
        try:
            d_eps, d_gam = fctx.nfs_ctx.eig_grad(fctx.Y, w)
        finally:
            fctx.nfs_ctx.close()
            fctx.Y = None
        if eps_voxel:
            d_eps = d_eps.sum(0)
        if gam_voxel:
            d_gam = d_gam.sum(0)
        return d_eps.to(edev, edt), d_gam.to(gdev, gdt), None, None, None, None, None


def chiral_eigenvalues(eps, gamma, grid, kdota, nev=5, precision="fp64", **options):
    """The nev smallest positive eigenvalues of a chiral medium (mu = 1) given
    eps and gamma either per voxel (n3, n2, n1) -- the same value for the three
    field components -- or per component (3, n3, n2, n1); differentiable with
    respect to both."""
    if not (torch.is_grad_enabled() and (eps.requires_grad or gamma.requires_grad)):
        # inference: nothing to differentiate later, so no eigenvectors are
        # kept and the library context is released before returning
        n1, n2, n3 = grid
        shape3 = (3, n3, n2, n1)
        medium = wl.Medium(tuple(grid), "chiral", _as_components(eps, shape3)[0], _as_components(gamma, shape3)[0])
        ctx = nfs.Context(grid, kdota, medium, precision=precision, **options)
        try:
            omega, _, _ = ctx.eigs(int(nev), vectors=False)
        finally:
            ctx.close()
        return torch.as_tensor(omega, dtype=torch.float64, device=eps.device)
    return NSFEigenvalues.apply(eps, gamma, tuple(grid), tuple(kdota), int(nev), precision, dict(options))
