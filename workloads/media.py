"""Synthetic media and k-points on a simple-cubic Yee grid.

Conventions (shared by every consumer):

* grid = (n1, n2, n3) points along x, y, z; arrays are shaped (n3, n2, n1),
  i.e. x is the fastest index, matching the linear index
  (k-1) n1 n2 + (j-1) n1 + i of the paper's appendix.
* The lattice is simple cubic with constant ``a`` (default 1); the mesh
  lengths are a / n_l.
* Material coefficients are sampled per field component at that component's
  Yee edge location: component c of voxel (i, j, k) sits at
  ((i, j, k) + 0.5 e_c) * delta.  The paper (Section 3, last paragraph) only
  says coefficients are averaged over neighbouring grid points; this module
  fixes one concrete discretisation and every consumer uses the same arrays.
* ``kdota`` is the triple (k . a_1, k . a_2, k . a_3): the Bloch phase across
  one lattice vector a_l is exp(i 2 pi k . a_l) (eq. (quasi_periodic)).

A :class:`Medium` is a plain record of per-component real arrays:

* chiral:        eps[3][n3][n2][n1] > 0, gamma[3][n3][n2][n1], mu = None (1)
* pseudochiral:  eps[3][...], gamma[n3][n2][n1] (one coupling per voxel),
                 coupled axis pair ``axes`` = (a, b), mu = None (1)
* biisotropic:   eps[3][...] and mu[3][...] (complex allowed: loss),
                 gamma[3][...] and chi[3][...] (complex allowed): the
                 chirality and Tellegen parameters of each component

Turning these into the magnetoelectric tensors xi, zeta is the method's job
and is done separately by each consumer.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

CHIRAL = "chiral"
PSEUDOCHIRAL = "pseudochiral"
BIISOTROPIC = "biisotropic"


@dataclasses.dataclass
class Medium:
    grid: Tuple[int, int, int]
    kind: str
    eps: np.ndarray                 # (3, n3, n2, n1) float64
    gamma: np.ndarray               # chiral: (3, n3, n2, n1); pseudochiral: (n3, n2, n1)
    mu: Optional[np.ndarray] = None  # (3, n3, n2, n1) or None meaning mu = 1
    axes: Tuple[int, int] = (0, 1)   # pseudochiral coupled pair
    a: float = 1.0
    chi: Optional[np.ndarray] = None  # biisotropic Tellegen parameter (3, n3, n2, n1)

    @property
    def n(self) -> int:
        n1, n2, n3 = self.grid
        return n1 * n2 * n3


def _yee_coords(grid, comp, a=1.0):
    """Coordinates (x, y, z), each shaped (n3, n2, n1), of component ``comp``."""
    n1, n2, n3 = grid
    off = [0.0, 0.0, 0.0]
    if comp is not None:
        off[comp] = 0.5
    x = (np.arange(n1) + off[0]) * (a / n1)
    y = (np.arange(n2) + off[1]) * (a / n2)
    z = (np.arange(n3) + off[2]) * (a / n3)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _periodic_delta(d, a):
    return d - a * np.round(d / a)


def sphere_indicator(grid, center, radius, comp, a=1.0):
    X, Y, Z = _yee_coords(grid, comp, a)
    dx = _periodic_delta(X - center[0], a)
    dy = _periodic_delta(Y - center[1], a)
    dz = _periodic_delta(Z - center[2], a)
    return (dx * dx + dy * dy + dz * dz) <= radius * radius


def cylinders_indicator(grid, centers_xy, radius, comp, a=1.0):
    """Union of z-directed circular cylinders (periodic images included)."""
    X, Y, _ = _yee_coords(grid, comp, a)
    ind = np.zeros(X.shape, dtype=bool)
    for cx, cy in centers_xy:
        dx = _periodic_delta(X - cx, a)
        dy = _periodic_delta(Y - cy, a)
        ind |= (dx * dx + dy * dy) <= radius * radius
    return ind


def chiral_sphere(grid, radius=0.25, eps_in=13.0, eps_out=1.0, gamma=0.5,
                  center=(0.5, 0.5, 0.5), a=1.0) -> Medium:
    """Dielectric chiral sphere: eps_in, gamma inside; eps_out, 0 outside."""
    n1, n2, n3 = grid
    eps = np.empty((3, n3, n2, n1))
    gam = np.empty((3, n3, n2, n1))
    for c in range(3):
        ind = sphere_indicator(grid, center, radius, c, a)
        eps[c] = np.where(ind, eps_in, eps_out)
        gam[c] = np.where(ind, gamma, 0.0)
    return Medium(tuple(grid), CHIRAL, eps, gam, None, (0, 1), a)


def biisotropic_sphere(grid, radius=0.25, eps_in=13.0, eps_out=1.0, gamma=0.5, chi=0.0, mu_in=1.0,
                       center=(0.5, 0.5, 0.5), a=1.0) -> Medium:
    """Bi-isotropic sphere: eps_in, mu_in, chirality gamma and Tellegen
    parameter chi inside (complex values allowed); eps_out, 1, 0, 0 outside."""
    n1, n2, n3 = grid
    shape = (3, n3, n2, n1)
    eps = np.empty(shape, np.complex128)
    mu = np.empty(shape, np.complex128)
    gam = np.empty(shape, np.complex128)
    ch = np.empty(shape, np.complex128)
    for c in range(3):
        ind = sphere_indicator(grid, center, radius, c, a)
        eps[c] = np.where(ind, eps_in, eps_out)
        mu[c] = np.where(ind, mu_in, 1.0)
        gam[c] = np.where(ind, gamma, 0.0)
        ch[c] = np.where(ind, chi, 0.0)
    return Medium(tuple(grid), BIISOTROPIC, eps, gam, mu, (0, 1), a, ch)


def homogeneous(grid, eps=1.0, gamma=0.0, a=1.0) -> Medium:
    n1, n2, n3 = grid
    return Medium(tuple(grid), CHIRAL, np.full((3, n3, n2, n1), float(eps)),
                  np.full((3, n3, n2, n1), float(gamma)), None, (0, 1), a)


def pseudochiral_cylinders(grid, n_cyl=4, radius=0.1, eps_in=13.0, eps_out=1.0,
                           gamma=0.4, axes=(0, 1), seed=0, a=1.0) -> Medium:
    """z-directed dielectric cylinders with seeded centres in the xy cell and
    a constant pseudochiral coupling ``gamma`` everywhere."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, a, size=(n_cyl, 2))
    n1, n2, n3 = grid
    eps = np.empty((3, n3, n2, n1))
    for c in range(3):
        ind = cylinders_indicator(grid, centers, radius, c, a)
        eps[c] = np.where(ind, eps_in, eps_out)
    gam = np.full((n3, n2, n1), float(gamma))
    return Medium(tuple(grid), PSEUDOCHIRAL, eps, gam, None, tuple(axes), a)


def smoothed_field(grid, seed, sigma=0.05, a=1.0):
    """Seeded white noise smoothed by a periodic Gaussian of width ``sigma``
    (in lattice units) and min-max normalised to [0, 1]."""
    n1, n2, n3 = grid
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n3, n2, n1))
    f1 = np.fft.fftfreq(n1, d=a / n1)
    f2 = np.fft.fftfreq(n2, d=a / n2)
    f3 = np.fft.fftfreq(n3, d=a / n3)
    F3, F2, F1 = np.meshgrid(f3, f2, f1, indexing="ij")
    kernel = np.exp(-2.0 * (math.pi * sigma) ** 2 * (F1 ** 2 + F2 ** 2 + F3 ** 2))
    s = np.real(np.fft.ifftn(np.fft.fftn(noise) * kernel))
    s -= s.min()
    top = s.max()
    return s / top if top > 0 else s


def smoothed_chiral_field(grid, seed=0, eps_lo=1.0, eps_hi=13.0, gamma_hi=0.8,
                          sigma=0.05, a=1.0) -> Medium:
    """Per-voxel eps in [eps_lo, eps_hi] and gamma in [0, gamma_hi] from two
    seeded smoothed fields; the same value is used for all three components."""
    s1 = smoothed_field(grid, seed, sigma, a)
    s2 = smoothed_field(grid, seed + 1, sigma, a)
    eps = np.broadcast_to(eps_lo + (eps_hi - eps_lo) * s1, (3,) + s1.shape).copy()
    gam = np.broadcast_to(gamma_hi * s2, (3,) + s2.shape).copy()
    return Medium(tuple(grid), CHIRAL, eps, gam, None, (0, 1), a)


def bz_path_midpoints(count=48):
    """k-points (as k.a_l triples) at arc-length midpoints (j + 1/2)/count of
    the simple-cubic path G-X-M-R-G.  G itself (all k.a_l integer) is never
    sampled."""
    corners = np.array([[0, 0, 0], [0.5, 0, 0], [0.5, 0.5, 0],
                        [0.5, 0.5, 0.5], [0, 0, 0]], dtype=float)
    seg = np.linalg.norm(np.diff(corners, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    total = cum[-1]
    out = []
    for j in range(count):
        t = (j + 0.5) / count * total
        s = min(np.searchsorted(cum, t, side="right") - 1, len(seg) - 1)
        frac = (t - cum[s]) / seg[s]
        out.append(corners[s] + frac * (corners[s + 1] - corners[s]))
    return np.array(out)


def random_complex(shape, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return z.astype(dtype)


# ---------------------------------------------------------------------------
# Named workloads (sizes, media and k-points of the benchmarked problems).
# ---------------------------------------------------------------------------

DEFAULT_K = (0.1, 0.2, 0.3)


def workload(name: str, seed: int = 0):
    """Return a dict describing one named workload.

    Keys: grid, medium (Medium or list of Medium), kdota (triple or list),
    nev, precision ('fp64' or 'mixed').
    """
    if name == "sphere8":
        g = (8, 8, 8)
        return dict(grid=g, medium=chiral_sphere(g, 0.25, 13.0, 1.0, 0.5),
                    kdota=DEFAULT_K, nev=10, precision="fp64")
    if name == "sphere64":
        rng = np.random.default_rng(seed)
        r = float(rng.uniform(0.2, 0.3))
        gam = float(rng.uniform(0.3, 0.8))
        g = (64, 64, 64)
        return dict(grid=g, medium=chiral_sphere(g, r, 13.0, 1.0, gam),
                    kdota=DEFAULT_K, nev=20, precision="fp64")
    if name == "pseudo96":
        g = (96, 96, 96)
        return dict(grid=g, medium=pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4,
                                                          (0, 1), seed),
                    kdota=DEFAULT_K, nev=20, precision="mixed")
    if name.startswith("pseudo") and name[6:].isdigit():
        # the headline medium on another grid (a size whose oracle solve is short)
        s = int(name[6:])
        g = (s, s, s)
        return dict(grid=g, medium=pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), seed),
                    kdota=DEFAULT_K, nev=20, precision="mixed")
    if name == "bz48":
        ks = bz_path_midpoints(48)
        rng = np.random.default_rng(seed)
        sizes = [32] * 16 + [48] * 16 + [64] * 16
        gams = rng.uniform(0.2, 0.8, size=48)
        media = [chiral_sphere((s, s, s), 0.25, 13.0, 1.0, float(gm))
                 for s, gm in zip(sizes, gams)]
        return dict(grid=[(s, s, s) for s in sizes], medium=media,
                    kdota=[tuple(k) for k in ks], nev=10, precision="mixed")
    if name.startswith("field"):
        s = int(name[len("field"):])
        g = (s, s, s)
        return dict(grid=g, medium=smoothed_chiral_field(g, seed),
                    kdota=DEFAULT_K, nev=5, precision="fp64")
    raise KeyError(name)


WORKLOADS = ("sphere8", "sphere64", "pseudo48", "pseudo96", "bz48", "field16", "field64", "field128")
