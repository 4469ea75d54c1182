"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
The large tier-O3 solves of the benchmark workloads take from an hour to
several hours of CPU time each and run only when named:
    python tests/golden/make_golden.py sphere64 pseudo96

Every file records the workload, the oracle tier that produced it and the
paper's passage that defines the quantity.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import gep, nfgep, nfsep  # noqa: E402


def write(name, header, values):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for v in values:
            f.write(f"{v:.17e}\n")


def main():
    # sphere8: 8^3, chiral sphere r = 0.25 (eps 13, gamma 0.5 inside; 1, 0 outside),
    # k.a = (0.1, 0.2, 0.3), 10 smallest positive eigenvalues.
    w8 = wl.workload("sphere8")
    w, _, idx = gep.dense_eigs(w8["grid"], w8["kdota"], w8["medium"], 10)
    write("sphere8_omega.txt", """
10 smallest positive eigenvalues omega of the discrete GEP (Sec. 3, eq. (discrete_GEP_EH))
workload sphere8: grid 8x8x8, a = 1, chiral sphere radius 0.25 centred in the cell,
(eps_i, eps_o, gamma) = (13, 1, 0.5), mu = 1, k.a = (0.1, 0.2, 0.3)
oracle tier O1: dense Hermitian-definite pencil (oracle.gep.dense_eigs), FP64
""", w[idx])
    # pseudochiral 8^3 (x-y coupling, constant gamma 0.4, 4 cylinders r = 0.1, seed 0)
    g = (8, 8, 8)
    med = wl.pseudochiral_cylinders(g, 4, 0.1, 13.0, 1.0, 0.4, (0, 1), seed=0)
    w, _, idx = gep.dense_eigs(g, (0.1, 0.2, 0.3), med, 10)
    write("pseudo8_omega.txt", """
10 smallest positive eigenvalues omega of the discrete GEP (Sec. 3, eq. (discrete_GEP_EH))
with the pseudochiral tensors of eq. (pseudo_chiral_para_mtx) on the x-y axis pair
workload pseudo8: grid 8x8x8, 4 z-cylinders radius 0.1 (seed 0), eps 13 inside, 1 outside,
gamma = 0.4 everywhere, mu = 1, k.a = (0.1, 0.2, 0.3)
oracle tier O1: dense Hermitian-definite pencil (oracle.gep.dense_eigs), FP64
""", w[idx])

    # mesh: the third validation of Section 5.1 (Fig. diff_mesh) -- the three
    # smallest eigenvalues of the chiral sphere (13, 1, 0.5) at k = (0.5, 0, 0)
    # on n^3 grids; tier O1 at 8^3, tier O2 (sparse shift-invert about
    # sigma = 1.8, above half of every wanted omega) at 16^3, tier O3 (FFT
    # NFGEP, ARPACK with CG) at 24^3 and 32^3.
    rows = []
    for n in (8, 16, 24, 32):
        g = (n, n, n)
        med = wl.chiral_sphere(g, 0.25, 13.0, 1.0, 0.5)
        if n == 8:
            w, _, idx = gep.dense_eigs(g, (0.5, 0.0, 0.0), med, 3)
            om = w[idx[:3]]
        elif n == 16:
            om, _ = gep.sparse_eigs(g, (0.5, 0.0, 0.0), med, 3, sigma=1.8, tol=1e-12)
        else:
            om, _ = nfgep.NFGEP(g, (0.5, 0.0, 0.0), med).eigs(3, tol=1e-12, cg_tol=1e-13)
        rows.append([n] + [float(x) for x in om])
    with open(os.path.join(HERE, "mesh_sphere_omega.txt"), "w") as f:
        f.write("""# 3 smallest positive eigenvalues omega of the discrete GEP (Sec. 3, eq. (discrete_GEP_EH))
# on n x n x n grids (Sec. 5.1, third validation, Fig. diff_mesh): chiral sphere radius 0.25
# centred in the unit cell, (eps_i, eps_o, gamma) = (13, 1, 0.5), mu = 1, k = (0.5, 0, 0)
# oracle tier O1 (dense pencil) at n = 8, O2 (sparse shift-invert, sigma 1.8) at 16, O3 (FFT NFGEP) at 24, 32; FP64
# columns: n, omega_1, omega_2, omega_3
""")
        for r in rows:
            f.write(f"{r[0]:d} {r[1]:.17e} {r[2]:.17e} {r[3]:.17e}\n")

    # nfsep8: the four eigenvalues nearest sigma = 2 + 0.1i of the null space
    # free standard problem (thm:nfep, eq. NFSEP_org) of a lossy bi-isotropic
    # sphere, 8^3, k.a = (0.1, 0.2, 0.3): oracle shift-and-invert Arnoldi
    g = (8, 8, 8)
    med = wl.biisotropic_sphere(g, 0.25, 13.0 + 2.0j, 1.0, 0.5, 0.2)
    om, _ = nfsep.NFSEP(g, (0.1, 0.2, 0.3), med).eigs_near(2.0 + 0.1j, 4)
    with open(os.path.join(HERE, "nfsep8_omega.txt"), "w") as f:
        f.write("""# 4 eigenvalues nearest sigma = 2 + 0.1i of M y = omega y (eq. NFSEP_org; thm:nfep: the GEP's
# nonzero eigenvalues) for a bi-isotropic sphere outside the Assumption: radius 0.25, inside
# eps = 13 + 2i, gamma = 0.5, chi = 0.2, mu = 1; outside vacuum; grid 8x8x8, k.a = (0.1, 0.2, 0.3)
# oracle: FFT NFSEP operator, shift-and-invert Arnoldi with GMRES (oracle.nfsep.NFSEP.eigs_near), FP64
# columns: re, im (nearest sigma first)
""")
        for w in om:
            f.write(f"{w.real:.17e} {w.imag:.17e}\n")


def large(name):
    """The 20 smallest positive eigenvalues of a benchmark workload by the
    FFT NFGEP (tier O3: ARPACK invert Lanczos with CG solves at tolerance
    1e-13), with the wall time and the number of A_r products recorded."""
    w = wl.workload(name)
    O = nfgep.NFGEP(w["grid"], w["kdota"], w["medium"])
    t0 = time.time()
    om, _ = O.eigs(w["nev"], tol=1e-12, cg_tol=1e-13)
    dt = time.time() - t0
    g = w["grid"]
    desc = {
        "sphere64": "chiral sphere centred in the cell, radius U[0.2, 0.3] and gamma U[0.3, 0.8] drawn with seed 0,\n"
                    "eps 13 inside, 1 outside, mu = 1",
        "pseudo96": "4 z-cylinders radius 0.1 with seeded centres (seed 0), eps 13 inside, 1 outside,\n"
                    "pseudochiral x-y coupling (eq. (pseudo_chiral_para_mtx)) gamma = 0.4 everywhere, mu = 1",
        "pseudo48": "the pseudo96 medium on a 48^3 grid: 4 z-cylinders radius 0.1 with seeded centres (seed 0),\n"
                    "eps 13 inside, 1 outside, pseudochiral x-y coupling gamma = 0.4 everywhere, mu = 1",
    }[name]
    write(f"{name}_omega.txt", f"""
{w["nev"]} smallest positive eigenvalues omega of the discrete GEP (Sec. 3, eq. (discrete_GEP_EH)),
ascending; workload {name}: grid {g[0]}x{g[1]}x{g[2]}, a = 1, k.a = {tuple(w["kdota"])},
{desc}
oracle tier O3: FFT NFGEP (oracle.nfgep.NFGEP.eigs: ARPACK invert Lanczos, ncv {max(3 * w["nev"], 2 * w["nev"] + 1)},
tol 1e-12, CG tolerance 1e-13), FP64; {O.nmatvec} A_r products, {dt:.0f} s wall time on the build host
""", om)


def nfsep_grid(n):
    """The four eigenvalues nearest 2 + 0.1i of the null space free standard
    problem of the nfsep8 sphere on an n^3 grid (oracle shift-and-invert
    Arnoldi with GMRES), with the wall time recorded."""
    g = (n, n, n)
    med = wl.biisotropic_sphere(g, 0.25, 13.0 + 2.0j, 1.0, 0.5, 0.2)
    t0 = time.time()
    om, _ = nfsep.NFSEP(g, (0.1, 0.2, 0.3), med).eigs_near(2.0 + 0.1j, 4)
    dt = time.time() - t0
    with open(os.path.join(HERE, f"nfsep{n}_omega.txt"), "w") as f:
        f.write(f"""# 4 eigenvalues nearest sigma = 2 + 0.1i of M y = omega y (eq. NFSEP_org; thm:nfep: the GEP's
# nonzero eigenvalues) for a bi-isotropic sphere outside the Assumption: radius 0.25, inside
# eps = 13 + 2i, gamma = 0.5, chi = 0.2, mu = 1; outside vacuum; grid {n}x{n}x{n}, k.a = (0.1, 0.2, 0.3)
# oracle: FFT NFSEP operator, shift-and-invert Arnoldi with GMRES (oracle.nfsep.NFSEP.eigs_near), FP64;
# {dt:.0f} s on the host
# columns: re, im (nearest sigma first)
""")
        for w in om:
            f.write(f"{w.real:.17e} {w.imag:.17e}\n")


def bz48_problem(i):
    """The 10 smallest positive eigenvalues of problem i of the bz48 batch
    (48 k-points on G-X-M-R-G over 32^3, 48^3 and 64^3 chiral spheres) by
    the FFT NFGEP (tier O3), with the wall time and A_r products recorded."""
    w = wl.workload("bz48")
    g, k, med, nev = w["grid"][i], tuple(float(x) for x in w["kdota"][i]), w["medium"][i], w["nev"]
    O = nfgep.NFGEP(g, k, med)
    t0 = time.time()
    om, _ = O.eigs(nev, tol=1e-12, cg_tol=1e-13)
    dt = time.time() - t0
    write(f"bz48_{i}_omega.txt", f"""
{nev} smallest positive eigenvalues omega of the discrete GEP (Sec. 3, eq. (discrete_GEP_EH)),
ascending; problem {i} of workload bz48: grid {g[0]}x{g[1]}x{g[2]}, a = 1, k.a = {k},
chiral sphere of radius 0.25 centred in the cell, eps 13 inside, 1 outside, mu = 1,
gamma drawn per k-point (workloads.bz48)
oracle tier O3: FFT NFGEP (oracle.nfgep.NFGEP.eigs: ARPACK invert Lanczos, ncv {max(3 * nev, 2 * nev + 1)},
tol 1e-12, CG tolerance 1e-13), FP64; {O.nmatvec} A_r products, {dt:.0f} s wall time on the build host
""", om)


if __name__ == "__main__":
    if len(sys.argv) > 1:
        for name in sys.argv[1:]:
            if name.startswith("nfsep"):
                nfsep_grid(int(name[5:]))
            elif name.startswith("bz48_"):
                bz48_problem(int(name[5:]))
            else:
                large(name)
    else:
        main()
