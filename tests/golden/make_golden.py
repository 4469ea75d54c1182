"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py

Every file records the workload, the oracle tier that produced it and the
paper's passage that defines the quantity.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import gep  # noqa: E402


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


if __name__ == "__main__":
    main()
