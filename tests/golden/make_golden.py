"""Writes the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

fci8_energies.txt: the 8 lowest eigenvalues of H for the norb=8, 4+4 electron
workload over all 70 x 70 strings (seeded synthetic Hamiltonian), from the
oracle's dense H and numpy.linalg.eigvalsh.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from tbsci_inputs import WORKLOADS  # noqa: E402


def main():
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta)
    H = oracle.hamiltonian_dense(sp, h, eri, ecore)
    e = np.linalg.eigvalsh(H)[:8]
    np.savetxt(os.path.join(HERE, "fci8_energies.txt"), e, fmt="%.15f",
               header="lowest eigenvalues of H, norb=8, 4+4 electrons, full 70x70 string space, "
                      "synthetic Hamiltonian seed 1001 (oracle dense H + numpy eigvalsh)")


if __name__ == "__main__":
    main()
