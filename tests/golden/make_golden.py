"""Writes the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

fci8_energies.txt: the 8 lowest eigenvalues of H for the norb=8, 4+4 electron
workload over all 70 x 70 strings (seeded synthetic Hamiltonian), from the
oracle's dense H and numpy.linalg.eigvalsh.

sel12_energies.txt: the 3 lowest eigenvalues of H for norb=12, 6+6 electrons,
250 selected alpha x 260 selected beta strings (65,000 determinants, distinct
alpha and beta sets), beyond the reach of a dense solver (34 GB). Two
independent solvers driven by the oracle's sigma must agree to 1e-9 Eh before
the file is written: the oracle's Davidson at tight tolerances (|dE| < 1e-11,
||r|| < 1e-7) and ARPACK Lanczos (scipy.sparse.linalg.eigsh, smallest
algebraic). The Davidson values are stored.

    python tests/golden/make_golden.py [fci8] [sel12] [refs]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from tbsci_inputs import WORKLOADS  # noqa: E402


# norb=12 selected space of the stored Davidson energies (seeds of tbsci_inputs)
SEL12 = dict(norb=12, nelec=6, count_alpha=250, count_beta=260, seed_ints=4012, seed_alpha=4013,
             seed_beta=4014, nroots=3)


def sel12():
    import time

    from scipy.sparse.linalg import LinearOperator, eigsh

    from tbsci_inputs import selected_strings, synth_hamiltonian
    c = SEL12
    h, eri, ecore = synth_hamiltonian(c["norb"], c["seed_ints"])
    a = selected_strings(c["norb"], c["nelec"], c["count_alpha"], c["seed_alpha"])
    b = selected_strings(c["norb"], c["nelec"], c["count_beta"], c["seed_beta"])
    sp = oracle.make_space(c["norb"], c["nelec"], c["nelec"], a, b)
    t0 = time.time()
    e_dav, _, info = oracle.solve(sp, h, eri, ecore, c["nroots"], tol_e=1e-11, tol_r=1e-7)
    assert info["converged"], info
    t1 = time.time()
    op = LinearOperator((sp.ndet, sp.ndet), dtype=np.float64,
                        matvec=lambda x: oracle.sigma(sp, h, eri, ecore, np.asarray(x).reshape(1, -1))[0])
    e_lan = np.sort(eigsh(op, k=c["nroots"], which="SA", tol=1e-12, return_eigenvectors=False))
    t2 = time.time()
    diff = float(np.max(np.abs(e_dav - e_lan)))
    print("sel12: Davidson %s (%d it, %.0f s); Lanczos %s (%.0f s); max diff %.2e" %
          (e_dav, info["iterations"], t1 - t0, e_lan, t2 - t1, diff))
    assert diff < 1e-9, (e_dav, e_lan)
    np.savetxt(os.path.join(HERE, "sel12_energies.txt"), e_dav, fmt="%.15f",
               header="lowest 3 eigenvalues of H, norb=12, 6+6 electrons, 250 x 260 selected strings "
                      "(alpha seed 4013, beta seed 4014), synthetic Hamiltonian seed 4012; oracle Davidson "
                      "(|dE| < 1e-11, ||r|| < 1e-7), agreeing with ARPACK Lanczos on the oracle sigma to %.1e Eh"
                      % diff)


def fci8():
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta)
    H = oracle.hamiltonian_dense(sp, h, eri, ecore)
    e = np.linalg.eigvalsh(H)[:8]
    np.savetxt(os.path.join(HERE, "fci8_energies.txt"), e, fmt="%.15f",
               header="lowest eigenvalues of H, norb=8, 4+4 electrons, full 70x70 string space, "
                      "synthetic Hamiltonian seed 1001 (oracle dense H + numpy eigvalsh)")


def refs():
    """Prints the selection centres of the named selected workloads: the argmin of
    the one-spin string energy over all C(n, N) strings (the oracle's diagonal
    of the space with no beta electron), ties to the smaller integer. They are
    stored as constants in tbsci_inputs.WORKLOADS."""
    for name, wl in sorted(WORKLOADS.items()):
        if wl.count_alpha is None:
            continue
        h, eri, _ = wl.hamiltonian()
        sp = oracle.make_space(wl.norb, wl.nalpha, 0)
        E = oracle.diagonal(sp, h, eri, 0.0)
        print("%s reference=0b%s" % (name, bin(int(sp.sa[int(np.argmin(E))]))[2:]))


def main(argv):
    which = argv or ["fci8", "sel12"]
    if "refs" in which:
        refs()
    if "fci8" in which:
        fci8()
    if "sel12" in which:
        sel12()


if __name__ == "__main__":
    main(sys.argv[1:])
