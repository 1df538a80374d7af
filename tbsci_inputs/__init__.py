"""Seeded synthetic inputs for the TBSCI sigma / Davidson path.

This module only draws random numbers and picks bitstrings. It holds none of
the method's arithmetic (no string enumeration of the full space, no matrix
elements, no signs): both the CPU oracle and the CUDA library consume what it
returns, and neither is imported here.

Recipe (stands in for the paper's molecular FCIDUMP inputs, Sec. III.A,
Table II, which are not available):

* one-electron integrals ``h``: diagonal ``U(-2, 0)`` sorted ascending (orbital 0
  lowest), off-diagonal ``N(0, 0.05^2)`` mirrored to a symmetric matrix;
* two-electron integrals in chemists' notation ``(ij|kl) = sum_P L^P_ij L^P_kl``
  with ``2 * norb`` random symmetric factors ``L^P = 0.3 * (A + A^T) / 2``,
  ``A_ij ~ N(0, 1)``; this has the 8-fold permutational symmetry of real
  orbitals by construction and is positive semi-definite over orbital pairs;
* ``ecore = 0``.

Selected string sets follow the weight-selection shape of Sec. III.B: a
reference string, then every string within a double excitation of it, then a
seeded uniform sample of triples and quadruples (the order of candidates before
sampling is ascending integer value). The reference of a named workload is its
lowest-energy string (the argmin of the one-spin string energy over all
C(n, N) strings, ties to the smaller integer), stored below as a constant that
tests/golden/make_golden.py computes with the oracle and a CPU test pins; other
selections (tests, the serving stream, whose per-request Hamiltonians would
need the string-energy formula here) use the aufbau string ``bits 0..N-1``.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "synth_hamiltonian",
    "reference_string",
    "excitation_candidates",
    "selected_strings",
    "random_vectors",
    "Workload",
    "WORKLOADS",
    "serving_stream",
    "excitation_level",
    "prune_by_total_level",
    "orbital_irreps",
    "synth_hamiltonian_symmetric",
]


def synth_hamiltonian(norb: int, seed: int, scale: float = 0.3, hoff_std: float = 0.05):
    """Return ``(h, eri, ecore)``: ``h`` is ``[n, n]`` float64, ``eri`` ``[n, n, n, n]``
    float64 in chemists' order ``eri[i, j, k, l] = (ij|kl)``, ``ecore = 0.0``."""
    rng = np.random.default_rng(seed)
    n = int(norb)
    diag = np.sort(rng.uniform(-2.0, 0.0, size=n))
    h = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, hoff_std, size=len(iu[0]))
    h[iu] = off
    h = h + h.T
    h[np.diag_indices(n)] = diag
    nfac = 2 * n
    A = rng.normal(0.0, 1.0, size=(nfac, n, n))
    L = scale * 0.5 * (A + np.transpose(A, (0, 2, 1)))
    eri = np.einsum("pij,pkl->ijkl", L, L)
    return h, np.ascontiguousarray(eri), 0.0


def orbital_irreps(norb: int, seed: int, nirrep: int = 8) -> np.ndarray:
    """Seeded irrep labels 0..nirrep-1 of the orbitals of an abelian point group
    (D2h: 8 irreps; labels multiply as bitwise XOR)."""
    return np.random.default_rng(seed).integers(0, nirrep, size=norb).astype(np.int32)


def synth_hamiltonian_symmetric(norb: int, seed: int, irreps, scale: float = 0.3, hoff_std: float = 0.05):
    """The recipe of ``synth_hamiltonian`` with point-group symmetry: h_ij = 0
    unless irreps i and j are equal, and each factor L^P carries an irrep G_P with
    L^P_ij = 0 unless irrep(i) XOR irrep(j) = G_P, so (ij|kl) = 0 unless the four
    labels XOR to 0 (8-fold symmetric and positive semi-definite as before)."""
    rng = np.random.default_rng(seed)
    n = int(norb)
    g = np.asarray(irreps, dtype=np.int64)
    diag = np.sort(rng.uniform(-2.0, 0.0, size=n))
    h = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    off = rng.normal(0.0, hoff_std, size=len(iu[0]))
    h[iu] = off
    h = h + h.T
    h[g[:, None] != g[None, :]] = 0.0
    h[np.diag_indices(n)] = diag
    nfac = 2 * n
    A = rng.normal(0.0, 1.0, size=(nfac, n, n))
    L = scale * 0.5 * (A + np.transpose(A, (0, 2, 1)))
    gp = rng.integers(0, int(g.max()) + 1 if len(g) else 1, size=nfac)
    mask = (g[:, None] ^ g[None, :])[None, :, :] == gp[:, None, None]
    L = L * mask
    eri = np.einsum("pij,pkl->ijkl", L, L)
    return h, np.ascontiguousarray(eri), 0.0


def reference_string(nelec: int) -> int:
    """The aufbau string: the ``nelec`` lowest orbitals occupied (``h_ii`` ascending)."""
    return (1 << nelec) - 1


def _strings_at_level(norb: int, nelec: int, level: int, ref: int | None = None) -> list[int]:
    """All strings that differ from the reference string (default: aufbau) by
    exactly ``level`` electrons, ascending by integer value."""
    if ref is None:
        ref = reference_string(nelec)
    occ = [i for i in range(norb) if (ref >> i) & 1]
    vir = [i for i in range(norb) if not (ref >> i) & 1]
    out = []
    for holes in itertools.combinations(occ, level):
        base = ref
        for h in holes:
            base &= ~(1 << h)
        for parts in itertools.combinations(vir, level):
            s = base
            for p in parts:
                s |= 1 << p
            out.append(s)
    out.sort()
    return out


def excitation_candidates(norb: int, nelec: int, max_level: int, ref: int | None = None) -> list[list[int]]:
    """``[level0, level1, ...]`` candidate lists up to ``max_level`` (inclusive)."""
    return [_strings_at_level(norb, nelec, k, ref) for k in range(max_level + 1)]


def selected_strings(norb: int, nelec: int, count: int, seed: int, shuffle: bool = True,
                     reference: int | None = None) -> np.ndarray:
    """Selected string set of ``min(count, C(norb, nelec))`` strings (uint64).

    ``reference`` (default: the aufbau string), all singles and doubles of it, then a seeded sample without
    replacement from the union of triples and quadruples. When ``count`` is below
    ``1 + #singles + #doubles`` the reference comes first, then singles, then
    doubles, each level in seeded random order, truncated. When ``count`` exceeds
    what levels <= 4 hold, higher levels are drawn from in turn. The result is
    returned in a seeded random order (both consumers must sort it) unless
    ``shuffle`` is False.
    """
    rng = np.random.default_rng(seed)
    total = math.comb(norb, nelec)
    count = int(min(count, total))
    maxlev = min(nelec, norb - nelec)
    if reference is not None and (bin(int(reference)).count("1") != nelec or int(reference) >> norb):
        raise ValueError("reference string must have nelec bits below norb")
    levels = excitation_candidates(norb, nelec, min(2, maxlev), reference)
    low = [s for lev in levels for s in lev]
    if count <= len(low):
        chosen = []
        for lev in levels:
            order = rng.permutation(len(lev))
            chosen.extend(lev[i] for i in order)
        chosen = chosen[:count]
    else:
        chosen = list(low)
        need = count - len(low)
        lev = 3
        while need > 0 and lev <= maxlev:
            hi = lev + 1 if lev + 1 <= maxlev else lev
            pool = []
            for k in range(lev, hi + 1):
                pool.extend(_strings_at_level(norb, nelec, k, reference))
            pool.sort()
            take = min(need, len(pool))
            pick = rng.choice(len(pool), size=take, replace=False)
            chosen.extend(pool[i] for i in sorted(pick))
            need -= take
            lev = hi + 1
    arr = np.array(chosen, dtype=np.uint64)
    if shuffle:
        arr = arr[rng.permutation(len(arr))]
    return arr


def excitation_level(strings, nelec: int) -> np.ndarray:
    """Number of electrons of each string outside the aufbau orbitals 0..nelec-1."""
    ref = np.uint64(reference_string(nelec))
    s = np.asarray(strings, dtype=np.uint64) & ~ref
    out = np.zeros(len(s), dtype=np.int64)
    for b in range(64):
        out += ((s >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return out


def prune_by_total_level(alpha_sorted, beta_sorted, nalpha: int, nbeta: int, max_level: int):
    """A determinant-level selection inside a TPB space (the general space of
    Sec. II.A, Eq. 6): keep (w, u) when the alpha and beta excitation levels sum to
    at most ``max_level``. Inputs are the SORTED string sets; returns the CSR
    ``(off[la + 1], cols)`` of allowed beta indices per alpha string."""
    la_lev = excitation_level(alpha_sorted, nalpha)
    lb_lev = excitation_level(beta_sorted, nbeta)
    cols, off = [], [0]
    for w in range(len(la_lev)):
        keep = np.nonzero(lb_lev + la_lev[w] <= max_level)[0].astype(np.int32)
        cols.append(keep)
        off.append(off[-1] + len(keep))
    return np.array(off, dtype=np.int64), (np.concatenate(cols) if cols else np.zeros(0, dtype=np.int32))


def random_vectors(nvec: int, la: int, lb: int, seed: int, dtype=np.float64) -> np.ndarray:
    """``[nvec, la, lb]`` standard-normal vectors (seeded)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nvec, la, lb)).astype(dtype)


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: sizes plus the seeds of its integrals, strings and vectors."""

    name: str
    norb: int
    nalpha: int
    nbeta: int
    count_alpha: int | None  # None = full string space
    count_beta: int | None
    nroots: int
    nvec: int
    seed_ints: int
    seed_sel: int
    seed_vec: int
    notes: str = ""
    extras: dict = field(default_factory=dict)
    reference: int | None = None  # centre of the selection (None: aufbau)

    def hamiltonian(self):
        return synth_hamiltonian(self.norb, self.seed_ints)

    def alpha_selection(self):
        """Selected alpha strings (uint64, shuffled) or ``None`` for the full space."""
        if self.count_alpha is None:
            return None
        return selected_strings(self.norb, self.nalpha, self.count_alpha, self.seed_sel, reference=self.reference)

    def beta_selection(self, distinct: bool = False):
        """Selected beta strings; identical to the alpha set (closed shell) unless
        ``distinct`` (then drawn with ``seed_sel + 1``)."""
        if self.count_beta is None:
            return None
        seed = self.seed_sel + 1 if distinct else self.seed_sel
        return selected_strings(self.norb, self.nbeta, self.count_beta, seed, reference=self.reference)


WORKLOADS = {
    "fci8": Workload("fci8", 8, 4, 4, None, None, 1, 1, 1001, 2001, 3001,
                     "norb=8, 4+4 electrons, all 70 x 70 strings (4,900 determinants)"),
    "sel16": Workload("sel16", 16, 8, 8, 3000, 3000, 3, 3, 1002, 2002, 3002,
                      "norb=16, 8+8 electrons, 3,000 x 3,000 selected strings (9.0M determinants)",
                      reference=0b10010111001101),
    "fci16": Workload("fci16", 16, 8, 8, None, None, 1, 1, 1003, 2003, 3003,
                      "norb=16, 8+8 electrons, 12,870 x 12,870 strings (165.6M determinants)"),
    "sel24": Workload("sel24", 24, 12, 12, 40000, 40000, 1, 1, 1004, 2004, 3004,
                      "norb=24, 12+12 electrons, 40,000 x 40,000 selected strings (1.6B determinants)",
                      reference=0b101110011011111100),
}


def serving_stream(nreq: int = 512, seed: int = 5005, rate_hz: float = 1.0,
                   norbs=(8, 10, 12, 14, 16), lo: int = 50, hi: int = 3000):
    """Seeded stream of solve requests with Poisson arrivals.

    Each entry: ``dict(t_arrival, norb, nelec, count, nroots, seed_ints, seed_sel)``.
    ``count`` is log-uniform in ``[lo, hi]`` and capped at ``C(norb, norb/2)``.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=nreq)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(nreq):
        n = int(rng.choice(norbs))
        ne = n // 2
        cnt = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        cnt = min(cnt, math.comb(n, ne))
        out.append(dict(t_arrival=float(t[i]), norb=n, nelec=ne, count=cnt,
                        nroots=int(rng.integers(1, 4)), seed_ints=int(rng.integers(1 << 30)),
                        seed_sel=int(rng.integers(1 << 30))))
    return out
