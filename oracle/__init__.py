"""Plain FP64 CPU oracle for the TBSCI sigma / Davidson path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
CUDA library and its Python binding never import, link or call it, and share
no code with it; the only shared module is ``tbsci_inputs`` (seeded random
inputs, no method arithmetic).

What it computes (each function cites the passage it follows):

* ``fci_strings`` / ``sort_validate`` -- the alpha/beta string sets of the TPB
  space (Sec. II.A, Eq. 3), ascending integer order, 0-based index.
* ``links_single`` / ``links_double`` -- per-string single / double excitation
  links restricted to the selected set (BETA_SINGLE_LINK / BETA_DOUBLE_LINK,
  Sec. II.C; entry layout Sec. III.C), by explicit operator application.
* ``sigma`` / ``diagonal`` / ``hamiltonian_dense`` -- H restricted to the TPB
  space by the spin-orbital Slater-Condon rules (Sec. II.C, Eq. 8), sigma = H.c.
* ``davidson`` -- standard Davidson (Sec. III.A) with restart to the Ritz
  vectors when the subspace is full (Sec. III.C), in numpy FP64.
* ``string_weights`` / ``select_by_weight`` / ``coefficient_histogram`` -- the
  bitstring selection of Sec. III.B (weights as sums of squared coefficients,
  a threshold relative to the HF string's weight) and the coefficient
  distribution of Fig. 3 (counts of |c_K / c_HF| per logarithmic bin).
* ``PrunedSpace`` / ``sigma_pruned`` / ``diagonal_pruned`` -- the general TBSCI
  space D_TBSCI of Sec. II.A, Eq. 6: per alpha string w a set I_w of allowed beta
  strings; H on it is the principal submatrix of H on the member determinants.

Parity status: every function above is pinned by ``tests/test_oracle_pins.py``
(brute-force second quantisation, closed forms, library special cases,
invariants, paper-printed counts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tbsci_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc + OpenMP into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int
            lib.orc_fci_strings.argtypes = [i32, i32, P, i64]
            lib.orc_fci_strings.restype = i64
            lib.orc_sort_validate.argtypes = [i32, i32, P, i64, P]
            lib.orc_sort_validate.restype = i32
            lib.orc_links_single.argtypes = [i32, P, i64, P, P, P, P, P]
            lib.orc_links_single.restype = i64
            lib.orc_links_double.argtypes = [i32, P, i64, P, P, P, P, P, P, P]
            lib.orc_links_double.restype = i64
            lib.orc_row_capacity.argtypes = [i32, i32, i32]
            lib.orc_row_capacity.restype = i64
            lib.orc_row.argtypes = [i32, P, i64, P, i64, P, P, ctypes.c_double, i64, P, P]
            lib.orc_row.restype = i64
            lib.orc_sigma_rows.argtypes = [i32, i32, i32, P, i64, P, i64, P, P, ctypes.c_double,
                                           P, i32, P, i64, P, P, i32]
            lib.orc_sigma_rows.restype = None
            lib.orc_diagonal.argtypes = [i32, P, i64, P, i64, P, P, ctypes.c_double, P, i64, P]
            lib.orc_diagonal.restype = None
            lib.orc_sigma_pruned.argtypes = [i32, i32, i32, P, i64, P, i64, P, P, P, P, ctypes.c_double,
                                             P, i32, P, i64, P, P, i32]
            lib.orc_sigma_pruned.restype = None
            lib.orc_diagonal_pruned.argtypes = [i32, P, i64, P, P, P, P, P, ctypes.c_double, P, i64, P]
            lib.orc_diagonal_pruned.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ----------------------------------------------------------------- strings

def fci_strings(norb: int, nelec: int) -> np.ndarray:
    """All ``C(norb, nelec)`` strings, ascending (Sec. II.A, Eq. 3 with every
    string selected)."""
    lib = _load()
    m = lib.orc_fci_strings(norb, nelec, None, 0)
    out = np.zeros(m, dtype=np.uint64)
    lib.orc_fci_strings(norb, nelec, _ptr(out), m)
    return out


def sort_validate(norb: int, nelec: int, strings) -> tuple[int, np.ndarray]:
    """Sorted copy of a selected list and a status: 0 ok, 1 wrong electron count,
    2 bit at or above ``norb``, 3 duplicate."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(strings, dtype=np.uint64))
    out = np.zeros_like(a)
    st = lib.orc_sort_validate(norb, nelec, _ptr(a), len(a), _ptr(out))
    return int(st), out


# ------------------------------------------------------------ link tables

def links_single(norb: int, strings: np.ndarray):
    """Single links per source string (Sec. II.C BETA_SINGLE_LINK; entry fields of
    Sec. III.C): ``(off[l+1], tgt, sign, p, q)``; target ``a+_p a_q |J>``,
    rows ordered by ``(q, p)``."""
    lib = _load()
    s = np.ascontiguousarray(strings, dtype=np.uint64)
    l = len(s)
    off = np.zeros(l + 1, dtype=np.int64)
    m = lib.orc_links_single(norb, _ptr(s), l, _ptr(off), None, None, None, None)
    tgt = np.zeros(m, dtype=np.int32)
    sign = np.zeros(m, dtype=np.int8)
    p = np.zeros(m, dtype=np.uint8)
    q = np.zeros(m, dtype=np.uint8)
    lib.orc_links_single(norb, _ptr(s), l, _ptr(off), _ptr(tgt), _ptr(sign), _ptr(p), _ptr(q))
    return off, tgt, sign, p, q


def links_double(norb: int, strings: np.ndarray):
    """Double links per source string (Sec. II.C BETA_DOUBLE_LINK):
    ``(off, tgt, sign, p, r, q, s)``; target ``a+_p a+_r a_s a_q |J>``, q < s,
    p < r, rows ordered by ``(q, s, p, r)``."""
    lib = _load()
    st = np.ascontiguousarray(strings, dtype=np.uint64)
    l = len(st)
    off = np.zeros(l + 1, dtype=np.int64)
    m = lib.orc_links_double(norb, _ptr(st), l, _ptr(off), None, None, None, None, None, None)
    arrs = [np.zeros(m, dtype=np.int32), np.zeros(m, dtype=np.int8)] + [np.zeros(m, dtype=np.uint8) for _ in range(4)]
    lib.orc_links_double(norb, _ptr(st), l, _ptr(off), *[_ptr(a) for a in arrs])
    return (off, *arrs)


# ------------------------------------------------------------- Hamiltonian

class Space:
    """A TPB determinant space (Sec. II.A, Eq. 3): sorted alpha and beta sets."""

    def __init__(self, norb, nalpha, nbeta, alpha, beta):
        self.norb, self.na, self.nb = int(norb), int(nalpha), int(nbeta)
        self.sa = np.ascontiguousarray(alpha, dtype=np.uint64)
        self.sb = np.ascontiguousarray(beta, dtype=np.uint64)
        if len(self.sa) > 1 and not np.all(self.sa[1:] > self.sa[:-1]):
            raise ValueError("alpha strings must be strictly ascending")
        if len(self.sb) > 1 and not np.all(self.sb[1:] > self.sb[:-1]):
            raise ValueError("beta strings must be strictly ascending")
        self.la, self.lb = len(self.sa), len(self.sb)
        self.ndet = self.la * self.lb


def make_space(norb, nalpha, nbeta, alpha_sel=None, beta_sel=None) -> Space:
    """Space from optional selections (``None`` = full string space)."""
    if alpha_sel is None:
        sa = fci_strings(norb, nalpha)
    else:
        st, sa = sort_validate(norb, nalpha, alpha_sel)
        if st:
            raise ValueError("bad alpha selection (status %d)" % st)
    if beta_sel is None:
        sb = fci_strings(norb, nbeta)
    else:
        st, sb = sort_validate(norb, nbeta, beta_sel)
        if st:
            raise ValueError("bad beta selection (status %d)" % st)
    return Space(norb, nalpha, nbeta, sa, sb)


def _ham_arrays(h, eri):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = h.shape[0]
    assert eri.shape == (n, n, n, n)
    return h, eri


def sigma(space: Space, h, eri, ecore, C, rows=None, nthreads: int = 0, with_bound: bool = False):
    """sigma = H.c (Sec. II.B, Eq. 7 with one process) over the listed determinant rows.

    ``C``: ``[nvec, la, lb]`` or ``[nvec, ndet]`` float64. Returns ``[nvec, nrows]``
    (and ``sum_J |H_KJ||c_J|`` when ``with_bound``)."""
    lib = _load()
    h, eri = _ham_arrays(h, eri)
    C = np.ascontiguousarray(np.asarray(C, dtype=np.float64).reshape(-1, space.ndet))
    nvec = C.shape[0]
    if rows is None:
        nrows = space.ndet
        rows_arr = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = len(rows_arr)
    out = np.zeros((nvec, nrows))
    bound = np.zeros((nvec, nrows)) if with_bound else None
    lib.orc_sigma_rows(space.norb, space.na, space.nb, _ptr(space.sa), space.la, _ptr(space.sb), space.lb,
                       _ptr(h), _ptr(eri), float(ecore), _ptr(C), nvec, _ptr(rows_arr), nrows,
                       _ptr(out), _ptr(bound), int(nthreads))
    return (out, bound) if with_bound else out


def diagonal(space: Space, h, eri, ecore, rows=None) -> np.ndarray:
    """H_KK (Sec. II.C, the stored [0,0] class) for the listed rows (all by default)."""
    lib = _load()
    h, eri = _ham_arrays(h, eri)
    if rows is None:
        rows_arr, nrows = None, space.ndet
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = len(rows_arr)
    out = np.zeros(nrows)
    lib.orc_diagonal(space.norb, _ptr(space.sa), space.la, _ptr(space.sb), space.lb, _ptr(h), _ptr(eri),
                     float(ecore), _ptr(rows_arr), nrows, _ptr(out))
    return out


def row(space: Space, h, eri, ecore, K: int):
    """Non-zero elements ``(cols, vals)`` of row K of H, diagonal first."""
    lib = _load()
    h, eri = _ham_arrays(h, eri)
    cap = lib.orc_row_capacity(space.norb, space.na, space.nb)
    cols = np.zeros(cap, dtype=np.int64)
    vals = np.zeros(cap)
    m = lib.orc_row(space.norb, _ptr(space.sa), space.la, _ptr(space.sb), space.lb, _ptr(h), _ptr(eri),
                    float(ecore), int(K), _ptr(cols), _ptr(vals))
    return cols[:m].copy(), vals[:m].copy()


def hamiltonian_dense(space: Space, h, eri, ecore) -> np.ndarray:
    """Dense H over the space (small spaces only)."""
    H = np.zeros((space.ndet, space.ndet))
    for K in range(space.ndet):
        cols, vals = row(space, h, eri, ecore, K)
        H[K, cols] = vals
    return H


# ------------------------------------------- bitstring selection (Sec. III.B)

def string_weights(C, la: int, lb: int):
    """Weights of the alpha and beta strings of a TPB vector (Sec. III.B): after
    normalising, W_a(w) = sum_u c(w, u)^2 and W_b(u) = sum_w c(w, u)^2."""
    c = np.asarray(C, dtype=np.float64).reshape(la, lb)
    c = c / np.linalg.norm(c)
    return (c * c).sum(axis=1), (c * c).sum(axis=0)


def select_by_weight(weights, delta: float, ref: int | None = None):
    """Indices (ascending) of the strings whose weight is at least ``delta``
    times the HF string's weight (Sec. III.B). The HF string is ``ref`` when
    given, else the string of largest weight."""
    w = np.asarray(weights, dtype=np.float64)
    h = w[int(np.argmax(w))] if ref is None else w[ref]
    return np.nonzero(w >= delta * h)[0]


def coefficient_histogram(C, edges):
    """Counts of |c_K| per bin [edges[k], edges[k+1]) (Fig. 3 bins |c_K / c_HF|
    on a logarithmic scale; the caller scales the edges by |c_HF|). Returns
    ``nbins + 2`` counts: below edges[0], the bins, at or above edges[-1]."""
    a = np.abs(np.asarray(C, dtype=np.float64).ravel())
    e = np.asarray(edges, dtype=np.float64)
    idx = np.searchsorted(e, a, side="right")  # 0: below the first edge
    return np.bincount(idx, minlength=len(e) + 1).astype(np.int64)


# ---------------------------------------------------- pruned spaces (D_TBSCI)

class PrunedSpace:
    """The general TBSCI space (Sec. II.A, Eq. 6): the determinants (w, u) of a
    TPB space with u in I_w, given as CSR ``off[la + 1]`` and ascending beta
    indices ``cols``. Determinant (w, u) has the compressed index
    ``off[w] + position of u in I_w``."""

    def __init__(self, space: Space, off, cols):
        self.space = space
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        if len(self.off) != space.la + 1 or self.off[0] != 0 or np.any(np.diff(self.off) < 0):
            raise ValueError("off must be a CSR offset array of length la + 1")
        if self.off[-1] != len(self.cols):
            raise ValueError("off[la] must equal len(cols)")
        for w in range(space.la):
            row = self.cols[self.off[w]:self.off[w + 1]]
            if len(row) and (row.min() < 0 or row.max() >= space.lb or np.any(np.diff(row) <= 0)):
                raise ValueError("I_w must hold ascending beta indices inside the beta set")
        self.ndet = int(self.off[-1])

    def members(self) -> np.ndarray:
        """TPB indices w * lb + u of the member determinants, in compressed order."""
        w = np.repeat(np.arange(self.space.la, dtype=np.int64), np.diff(self.off))
        return w * self.space.lb + self.cols


def string_irrep(s: int, irreps) -> int:
    """Irrep of a string in an abelian point group: the XOR of the labels of its
    occupied orbitals (product of one-electron irreps, Sec. II.A on symmetry)."""
    out = 0
    for i in range(len(irreps)):
        if (int(s) >> i) & 1:
            out ^= int(irreps[i])
    return out


def symmetry_space(space: Space, irreps, target: int) -> PrunedSpace:
    """The symmetry-allowed determinants of a TPB space (Sec. II.A): (w, u) with
    irrep(w) XOR irrep(u) = target."""
    ga = [string_irrep(s, irreps) for s in space.sa]
    gb = [string_irrep(s, irreps) for s in space.sb]
    cols, off = [], [0]
    for w in range(space.la):
        row = [u for u in range(space.lb) if ga[w] ^ gb[u] == target]
        cols.extend(row)
        off.append(len(cols))
    return PrunedSpace(space, np.array(off, dtype=np.int64), np.array(cols, dtype=np.int32))


def sigma_pruned(ps: PrunedSpace, h, eri, ecore, C, rows=None, nthreads: int = 0, with_bound: bool = False):
    """sigma = H.c over a pruned space (Sec. II.A, Eq. 6; Sec. II.C, the membership
    test of Algorithm 1 written as a lookup in I_w). ``C``: ``[nvec, ndet]``
    compressed; returns ``[nvec, nrows]`` (and ``sum_J |H_KJ||c_J|``)."""
    lib = _load()
    h, eri = _ham_arrays(h, eri)
    sp = ps.space
    C = np.ascontiguousarray(np.asarray(C, dtype=np.float64).reshape(-1, ps.ndet))
    nvec = C.shape[0]
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = ps.ndet if rows is None else len(rows_arr)
    out = np.zeros((nvec, nrows))
    bound = np.zeros((nvec, nrows)) if with_bound else None
    lib.orc_sigma_pruned(sp.norb, sp.na, sp.nb, _ptr(sp.sa), sp.la, _ptr(sp.sb), sp.lb, _ptr(ps.off),
                         _ptr(ps.cols), _ptr(h), _ptr(eri), float(ecore), _ptr(C), nvec, _ptr(rows_arr), nrows,
                         _ptr(out), _ptr(bound), int(nthreads))
    return (out, bound) if with_bound else out


def diagonal_pruned(ps: PrunedSpace, h, eri, ecore, rows=None) -> np.ndarray:
    """H_KK of the member determinants (compressed order)."""
    lib = _load()
    h, eri = _ham_arrays(h, eri)
    sp = ps.space
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = ps.ndet if rows is None else len(rows_arr)
    out = np.zeros(nrows)
    lib.orc_diagonal_pruned(sp.norb, _ptr(sp.sa), sp.la, _ptr(sp.sb), _ptr(ps.off), _ptr(ps.cols), _ptr(h),
                            _ptr(eri), float(ecore), _ptr(rows_arr), nrows, _ptr(out))
    return out


def hamiltonian_dense_pruned(ps: PrunedSpace, h, eri, ecore) -> np.ndarray:
    """Dense H over a pruned space (small spaces only), column by column from
    sigma of unit vectors."""
    E = np.eye(ps.ndet)
    return sigma_pruned(ps, h, eri, ecore, E).T.copy()


def solve_pruned(ps: PrunedSpace, h, eri, ecore, nroots, nthreads=0, **kw):
    """Lowest eigenpairs of H on a pruned space: oracle sigma + oracle Davidson."""
    d = diagonal_pruned(ps, h, eri, ecore)

    def apply_h(V):
        return sigma_pruned(ps, h, eri, ecore, V, nthreads=nthreads)

    return davidson(apply_h, d, nroots, **kw)


# --------------------------------------------------------------- Davidson

def davidson(apply_h, diag, nroots, tol_e=1e-9, tol_r=1e-5, max_subspace=None, max_iter=1000,
             restart_keep=None, restart_prev=True):
    """Standard Davidson (Sec. III.A) for the lowest ``nroots`` eigenpairs.

    Steps, in order, each iteration: Rayleigh matrix G = V^T W; eigenpairs of G;
    Ritz vectors X = V Y and residuals R = W Y - X diag(theta); stop when every
    root has |theta - theta_prev| < tol_e and ||r|| < tol_r; otherwise precondition
    each unconverged residual by (theta - H_KK)^-1 (denominators of magnitude
    below 1e-8 clamped to +-1e-8, zero -> +1e-8); when the subspace would exceed
    ``max_subspace`` restart from the lowest ``restart_keep`` Ritz vectors
    (default ``max(nroots, max_subspace // 2)``; the paper's restart scheme,
    Sec. III.C, keeps a bounded number of vectors and says no more), and with
    ``restart_prev`` also the previous iteration's Ritz vectors, orthonormalised
    against the kept ones in the coefficient space of the basis (while room is
    left for one correction); orthogonalise
    the new directions twice against the basis and each other, normalise, and
    drop those whose norm fell below 1e-10 of their pre-projection norm.

    ``apply_h(V)`` maps ``[k, N]`` to ``[k, N]``. Guess: guess k is the unit
    vector at the k-th lowest diagonal entry (ties broken by index) plus
    0.1 * (1 + ((j + k) mod 4)) / 4 times the unit vector at the (nroots + j)-th
    lowest, j < 4, orthonormalised in order -- every guess then has components in
    every symmetry sector (with identical alpha and beta sets H commutes with the
    alpha-beta transpose, and a closed-shell guess alone would never leave its
    sector). Returns ``(energies, vectors[nroots, N], info)``.
    """
    diag = np.asarray(diag, dtype=np.float64)
    N = len(diag)
    if max_subspace is None:
        max_subspace = max(8 * nroots, nroots + 2)
    if restart_keep is None:
        restart_keep = max(nroots, max_subspace // 2)
    order = np.lexsort((np.arange(N), diag))
    extra = min(4, N - nroots)
    V = np.zeros((nroots, N))
    for k in range(nroots):
        V[k, order[k]] = 1.0
        for j in range(extra):
            V[k, order[nroots + j]] += 0.1 * (1.0 + ((j + k) % 4)) / 4.0
    for k in range(nroots):
        for i in range(k):
            V[k] -= (V[i] @ V[k]) * V[i]
        V[k] /= np.linalg.norm(V[k])
    W = apply_h(V)
    nsigma = nroots
    theta_prev = None
    p_prev = None  # the previous iteration's Ritz vectors, coefficients in the current basis
    info = dict(iterations=0, converged=False, nsigma=0)
    for it in range(1, max_iter + 1):
        G = V @ W.T
        G = 0.5 * (G + G.T)
        evals, Yall = np.linalg.eigh(G)
        theta = evals[:nroots]
        Y = Yall[:, :nroots]
        X = Y.T @ V
        WY = Y.T @ W
        R = WY - theta[:, None] * X
        rnorm = np.linalg.norm(R, axis=1)
        dE = np.full(nroots, np.inf) if theta_prev is None else np.abs(theta - theta_prev)
        theta_prev = theta.copy()
        info.update(iterations=it, rnorm=rnorm.copy(), nsigma=nsigma)
        if np.all(dE < tol_e) and np.all(rnorm < tol_r):
            info["converged"] = True
            return theta, X, info
        T = []
        for k in range(nroots):
            if rnorm[k] < tol_r:
                continue
            d = theta[k] - diag
            small = np.abs(d) < 1e-8
            d[small] = np.where(d[small] < 0, -1e-8, 1e-8)
            T.append(R[k] / d)
        p_cur = Y
        if V.shape[0] + len(T) > max_subspace:
            keep = min(restart_keep, V.shape[0])
            Q = Yall[:, :keep]
            if restart_prev and p_prev is not None:
                extra = []
                for z in p_prev.T:
                    z0 = np.linalg.norm(z)
                    for _ in range(2):
                        z = z - Q @ (Q.T @ z)
                        for u in extra:
                            z = z - (u @ z) * u
                    nz = np.linalg.norm(z)
                    if nz > 1e-8 * z0 and keep + len(extra) + 1 < max_subspace:
                        extra.append(z / nz)
                if extra:
                    Q = np.hstack([Q, np.array(extra).T])
            V, W = Q.T @ V, Q.T @ W
            p_cur = Q.T @ Y
        newV = []
        for t in T:
            t0 = np.linalg.norm(t)
            for _ in range(2):
                t = t - V.T @ (V @ t)
                for u in newV:
                    t = t - (u @ t) * u
            nt = np.linalg.norm(t)
            if nt <= 1e-10 * t0:
                continue
            newV.append(t / nt)
        if newV:
            Vn = np.array(newV)
            Wn = apply_h(Vn)
            nsigma += len(newV)
            V = np.vstack([V, Vn])
            W = np.vstack([W, Wn])
        p_prev = np.vstack([p_cur, np.zeros((V.shape[0] - p_cur.shape[0], nroots))])
    info["converged"] = False
    return theta_prev, X, info


def solve(space: Space, h, eri, ecore, nroots, nthreads=0, **kw):
    """Lowest eigenpairs of H on the space: oracle sigma + oracle Davidson."""
    d = diagonal(space, h, eri, ecore)

    def apply_h(V):
        return sigma(space, h, eri, ecore, V, nthreads=nthreads)

    return davidson(apply_h, d, nroots, **kw)
