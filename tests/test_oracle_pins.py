"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each check is chosen so that a plausible slip in the oracle (a dropped exchange
term, a wrong sign convention, a transposed integral index, a missed
excitation class, a wrong table order) fails at least one of them:

* brute-force second quantisation of H = sum h a+a + 1/2 sum (pq|rs) a+a+aa
  on tiny spaces (independent of the Slater-Condon rules the oracle uses);
* closed forms: one-electron systems, N_alpha = N_beta = 1 FCI Hamiltonian
  h x 1 + 1 x h + (ij|kl), one-electron eigenvalue sums;
* invariants: symmetry, particle-number shift, spin flip, total spin ([H, S^2] = 0
  with S^2 built from spin-orbital operators), variational order;
* paper-printed numbers: Table VI single-link entry counts (Sec. III.C).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from tbsci_inputs import synth_hamiltonian, selected_strings

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ brute force

def _annihilate(occ, P):
    if P not in occ:
        return 0, None
    i = occ.index(P)
    return (-1) ** i, occ[:i] + occ[i + 1:]


def _create(occ, P):
    if P in occ:
        return 0, None
    i = sum(1 for x in occ if x < P)
    return (-1) ** i, tuple(sorted(occ + (P,)))


def _apply(ops, occ):
    """Apply an operator product (leftmost acts last) to a determinant."""
    sign = 1
    for kind, P in reversed(ops):
        s, occ = (_create if kind == "c" else _annihilate)(occ, P)
        if s == 0:
            return 0, None
        sign *= s
    return sign, occ


def brute_force_h(n, sa, sb, h, eri, ecore):
    """Dense H over the TPB space from the second-quantised operator sum."""
    dets = []
    for a in sa:
        for b in sb:
            occ = tuple([p for p in range(n) if (int(a) >> p) & 1] + [n + p for p in range(n) if (int(b) >> p) & 1])
            dets.append(occ)
    index = {d: k for k, d in enumerate(dets)}
    N = len(dets)
    H = np.zeros((N, N))
    spins = (0, n)
    for J, occ in enumerate(dets):
        H[J, J] += ecore
        for sg in spins:
            for p in range(n):
                for q in range(n):
                    s, new = _apply([("c", sg + p), ("a", sg + q)], occ)
                    if s and new in index:
                        H[index[new], J] += s * h[p, q]
        for s1 in spins:
            for s2 in spins:
                for p, q, r, s_ in itertools.product(range(n), repeat=4):
                    v = eri[p, q, r, s_]
                    if v == 0.0:
                        continue
                    sgn, new = _apply([("c", s1 + p), ("c", s2 + r), ("a", s2 + s_), ("a", s1 + q)], occ)
                    if sgn and new in index:
                        H[index[new], J] += 0.5 * sgn * v
    return H


@pytest.mark.parametrize("n,na,nb,sel", [(3, 1, 1, None), (4, 2, 1, None), (4, 2, 2, None),
                                         (5, 2, 2, 6), (5, 3, 2, None)])
def test_dense_h_matches_second_quantisation(n, na, nb, sel):
    h, eri, _ = synth_hamiltonian(n, seed=11 + n + na)
    ecore = 0.37
    asel = None if sel is None else selected_strings(n, na, sel, seed=5)
    bsel = None if sel is None else selected_strings(n, nb, sel, seed=6)
    sp = oracle.make_space(n, na, nb, asel, bsel)
    H = oracle.hamiltonian_dense(sp, h, eri, ecore)
    Hb = brute_force_h(n, sp.sa, sp.sb, h, eri, ecore)
    assert np.max(np.abs(H - Hb)) < 1e-12


# ------------------------------------------------------------ closed forms

def test_one_electron_alpha_only_is_h():
    n = 7
    h, eri, _ = synth_hamiltonian(n, seed=3)
    sp = oracle.make_space(n, 1, 0)
    assert sp.la == n and sp.lb == 1
    H = oracle.hamiltonian_dense(sp, h, eri, 0.5)
    # one alpha electron, no beta: H = h + ecore exactly (two-electron terms vanish)
    assert np.max(np.abs(H - (h + 0.5 * np.eye(n)))) < 1e-14


def test_one_plus_one_fci_closed_form():
    n = 6
    h, eri, _ = synth_hamiltonian(n, seed=4)
    sp = oracle.make_space(n, 1, 1)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    I = np.eye(n)
    ref = np.kron(h, I) + np.kron(I, h) + eri.transpose(0, 2, 1, 3).reshape(n * n, n * n)
    assert np.max(np.abs(H - ref)) < 1e-13


def test_one_electron_operator_eigenvalue_sum():
    n, na, nb = 7, 3, 2
    h, eri, _ = synth_hamiltonian(n, seed=9)
    sp = oracle.make_space(n, na, nb)
    H = oracle.hamiltonian_dense(sp, h, np.zeros_like(eri), 0.0)
    e = np.linalg.eigvalsh(h)
    assert abs(np.linalg.eigvalsh(H)[0] - (e[:na].sum() + e[:nb].sum())) < 1e-12


# ---------------------------------------------------------------- invariants

def test_symmetry_and_slater_condon_sparsity():
    n, na, nb = 6, 3, 3
    h, eri, _ = synth_hamiltonian(n, seed=21)
    sp = oracle.make_space(n, na, nb)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    assert np.max(np.abs(H - H.T)) <= 1e-14 * np.max(np.abs(H))
    # Eq. 8: no coupling beyond two differing spin orbitals in total
    pc = np.vectorize(lambda x: bin(int(x)).count("1"))
    da = pc(np.bitwise_xor.outer(sp.sa, sp.sa)) // 2
    db = pc(np.bitwise_xor.outer(sp.sb, sp.sb)) // 2
    diff = (da[:, None, :, None] + db[None, :, None, :]).reshape(sp.ndet, sp.ndet)
    assert np.all(H[diff > 2] == 0.0)
    # all six classes [a,b] with a+b <= 2 occur
    classes = {(int(a), int(b)) for a in range(3) for b in range(3) if a + b <= 2}
    found = set()
    for a, b in classes:
        m = (da[:, None, :, None] == a) & (db[None, :, None, :] == b)
        if np.any(H[m.reshape(sp.ndet, sp.ndet)] != 0.0):
            found.add((a, b))
    assert found == classes


def test_sigma_matches_dense_and_bound():
    n, na, nb = 6, 3, 2
    h, eri, _ = synth_hamiltonian(n, seed=22)
    sp = oracle.make_space(n, na, nb, None, selected_strings(n, nb, 9, seed=1))
    H = oracle.hamiltonian_dense(sp, h, eri, 0.1)
    C = np.random.default_rng(0).standard_normal((2, sp.ndet))
    S, B = oracle.sigma(sp, h, eri, 0.1, C, with_bound=True)
    assert np.max(np.abs(S - C @ H.T)) < 1e-12
    assert np.max(np.abs(B - np.abs(C) @ np.abs(H).T)) < 1e-12
    rows = np.array([3, 0, sp.ndet - 1])
    assert np.max(np.abs(oracle.sigma(sp, h, eri, 0.1, C, rows=rows) - S[:, rows])) == 0.0
    assert np.max(np.abs(oracle.diagonal(sp, h, eri, 0.1) - np.diag(H))) < 1e-13


def test_particle_number_shift():
    n, na, nb = 8, 4, 3
    h, eri, _ = synth_hamiltonian(n, seed=23)
    sp = oracle.make_space(n, na, nb, selected_strings(n, na, 40, seed=2), None)
    C = np.random.default_rng(1).standard_normal((1, sp.ndet))
    eps = 0.25
    s0 = oracle.sigma(sp, h, eri, 0.0, C)
    s1 = oracle.sigma(sp, h + eps * np.eye(n), eri, 0.0, C)
    assert np.max(np.abs(s1 - s0 - eps * (na + nb) * C)) < 1e-12


def test_spin_flip_transpose():
    n = 8
    h, eri, _ = synth_hamiltonian(n, seed=24)
    sel = selected_strings(n, 4, 50, seed=3)
    sp = oracle.make_space(n, 4, 4, sel, sel)
    C = np.random.default_rng(2).standard_normal((sp.la, sp.lb))
    s = oracle.sigma(sp, h, eri, 0.0, C[None]).reshape(sp.la, sp.lb)
    st = oracle.sigma(sp, h, eri, 0.0, C.T.copy()[None]).reshape(sp.la, sp.lb)
    assert np.max(np.abs(st - s.T)) < 1e-12


def _s_plus(n, na, nb):
    """S+ = sum_p a+_{p alpha} a_{p beta} from the full (na, nb) space to the full
    (na + 1, nb - 1) space, spin orbitals ordered alpha block first, ascending
    inside each block (the determinant phase convention), determinants indexed
    alpha-major over ascending integer strings; written from the operator
    definition, independent of the oracle's Slater-Condon code."""
    def strings(N):
        return sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), N))
    sa, sb = strings(na), strings(nb)
    ta, tb = strings(na + 1), strings(nb - 1)
    ia, ib = {s: i for i, s in enumerate(ta)}, {s: i for i, s in enumerate(tb)}
    S = np.zeros((len(ta) * len(tb), len(sa) * len(sb)))
    for w, a in enumerate(sa):
        for u, b in enumerate(sb):
            for p in range(n):
                if not (b >> p) & 1 or (a >> p) & 1:
                    continue
                # a_{p beta}: passes all na alpha electrons and the betas below p
                sign = (-1) ** (na + bin(b & ((1 << p) - 1)).count("1"))
                # a+_{p alpha}: passes the alphas below p
                sign *= (-1) ** bin(a & ((1 << p) - 1)).count("1")
                a2, b2 = a | (1 << p), b & ~(1 << p)
                S[ia[a2] * len(tb) + ib[b2], w * len(sb) + u] += sign
    return S


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (6, 3, 2), (7, 3, 3)])
def test_hamiltonian_commutes_with_total_spin(n, na, nb):
    """[H, S^2] = 0 for the oracle's H on full string spaces, and every eigenvector
    has <S^2> = s(s + 1): an exchange sign, a dropped exchange term or a phase
    convention that disagrees between the classes breaks spin symmetry."""
    h, eri, _ = synth_hamiltonian(n, seed=50 + n)
    sp = oracle.make_space(n, na, nb)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    Sp = _s_plus(n, na, nb)
    sz = (na - nb) / 2.0
    S2 = Sp.T @ Sp + (sz * sz + sz) * np.eye(H.shape[0])
    assert np.max(np.abs(H @ S2 - S2 @ H)) < 1e-11 * np.max(np.abs(H))
    w, U = np.linalg.eigh(H)
    gaps = np.diff(w)
    for k in range(min(12, len(w))):
        if (k > 0 and gaps[k - 1] < 1e-8) or (k + 1 < len(w) and gaps[k] < 1e-8):
            continue  # degenerate: any mix of the multiplets is an eigenvector
        s2 = U[:, k] @ S2 @ U[:, k]
        s = (-1 + math.sqrt(1 + 4 * s2)) / 2
        assert abs(s2 - round(2 * s) / 2 * (round(2 * s) / 2 + 1)) < 1e-8, (k, s2)
        assert round(2 * s) % 2 == (na - nb) % 2 and round(2 * s) >= abs(na - nb)


def test_variational_nested_selections():
    n, na, nb = 8, 4, 4
    h, eri, _ = synth_hamiltonian(n, seed=25)
    full = oracle.make_space(n, na, nb)
    e_fci = np.linalg.eigvalsh(oracle.hamiltonian_dense(full, h, eri, 0.0))[0]
    last = np.inf
    order = selected_strings(n, na, 70, seed=4, shuffle=False)
    for cnt in (10, 25, 45, 70):
        sub = order[:cnt]
        sp = oracle.make_space(n, na, nb, sub, sub)
        e0 = np.linalg.eigvalsh(oracle.hamiltonian_dense(sp, h, eri, 0.0))[0]
        assert e0 <= last + 1e-12
        assert e0 >= e_fci - 1e-12
        last = e0
    assert abs(last - e_fci) < 1e-10


# ------------------------------------------------------------ strings / links

def test_fci_strings_against_combinations():
    for n, N in [(1, 0), (1, 1), (6, 3), (10, 4), (12, 6)]:
        s = oracle.fci_strings(n, N)
        ref = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), N))
        assert list(map(int, s)) == ref


def test_sort_validate_errors():
    ok, out = oracle.sort_validate(6, 2, [0b110000, 0b11, 0b101])
    assert ok == 0 and list(map(int, out)) == [0b11, 0b101, 0b110000]
    assert oracle.sort_validate(6, 2, [0b111])[0] == 1
    assert oracle.sort_validate(6, 2, [0b1000001])[0] == 2
    assert oracle.sort_validate(6, 2, [0b11, 0b11])[0] == 3


def _bf_single_links(n, strs):
    index = {int(s): i for i, s in enumerate(strs)}
    rows = []
    for s in strs:
        occ = tuple(p for p in range(n) if (int(s) >> p) & 1)
        row = []
        for q in range(n):
            for p in range(n):
                if p == q:
                    continue
                sg, new = _apply([("c", p), ("a", q)], occ)
                if sg == 0:
                    continue
                t = sum(1 << x for x in new)
                if t in index:
                    row.append((index[t], sg, p, q))
        rows.append(row)
    return rows


def _bf_double_links(n, strs):
    index = {int(s): i for i, s in enumerate(strs)}
    rows = []
    for s in strs:
        occ = tuple(p for p in range(n) if (int(s) >> p) & 1)
        vir = [p for p in range(n) if p not in occ]
        row = []
        for q, s_ in itertools.combinations(occ, 2):
            for p, r in itertools.combinations(vir, 2):
                sg, new = _apply([("c", p), ("c", r), ("a", s_), ("a", q)], occ)
                t = sum(1 << x for x in new)
                if t in index:
                    row.append((index[t], sg, p, r, q, s_))
        rows.append(row)
    return rows


@pytest.mark.parametrize("n,N,sel", [(6, 3, None), (8, 4, None), (9, 3, 30), (10, 5, 60)])
def test_links_against_brute_force(n, N, sel):
    strs = oracle.fci_strings(n, N) if sel is None else oracle.sort_validate(n, N, selected_strings(n, N, sel, 7))[1]
    off, tgt, sign, p, q = oracle.links_single(n, strs)
    bf = _bf_single_links(n, strs)
    for i, row in enumerate(bf):
        got = list(zip(tgt[off[i]:off[i + 1]].tolist(), sign[off[i]:off[i + 1]].tolist(),
                       p[off[i]:off[i + 1]].tolist(), q[off[i]:off[i + 1]].tolist()))
        assert got == row
    off2, tgt2, sg2, p2, r2, q2, s2 = oracle.links_double(n, strs)
    bf2 = _bf_double_links(n, strs)
    for i, row in enumerate(bf2):
        sl = slice(off2[i], off2[i + 1])
        got = list(zip(tgt2[sl].tolist(), sg2[sl].tolist(), p2[sl].tolist(), r2[sl].tolist(),
                       q2[sl].tolist(), s2[sl].tolist()))
        assert got == row
    if sel is None:
        assert off[-1] == math.comb(n, N) * N * (n - N)
        assert off2[-1] == math.comb(n, N) * math.comb(N, 2) * math.comb(n - N, 2)


def test_single_link_reciprocity():
    n, N = 10, 5
    strs = oracle.sort_validate(n, N, selected_strings(n, N, 80, 8))[1]
    off, tgt, sign, p, q = oracle.links_single(n, strs)
    fwd = set()
    for j in range(len(strs)):
        for k in range(off[j], off[j + 1]):
            fwd.add((j, int(tgt[k]), int(sign[k]), int(p[k]), int(q[k])))
    for (j, i, sg, pp, qq) in fwd:
        assert (i, j, sg, qq, pp) in fwd


def _read_table6():
    rows = []
    with open(os.path.join(GOLDEN, "table6_single_links.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, n, nb, entries, gb = line.split()
                rows.append((name, int(n), int(nb), int(entries), float(gb)))
    return rows


def test_table6_single_link_counts_closed_form():
    """Paper Table VI (Sec. III.C): FCI single-link entry counts and their 7-byte
    footprint. The oracle's link count equals C(n,N) N (n-N) on full spaces
    (checked above by brute force), so this pins the count and byte model to the
    printed values."""
    rows = _read_table6()
    assert len(rows) == 4
    for name, n, nb, entries, gb in rows:
        assert math.comb(n, nb) * nb * (n - nb) == entries, name
        assert abs(entries * 7 / 2 ** 30 - gb) < 0.006, name


def test_oracle_link_count_matches_closed_form_medium():
    for n, N in [(12, 6), (14, 3)]:
        strs = oracle.fci_strings(n, N)
        off, *_ = oracle.links_single(n, strs)
        assert off[-1] == math.comb(n, N) * N * (n - N)


# ------------------------------------------------------------------ Davidson

def test_davidson_matches_dense_small():
    n, na, nb = 6, 3, 3
    h, eri, _ = synth_hamiltonian(n, seed=31)
    sp = oracle.make_space(n, na, nb)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    ref = np.linalg.eigvalsh(H)[:4]
    e, X, info = oracle.solve(sp, h, eri, 0.0, nroots=4, max_subspace=16)
    assert info["converged"]
    assert np.max(np.abs(e - ref)) < 1e-8
    for k in range(4):
        r = H @ X[k] - e[k] * X[k]
        assert np.linalg.norm(r) < 1e-5


def test_fci8_golden_energies():
    """Config norb=8, 4+4, all 70 x 70 strings: dense eigenvalues stored by
    tests/golden/make_golden.py (oracle + numpy eigh) and the oracle Davidson."""
    path = os.path.join(GOLDEN, "fci8_energies.txt")
    ref = np.loadtxt(path)
    from tbsci_inputs import WORKLOADS
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta)
    e, X, info = oracle.solve(sp, h, eri, ecore, nroots=3)
    assert info["converged"]
    assert np.max(np.abs(e - ref[:3])) < 1e-8


def test_davidson_finds_a_transpose_antisymmetric_ground_state():
    """norb 6, 3+3 electrons, all strings, seed 12: the lowest eigenvector is
    antisymmetric under the alpha-beta transpose while the lowest diagonal entry is
    a closed-shell determinant; the Davidson guess must still reach it."""
    n, N = 6, 3
    h, eri, _ = synth_hamiltonian(n, seed=12)
    sp = oracle.make_space(n, N, N)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    w, U = np.linalg.eigh(H)
    x = U[:, 0].reshape(sp.la, sp.lb)
    assert np.linalg.norm(x + x.T) < 1e-8
    d = np.diag(H)
    K = np.lexsort((np.arange(len(d)), d))[0]
    assert K // sp.lb == K % sp.lb
    for nroots in (1, 2, 3):
        e, X, info = oracle.davidson(lambda V: V @ H.T, d, nroots)
        assert info["converged"]
        assert np.max(np.abs(e - w[:nroots])) < 1e-8


# ------------------------------------------------- pruned spaces (D_TBSCI)

def _pruned_case(n, na, nb, acnt, bcnt, max_level, seed):
    from tbsci_inputs import prune_by_total_level
    h, eri, _ = synth_hamiltonian(n, seed=seed)
    asel = None if acnt is None else selected_strings(n, na, acnt, seed + 1)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, seed + 2)
    sp = oracle.make_space(n, na, nb, asel, bsel)
    off, cols = prune_by_total_level(sp.sa, sp.sb, na, nb, max_level)
    return sp, oracle.PrunedSpace(sp, off, cols), h, eri


def test_pruned_h_is_the_brute_force_h_on_the_members():
    """Second quantisation (independent of the Slater-Condon rules) on the
    member determinants only: the pruned oracle's dense H equals it."""
    n, na, nb = 5, 2, 2
    sp, ps, h, eri = _pruned_case(n, na, nb, None, None, 2, seed=71)
    assert 0 < ps.ndet < sp.ndet
    H = oracle.hamiltonian_dense_pruned(ps, h, eri, 0.4)
    Hb = brute_force_h(n, sp.sa, sp.sb, h, eri, 0.4)
    m = ps.members()
    assert np.max(np.abs(H - Hb[np.ix_(m, m)])) < 1e-12


@pytest.mark.parametrize("n,na,nb,acnt,bcnt,lev", [(8, 4, 4, None, None, 3), (8, 4, 3, 40, None, 2),
                                                   (10, 5, 5, 120, 130, 4)])
def test_pruned_sigma_is_the_principal_submatrix_product(n, na, nb, acnt, bcnt, lev):
    """H restricted to D_TBSCI is the principal submatrix of H on its
    determinants: sigma_pruned(c) equals H_TPB applied to c zero-padded outside
    the space, read back at the members."""
    sp, ps, h, eri = _pruned_case(n, na, nb, acnt, bcnt, lev, seed=81 + n)
    assert 0 < ps.ndet < sp.ndet
    rng = np.random.default_rng(3)
    c = rng.standard_normal((2, ps.ndet))
    full = np.zeros((2, sp.ndet))
    full[:, ps.members()] = c
    want = oracle.sigma(sp, h, eri, 0.1, full)[:, ps.members()]
    got, bound = oracle.sigma_pruned(ps, h, eri, 0.1, c, with_bound=True)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(bound)
    assert np.allclose(oracle.diagonal_pruned(ps, h, eri, 0.1), oracle.diagonal(sp, h, eri, 0.1)[ps.members()],
                       atol=0, rtol=0)


def test_pruning_nothing_is_the_tpb_space():
    """I_w = every beta string: the pruned sigma is the TPB sigma bit for bit."""
    n, na, nb = 8, 4, 4
    h, eri, _ = synth_hamiltonian(n, seed=91)
    sp = oracle.make_space(n, na, nb, selected_strings(n, na, 50, 92), None)
    off = np.arange(sp.la + 1, dtype=np.int64) * sp.lb
    cols = np.tile(np.arange(sp.lb, dtype=np.int32), sp.la)
    ps = oracle.PrunedSpace(sp, off, cols)
    c = np.random.default_rng(4).standard_normal((1, sp.ndet))
    assert np.array_equal(oracle.sigma_pruned(ps, h, eri, 0.0, c), oracle.sigma(sp, h, eri, 0.0, c))


def test_pruned_spectrum_interlaces_and_is_variational():
    """Cauchy interlacing for a principal submatrix of size m of an N x N
    symmetric H: lambda_k(H) <= lambda_k(H_D) <= lambda_{k+N-m}(H); nested
    prunings give non-increasing ground-state energies (variational, Sec. II.A)."""
    n, na, nb = 8, 4, 4
    h, eri, _ = synth_hamiltonian(n, seed=93)
    sp = oracle.make_space(n, na, nb)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(sp, h, eri, 0.0))
    from tbsci_inputs import prune_by_total_level
    e0 = []
    for lev in (2, 4, 6, 8):
        off, cols = prune_by_total_level(sp.sa, sp.sb, na, nb, lev)
        ps = oracle.PrunedSpace(sp, off, cols)
        wd = np.linalg.eigvalsh(oracle.hamiltonian_dense_pruned(ps, h, eri, 0.0))
        m, N = ps.ndet, sp.ndet
        assert np.all(w[:m] <= wd + 1e-10) and np.all(wd <= w[N - m:] + 1e-10)
        e0.append(wd[0])
    assert all(a >= b - 1e-12 for a, b in zip(e0, e0[1:]))
    assert abs(e0[-1] - w[0]) < 1e-10  # level 8 keeps every determinant


def test_pruned_space_validation():
    sp = oracle.make_space(6, 3, 3)
    with pytest.raises(ValueError):
        oracle.PrunedSpace(sp, np.zeros(sp.la, dtype=np.int64), np.zeros(0, dtype=np.int32))
    off = np.zeros(sp.la + 1, dtype=np.int64)
    off[1:] = 2
    with pytest.raises(ValueError):  # descending beta indices
        oracle.PrunedSpace(sp, off, np.array([3, 1], dtype=np.int32))


def test_pruned_davidson_matches_dense():
    n, na, nb = 8, 4, 4
    sp, ps, h, eri = _pruned_case(n, na, nb, None, None, 3, seed=95)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense_pruned(ps, h, eri, 0.0))
    e, _, info = oracle.solve_pruned(ps, h, eri, 0.0, 3)
    assert info["converged"] and np.max(np.abs(e - w[:3])) < 1e-8


@pytest.mark.parametrize("name", ["sel16", "sel24"])
def test_workload_selection_centre_is_the_lowest_energy_string(name):
    """The selected workloads are centred on their lowest-energy string: the
    argmin over all C(n, N) strings of the one-spin string energy (the oracle's
    diagonal with no beta electron), ties to the smaller integer. The constant
    stored in tbsci_inputs must be that string, and the selection must hold it
    and every string within a double excitation of it."""
    from tbsci_inputs import WORKLOADS
    wl = WORKLOADS[name]
    h, eri, _ = wl.hamiltonian()
    sp = oracle.make_space(wl.norb, wl.nalpha, 0)
    E = oracle.diagonal(sp, h, eri, 0.0)
    assert int(sp.sa[int(np.argmin(E))]) == wl.reference
    sel = set(int(x) for x in wl.alpha_selection())
    ref = wl.reference
    near = [int(s) for s in sp.sa if bin(int(s) ^ ref).count("1") <= 4]
    assert ref in sel and all(s in sel for s in near)
    assert len(sel) == wl.count_alpha


# ------------------------------------------- bitstring selection (Sec. III.B)

def test_string_weights_sum_to_one_and_brute_force():
    rng = np.random.default_rng(11)
    C = rng.standard_normal((7, 5))
    wa, wb = oracle.string_weights(C, 7, 5)
    assert abs(wa.sum() - 1.0) < 1e-14 and abs(wb.sum() - 1.0) < 1e-14
    n2 = sum(C[i, j] ** 2 for i in range(7) for j in range(5))
    for i in range(7):
        assert abs(wa[i] - sum(C[i, j] ** 2 for j in range(5)) / n2) < 1e-15
    for j in range(5):
        assert abs(wb[j] - sum(C[i, j] ** 2 for i in range(7)) / n2) < 1e-15
    # a single determinant carries all the weight of its two strings
    D = np.zeros((7, 5))
    D[3, 2] = -2.0
    wa, wb = oracle.string_weights(D, 7, 5)
    assert wa[3] == 1.0 and wb[2] == 1.0 and wa.sum() == 1.0


def test_select_by_weight_threshold_semantics():
    w = np.array([0.5, 0.2, 0.05, 0.2, 0.05])
    assert list(oracle.select_by_weight(w, 1.0)) == [0]
    assert list(oracle.select_by_weight(w, 0.4)) == [0, 1, 3]
    assert list(oracle.select_by_weight(w, 0.1)) == [0, 1, 2, 3, 4]
    assert list(oracle.select_by_weight(w, 1.0, ref=1)) == [0, 1, 3]
    assert list(oracle.select_by_weight(w, 0.0)) == [0, 1, 2, 3, 4]


def test_coefficient_histogram_brute_force():
    rng = np.random.default_rng(12)
    c = rng.standard_normal(500) * 10.0 ** rng.uniform(-6, 0, 500)
    c[:3] = 0.0
    edges = 10.0 ** np.arange(-6, 1)
    got = oracle.coefficient_histogram(c, edges)
    want = np.zeros(len(edges) + 1, dtype=np.int64)
    for x in np.abs(c):
        k = 0
        while k < len(edges) and x >= edges[k]:
            k += 1
        want[k] += 1
    assert np.array_equal(got, want) and got.sum() == 500


# ------------------------------------------------ point-group symmetry blocks

@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (7, 3, 2)])
def test_symmetric_h_is_block_diagonal_and_blocks_give_the_spectrum(n, na, nb):
    """With D2h-labelled integrals (h and (ij|kl) vanish unless the labels
    multiply to the totally symmetric irrep) H couples only determinants of equal
    irrep: every element between different blocks is zero, and the union of the
    spectra of the eight symmetry blocks is the spectrum of H (dense, exact)."""
    from tbsci_inputs import orbital_irreps, synth_hamiltonian_symmetric
    g = orbital_irreps(n, seed=900 + n)
    h, eri, _ = synth_hamiltonian_symmetric(n, 901 + n, g)
    # the integrals obey the selection rule
    for i, j, k, l in itertools.product(range(n), repeat=4):
        if g[i] ^ g[j] ^ g[k] ^ g[l]:
            assert eri[i, j, k, l] == 0.0
    sp = oracle.make_space(n, na, nb)
    H = oracle.hamiltonian_dense(sp, h, eri, 0.0)
    Hb = brute_force_h(n, sp.sa, sp.sb, h, eri, 0.0)
    assert np.max(np.abs(H - Hb)) < 1e-12
    irr = np.array([oracle.string_irrep(a, g) ^ oracle.string_irrep(b, g) for a in sp.sa for b in sp.sb])
    assert np.all(H[irr[:, None] != irr[None, :]] == 0.0)
    spectra = []
    total = 0
    for t in range(8):
        ps = oracle.symmetry_space(sp, g, t)
        total += ps.ndet
        if ps.ndet:
            assert np.array_equal(ps.members(), np.nonzero(irr == t)[0])
            spectra.append(np.linalg.eigvalsh(oracle.hamiltonian_dense_pruned(ps, h, eri, 0.0)))
    assert total == sp.ndet
    assert np.max(np.abs(np.sort(np.concatenate(spectra)) - np.linalg.eigvalsh(H))) < 1e-10


def test_string_irrep_brute_force():
    g = [1, 2, 4, 3, 0, 7]
    for s in range(64):
        want = 0
        for i in range(6):
            if s & (1 << i):
                want ^= g[i]
        assert oracle.string_irrep(s, g) == want
