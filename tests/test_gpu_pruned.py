"""Pruned TBSCI spaces (D_TBSCI, Sec. II.A, Eq. 6): GPU sigma, diagonal and
Davidson on compressed vectors against the oracle's restriction of H to the
member determinants."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_sigma_close
from tbsci_inputs import WORKLOADS, prune_by_total_level, selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


@pytest.fixture(scope="module")
def ctx(tb):
    c = tb.Context(0)
    yield c
    c.close()


def _case(tb, ctx, n, na, nb, acnt, bcnt, level, seed, ecore=0.0):
    h, eri, _ = synth_hamiltonian(n, seed=seed)
    asel = None if acnt is None else selected_strings(n, na, acnt, seed + 1)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, seed + 2)
    sp = tb.Space(ctx, n, na, nb, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    off, cols = prune_by_total_level(osp.sa, osp.sb, na, nb, level)
    return sp, sp.prune(off, cols), oracle.PrunedSpace(osp, off, cols), h, eri


CASES = [
    # n, na, nb, alpha count, beta count, total excitation level, nvec
    (8, 4, 4, None, None, 3, 1),
    (8, 4, 3, 40, None, 2, 2),
    (10, 5, 5, 120, 257, 4, 3),   # ragged beta set; many rows with members scattered
    (12, 6, 6, 300, 280, 4, 1),
    (12, 6, 6, 300, 280, 1, 2),   # heavy pruning: most alpha rows empty
]


@pytest.mark.parametrize("n,na,nb,acnt,bcnt,level,nvec", CASES)
def test_pruned_sigma_f64_parity(tb, ctx, n, na, nb, acnt, bcnt, level, nvec):
    import torch
    sp, pr, ops, h, eri = _case(tb, ctx, n, na, nb, acnt, bcnt, level, seed=200 + n + level, ecore=0.3)
    assert pr.ndet == ops.ndet and 0 < pr.ndet < sp.ndet
    C = np.random.default_rng(n).standard_normal((nvec, pr.ndet))
    s = pr.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    ref, bound = oracle.sigma_pruned(ops, h, eri, 0.3, C, with_bound=True)
    assert_sigma_close(s, ref, bound)
    d = pr.diagonal().cpu().numpy()
    dref = oracle.diagonal_pruned(ops, h, eri, 0.3)
    assert np.max(np.abs(d - dref)) <= 1e-12 * max(1.0, np.max(np.abs(dref)))
    pr.close()
    sp.close()


def test_pruned_sigma_f32_parity(tb, ctx):
    import torch
    sp, pr, ops, h, eri = _case(tb, ctx, 12, 6, 6, 300, 280, 4, seed=311)
    C = np.random.default_rng(5).standard_normal((2, pr.ndet)).astype(np.float32)
    s = pr.sigma(torch.from_numpy(C).cuda()).double().cpu().numpy()
    ref, bound = oracle.sigma_pruned(ops, h, eri, 0.0, C.astype(np.float64), with_bound=True)
    assert_sigma_close(s, ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    pr.close()
    sp.close()


def test_pruning_nothing_matches_the_tpb_sigma(tb, ctx):
    """I_w = every beta string: the compressed vector is the dense one, and the
    pruned kernel gives the TPB kernel's sigma (different summation order)."""
    import torch
    n, na, nb = 10, 5, 5
    h, eri, _ = synth_hamiltonian(n, seed=17)
    sp = tb.Space(ctx, n, na, nb, h, eri, alpha=selected_strings(n, na, 90, 18), beta=selected_strings(n, nb, 70, 19))
    off = np.arange(sp.la + 1, dtype=np.int64) * sp.lb
    cols = np.tile(np.arange(sp.lb, dtype=np.int32), sp.la)
    pr = sp.prune(off, cols)
    C = torch.from_numpy(np.random.default_rng(6).standard_normal((2, sp.la, sp.lb))).cuda()
    dense = sp.sigma(C).cpu().numpy().reshape(2, -1)
    got = pr.sigma(C.reshape(2, -1).contiguous()).cpu().numpy()
    osp = oracle.make_space(n, na, nb, selected_strings(n, na, 90, 18), selected_strings(n, nb, 70, 19))
    _, bound = oracle.sigma(osp, h, eri, 0.0, C.cpu().numpy(), with_bound=True)
    assert_sigma_close(got, dense, bound)
    pr.close()
    sp.close()


def test_pruned_rows_longer_than_shared_memory(tb, ctx):
    """Full beta string space of norb 18 with 9 beta electrons (48,620 strings:
    389 KB per FP64 row) and 5 selected alpha strings, pruned by excitation level:
    c(Ja, Jb) is looked up by binary search in I_Ja. 400 sampled rows."""
    import torch
    n, na, nb = 18, 9, 9
    sp, pr, ops, h, eri = _case(tb, ctx, n, na, nb, 5, None, 4, seed=401)
    assert sp.lb == math.comb(18, 9) and pr.ndet > 0
    C = np.random.default_rng(7).standard_normal((1, pr.ndet))
    s = pr.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    rows = np.sort(np.random.default_rng(8).choice(pr.ndet, 400, replace=False))
    ref, bound = oracle.sigma_pruned(ops, h, eri, 0.0, C, rows=rows, with_bound=True)
    assert_sigma_close(s[:, rows], ref, bound)
    pr.close()
    sp.close()


@pytest.mark.parametrize("mixed", [0, 1])
def test_pruned_davidson_vs_dense(tb, ctx, mixed):
    sp, pr, ops, h, eri = _case(tb, ctx, 8, 4, 4, None, None, 3, seed=501, ecore=0.2)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense_pruned(ops, h, eri, 0.2))
    e, info, X = pr.davidson(3, want_vectors=True, mixed=mixed)
    assert info["converged"], info
    assert np.max(np.abs(e - w[:3])) < 1e-8, (e, w[:3])
    X = X.cpu().numpy()
    for k in range(3):
        hx = oracle.sigma_pruned(ops, h, eri, 0.2, X[k][None])[0]
        assert np.linalg.norm(hx - e[k] * X[k]) < 2e-5
    # variational: the pruned ground state lies above the TPB one
    e_tpb, _ = sp.davidson(1)
    assert e[0] >= e_tpb[0] - 1e-10
    pr.close()
    sp.close()


def test_pruned_sel16_sampled_rows_and_solves(tb, ctx):
    """norb 16, 3,000 x 3,000 selected strings pruned to total excitation level
    <= 4: 1,500 sampled rows of the FP64 sigma against the oracle, and the FP64
    and mixed-precision solves agree to 1e-8 Eh."""
    import torch
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, bsel)
    off, cols = prune_by_total_level(osp.sa, osp.sb, wl.nalpha, wl.nbeta, 4)
    pr = sp.prune(off, cols)
    ops = oracle.PrunedSpace(osp, off, cols)
    assert 0 < pr.ndet < sp.ndet
    C = np.random.default_rng(9).standard_normal((1, pr.ndet))
    s = pr.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    rows = np.sort(np.random.default_rng(10).choice(pr.ndet, 1500, replace=False))
    ref, bound = oracle.sigma_pruned(ops, h, eri, ecore, C, rows=rows, with_bound=True)
    assert_sigma_close(s[:, rows], ref, bound)
    e64, i64 = pr.davidson(1)
    e32, i32 = pr.davidson(1, mixed=1)
    assert i64["converged"] and i32["converged"]
    assert abs(e64[0] - e32[0]) < 1e-8
    pr.close()
    sp.close()


def test_pruned_edge_cases_and_errors(tb, ctx):
    import torch
    n, na, nb = 6, 3, 3
    h, eri, _ = synth_hamiltonian(n, seed=23)
    sp = tb.Space(ctx, n, na, nb, h, eri)
    # empty pruned space: nothing to compute, no error
    pr = sp.prune(np.zeros(sp.la + 1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    assert pr.ndet == 0
    z = torch.zeros(1, 0, dtype=torch.float64, device="cuda")
    tb.tbsci_sigma_pruned(ctx.handle, sp.ham, sp.ta, sp.tb, pr.handle, z, torch.zeros_like(z), 1)
    pr.close()
    # one determinant: sigma = H_00 c
    off = np.zeros(sp.la + 1, dtype=np.int64)
    off[4:] = 1
    pr = sp.prune(off, np.array([7], dtype=np.int32))
    osp = oracle.make_space(n, na, nb)
    s = pr.sigma(torch.tensor([[2.0]], dtype=torch.float64, device="cuda")).cpu().numpy()
    assert abs(s[0, 0] - 2.0 * oracle.diagonal(osp, h, eri, 0.0)[3 * sp.lb + 7]) < 1e-12
    pr.close()
    bad = [
        (np.r_[np.zeros(sp.la, dtype=np.int64), [2]], np.array([3, 3], dtype=np.int32)),      # repeated index
        (np.r_[np.zeros(sp.la, dtype=np.int64), [1]], np.array([sp.lb], dtype=np.int32)),     # out of range
        (np.r_[[0, 2], np.ones(sp.la - 1, dtype=np.int64)], np.array([1, 2], dtype=np.int32)),  # decreasing off
    ]
    for off, cols in bad:
        with pytest.raises(tb.B.TbsciError) as err:
            sp.prune(off, cols)
        assert err.value.status == tb.TBSCI_EINVAL
    sp.close()
