"""The split sigma path for rows longer than shared memory (row a4-a6 at the
norb-24 workload): the row kernel with c rows staged in column parts (stage 3:
one CTA per alpha row accumulating in the output row; 4, 5: two or four CTAs
per alpha row, each keeping the sigma accumulators of its share of the columns
in shared memory; 6: as 3 with parts short enough for two CTAs per SM), plus the
alpha-double and beta-double classes as column-tiled sparse x dense products
(the latter on the transposed vector). Each launch shape is pinned through a
tune-cache file and compared with the oracle element by element, on spaces that
span several column parts, tiles of the double-class product and ragged edges."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_sigma_close
from tbsci_inputs import selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


def _space(tb, ctx, n, na, nb, acnt, bcnt, seed, ecore=0.0):
    h, eri, _ = synth_hamiltonian(n, seed=seed)
    asel = None if acnt is None else selected_strings(n, na, acnt, seed + 1)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, seed + 2)
    sp = tb.Space(ctx, n, na, nb, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    return sp, osp, h, eri


def _ctx_with_shape(tb, tmp_path, n, la, lb, dtype, threads, stage):
    """A context whose tune cache pins the SIMT launch shape of this space."""
    f64 = (threads, 1, stage) if dtype == "f64" else (0, 0, 0)
    f32 = (threads, 1, stage) if dtype == "f32" else (0, 0, 0)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d %d %d %d %d %d %d 0 0\n" % ((n, la, lb) + f64 + f32))
    ctx = tb.Context(0)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    return ctx


CASES = [
    # n, na, nb, alpha count, beta count, nvec
    (8, 4, 4, None, None, 2),
    (10, 5, 5, 120, 257, 3),    # all 252 beta strings: ragged slices, transpose tiles and column tiles
    (12, 6, 6, 300, 280, 1),
    (12, 4, 6, None, 200, 2),   # distinct alpha and beta sets of different sizes
    (9, 1, 0, None, None, 1),   # no beta electron
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("threads,stage", [(512, 3), (1024, 3), (1024, 4), (512, 5), (512, 6)])
@pytest.mark.parametrize("n,na,nb,acnt,bcnt,nvec", CASES)
def test_split_sigma_parity(tb, tmp_path, n, na, nb, acnt, bcnt, nvec, threads, stage, dtype):
    import torch
    probe = oracle.make_space(n, na, nb, None if acnt is None else selected_strings(n, na, acnt, 601 + n),
                              None if bcnt is None else selected_strings(n, nb, bcnt, 602 + n))
    ctx = _ctx_with_shape(tb, tmp_path, n, probe.la, probe.lb, dtype, threads, stage)
    sp, osp, h, eri = _space(tb, ctx, n, na, nb, acnt, bcnt, seed=600 + n, ecore=0.15)
    cnt = sp.counts()
    ti = 0 if dtype == "f64" else 1
    assert cnt["tuned_stage"][ti] == stage and cnt["tuned_threads"][ti] == threads
    C = np.random.default_rng(n).standard_normal((nvec, sp.la, sp.lb))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ct = torch.from_numpy(C).to(tdt).cuda()
    s = sp.sigma(Ct).double().cpu().numpy().reshape(nvec, -1)
    ref, bound = oracle.sigma(osp, h, eri, 0.15, Ct.double().cpu().numpy(), with_bound=True)
    if dtype == "f64":
        assert_sigma_close(s, ref, bound)
    else:
        assert_sigma_close(s, ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    # deterministic: a second evaluation is bit-identical
    assert np.array_equal(sp.sigma(Ct).double().cpu().numpy().reshape(nvec, -1), s)
    sp.close()
    ctx.close()


@pytest.mark.parametrize("n,dtype,stage", [(18, "f64", 3), (18, "f64", 5), (19, "f64", 4), (19, "f32", 3)])
def test_split_sigma_long_rows(tb, tmp_path, n, dtype, stage):
    """Full beta string spaces of norb 18 / 19 (48,620 / 92,378 strings; 389 KB /
    739 KB per FP64 row, so many column parts) with 6 selected alpha strings:
    500 sampled rows against the oracle."""
    import torch
    na = nb = 9
    asel = selected_strings(n, na, 6, 701 + n)
    ctx = _ctx_with_shape(tb, tmp_path, n, 6, math.comb(n, nb), dtype, 512, stage)
    h, eri, _ = synth_hamiltonian(n, seed=700 + n)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.5, alpha=asel)
    osp = oracle.make_space(n, na, nb, asel, None)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ct = torch.from_numpy(np.random.default_rng(n).standard_normal((1, sp.la, sp.lb))).to(tdt).cuda()
    s = sp.sigma(Ct).double().cpu().numpy().reshape(1, -1)
    rows = np.sort(np.random.default_rng(n + 1).choice(sp.ndet, 500, replace=False))
    ref, bound = oracle.sigma(osp, h, eri, 0.5, Ct.double().cpu().numpy().reshape(1, -1), rows=rows,
                              with_bound=True)
    if dtype == "f64":
        assert_sigma_close(s[:, rows], ref, bound)
    else:
        assert_sigma_close(s[:, rows], ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    sp.close()
    ctx.close()


def test_split_davidson_matches_dense(tb, tmp_path):
    """Davidson on the split path (FP64 and mixed) reaches the dense eigenvalues."""
    n, na, nb = 8, 4, 3
    asel = selected_strings(n, na, 50, 42)
    probe = oracle.make_space(n, na, nb, asel, None)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d 512 1 4 1024 1 3 0 0\n" % (n, probe.la, probe.lb))
    ctx = tb.Context(0)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    h, eri, _ = synth_hamiltonian(n, seed=41)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(probe, h, eri, 0.1))
    for mixed in (0, 1):
        e, info = sp.davidson(4, mixed=mixed, max_subspace=16)
        assert info["converged"] and np.max(np.abs(e - w[:4])) < 1e-8
    sp.close()
    ctx.close()
