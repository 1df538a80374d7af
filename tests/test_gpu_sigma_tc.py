"""Tensor-core sigma modes (tcgen05, row a6): the alpha-beta classes, alpha
singles and diagonal from split-TF32 (3 products per term) or BF16 products
with FP32 accumulation, the other classes on the FP32 SIMT path or as dense
products on the tensor cores (rest mode 5). Compared with
the oracle applied to the FP32-rounded vector: split TF32 within FP32-level
accumulation error, BF16 within its 8-bit-mantissa error."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import assert_sigma_close
from tbsci_inputs import WORKLOADS, random_vectors, selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"tf32": (2e-5, 1e-5), "bf16": (2e-2, 1e-2)}


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


@pytest.fixture(scope="module")
def ctx(tb):
    c = tb.Context(0)
    yield c
    c.close()


CASES = [
    (8, 4, 4, None, None, 1),
    (10, 5, 5, 120, 257, 2),   # ragged: 257 beta columns, a partial last 64-column tile
    (12, 6, 6, 300, 300, 1),
    (12, 4, 6, None, 200, 1),
    (16, 8, 8, 700, 650, 1),   # the largest norb of the tensor-core tile (120 pairs)
    (18, 9, 9, 300, 300, 1),   # 153 pairs: falls back to the FP32 SIMT path
]


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("n,na,nb,acnt,bcnt,nvec", CASES)
def test_tc_sigma_parity(tb, ctx, mode, n, na, nb, acnt, bcnt, nvec):
    import torch
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel = None if acnt is None else selected_strings(n, na, acnt, 31 + n)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, 37 + n)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    C = random_vectors(nvec, sp.la, sp.lb, seed=n).astype(np.float32)
    dt = tb.TBSCI_F32_TC_TF32 if mode == "tf32" else tb.TBSCI_F32_TC_BF16
    s = sp.sigma(torch.from_numpy(C).cuda(), dtype=dt).double().cpu().numpy().reshape(nvec, -1)
    ref, bound = oracle.sigma(osp, h, eri, 0.2, C.astype(np.float64), with_bound=True)
    rel, norm_rel = TOL[mode] if n <= 16 else (64 * 2.0 ** -24, 1e-5)
    assert_sigma_close(s, ref, bound, rel=rel, norm_rel=norm_rel)
    sp.close()


def test_tc_sigma_sel16_sampled(tb, ctx):
    """norb=16, 3,000 x 3,000 (9.0M determinants), split TF32, 3 vectors."""
    import torch
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, bsel)
    C = random_vectors(3, sp.la, sp.lb, seed=wl.seed_vec).astype(np.float32)
    s = sp.sigma(torch.from_numpy(C).cuda(), dtype=tb.TBSCI_F32_TC_TF32).double().cpu().numpy().reshape(3, -1)
    rows = np.random.default_rng(5).choice(sp.ndet, 2000, replace=False)
    ref, bound = oracle.sigma(osp, h, eri, ecore, C.astype(np.float64).reshape(3, -1), rows=rows, with_bound=True)
    assert_sigma_close(s[:, rows], ref, bound, rel=2e-5, norm_rel=1e-5)
    sp.close()


@pytest.mark.parametrize("mixed", [2, 3])
def test_tc_mixed_davidson_golden(tb, ctx, mixed):
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    ref = np.loadtxt(os.path.join(GOLDEN, "fci8_energies.txt"))
    e, info = sp.davidson(3, mixed=mixed)
    assert info["converged"] and info["nsigma_f32"] > 0
    assert np.max(np.abs(e - ref[:3])) < 1e-8
    sp.close()


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("n,na,nb,acnt,bcnt", [(10, 5, 5, 120, 257), (16, 8, 8, 700, 650)])
def test_tc_sigma_parity_after_autotune(tb, ctx, mode, n, na, nb, acnt, bcnt):
    """Tuning a tensor-core sigma type picks the shared-memory mode and CTA size of
    the SIMT pass for the other classes; sigma still matches the oracle."""
    import torch
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel = selected_strings(n, na, acnt, 31 + n)
    bsel = selected_strings(n, nb, bcnt, 37 + n)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    C = random_vectors(1, sp.la, sp.lb, seed=n).astype(np.float32)
    dt = tb.TBSCI_F32_TC_TF32 if mode == "tf32" else tb.TBSCI_F32_TC_BF16
    Ct = torch.from_numpy(C).cuda()
    out = torch.empty_like(Ct)
    ms = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, Ct, out, 1, dt)
    assert ms > 0
    cnt = sp.counts()
    assert cnt["tuned_rest"][0] in (0, 1, 2, 3, 4, 5) and cnt["tuned_rest"][1] in (128, 256, 512)
    ref, bound = oracle.sigma(osp, h, eri, 0.2, C.astype(np.float64), with_bound=True)
    rel, norm_rel = TOL[mode]
    for s in (out, sp.sigma(Ct, dtype=dt)):
        assert_sigma_close(s.double().cpu().numpy().reshape(1, -1), ref, bound, rel=rel, norm_rel=norm_rel)
    sp.close()


@pytest.mark.parametrize("rest_mode,threads", [(3, 512), (3, 128), (1, 256), (2, 512), (4, 256)])
@pytest.mark.parametrize("n,na,nb,acnt,bcnt", [(10, 5, 5, 120, 257), (12, 4, 6, None, 200), (16, 8, 8, 700, 650)])
def test_tc_sigma_rest_modes_from_tune_cache(tb, n, na, nb, acnt, bcnt, rest_mode, threads, tmp_path):
    """Every mode of the pass for the classes the tensor cores leave out, pinned
    through a tune cache file loaded into a fresh context: mode 3 serves two alpha
    rows per CTA when l_alpha is even (120, 700) and falls back to mode 1 when it
    is odd (495); mode 4 runs them as column-tiled products; sigma matches the
    oracle in each."""
    import torch
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel = None if acnt is None else selected_strings(n, na, acnt, 31 + n)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, 37 + n)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d 0 0 0 0 0 0 %d %d\n" % (n, osp.la, osp.lb, rest_mode, threads))
    ctx = tb.Context(0)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    assert sp.counts()["tuned_rest"] == [rest_mode, threads]
    C = random_vectors(2, sp.la, sp.lb, seed=n + 1).astype(np.float32)
    s = sp.sigma(torch.from_numpy(C).cuda(), dtype=tb.TBSCI_F32_TC_TF32).double().cpu().numpy().reshape(2, -1)
    ref, bound = oracle.sigma(osp, h, eri, 0.2, C.astype(np.float64), with_bound=True)
    rel, norm_rel = TOL["tf32"]
    assert_sigma_close(s, ref, bound, rel=rel, norm_rel=norm_rel)
    sp.close()
    ctx.close()


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("n,na,nb,acnt,bcnt", [(10, 5, 5, 120, 257), (12, 4, 6, None, 200), (16, 8, 8, 700, 650)])
def test_tc_sigma_dense_same_spin(tb, n, na, nb, acnt, bcnt, mode, tmp_path):
    """Rest mode 5: the same-spin classes as dense products on the tensor cores
    (split TF32 for the TF32 type, one BF16 product for the BF16 type), pinned
    through a tune cache; two vectors against the oracle at the type's
    tolerance, twice."""
    import torch
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel = None if acnt is None else selected_strings(n, na, acnt, 31 + n)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, 37 + n)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d 0 0 0 0 0 0 5 256\n" % (n, osp.la, osp.lb))
    ctx = tb.Context(0)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    assert sp.counts()["tuned_rest"] == [5, 256]
    dt = tb.TBSCI_F32_TC_TF32 if mode == "tf32" else tb.TBSCI_F32_TC_BF16
    C = random_vectors(2, sp.la, sp.lb, seed=n + 3).astype(np.float32)
    Ct = torch.from_numpy(C).cuda()
    s = sp.sigma(Ct, dtype=dt).double().cpu().numpy().reshape(2, -1)
    ref, bound = oracle.sigma(osp, h, eri, 0.2, C.astype(np.float64), with_bound=True)
    rel, norm_rel = TOL[mode]
    assert_sigma_close(s, ref, bound, rel=rel, norm_rel=norm_rel)
    # the tensor-core kernel's scatter sums with shared-memory atomics, so a second
    # evaluation agrees to rounding, not bit for bit
    assert_sigma_close(sp.sigma(Ct, dtype=dt).double().cpu().numpy().reshape(2, -1), ref, bound, rel=rel,
                       norm_rel=norm_rel)
    sp.close()
    ctx.close()


def test_tc_dense_mode_respects_the_budget(tb, tmp_path):
    """Under a device-memory budget that holds the space and the column-tiled
    products but not the dense same-spin matrices, tuning a tensor-core type
    skips rest mode 5 (its set-up is refused with ENOMEM and leaves nothing
    counted) and sigma still matches the oracle."""
    import torch
    n, na, nb, acnt, bcnt = 16, 8, 8, 700, 650
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel, bsel = selected_strings(n, na, acnt, 31 + n), selected_strings(n, nb, bcnt, 37 + n)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    C = random_vectors(1, osp.la, osp.lb, seed=5).astype(np.float32)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d 0 0 0 0 0 0 4 256\n" % (n, osp.la, osp.lb))
    # bytes the space needs with the column-tiled products (measured without a budget)
    free = tb.Context(0)
    tb.tbsci_tune_cache_load(free.handle, str(path))
    sp = tb.Space(free, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    sp.sigma(torch.from_numpy(C).cuda(), dtype=tb.TBSCI_F32_TC_TF32)
    need = tb.tbsci_hbm_used(free.handle)
    sp.close()
    free.close()
    dense = 8 * ((osp.la + 31) // 32 * 32) ** 2  # the alpha matrix alone, split-TF32 planes
    ctx = tb.Context(0, hbm_budget=need + dense // 2)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.2, alpha=asel, beta=bsel)
    Ct = torch.from_numpy(C).cuda()
    out = torch.empty_like(Ct)
    sp.sigma(Ct, out, dtype=tb.TBSCI_F32_TC_TF32)
    before = tb.tbsci_hbm_used(ctx.handle)
    assert tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, Ct, out, 1, tb.TBSCI_F32_TC_TF32) > 0
    assert sp.counts()["tuned_rest"][0] != 5
    assert tb.tbsci_hbm_used(ctx.handle) == before
    ref, bound = oracle.sigma(osp, h, eri, 0.2, C.astype(np.float64), with_bound=True)
    rel, norm_rel = TOL["tf32"]
    s = sp.sigma(Ct, dtype=tb.TBSCI_F32_TC_TF32).double().cpu().numpy().reshape(1, -1)
    assert_sigma_close(s, ref, bound, rel=rel, norm_rel=norm_rel)
    sp.close()
    ctx.close()


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tc_sigma_fci16_sampled_tuned(tb, ctx, mode):
    """norb=16 full string space (12,870^2 = 165.6M determinants), 1 vector, in the
    launch configuration the bench times for the tensor-core types: autotuned
    first (SIMT pass shape), then 600 seeded rows recomputed by the oracle from
    the FP32-rounded vector, at the tensor-core tolerances."""
    import torch
    wl = WORKLOADS["fci16"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta)
    assert sp.ndet == 12870 * 12870
    dt = tb.TBSCI_F32_TC_TF32 if mode == "tf32" else tb.TBSCI_F32_TC_BF16
    g = torch.Generator(device="cuda").manual_seed(wl.seed_vec)
    C = torch.randn((1, sp.la, sp.lb), generator=g, device="cuda", dtype=torch.float32)
    S = torch.empty_like(C)
    ms = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, S, 1, dt)
    assert ms > 0
    S = sp.sigma(C, S, dtype=dt)
    rows = np.sort(np.random.default_rng(wl.seed_vec + 1).choice(sp.ndet, 600, replace=False))
    got = S.reshape(-1)[torch.from_numpy(rows).cuda()].double().cpu().numpy()[None]
    Ch = C.reshape(1, -1).double().cpu().numpy()
    del S, C
    ref, bound = oracle.sigma(osp, h, eri, ecore, Ch, rows=rows, with_bound=True)
    rel, norm_rel = TOL[mode]
    assert_sigma_close(got, ref, bound, rel=rel, norm_rel=norm_rel)
    sp.close()
    torch.cuda.empty_cache()
