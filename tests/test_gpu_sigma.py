"""GPU sigma = H.c vs the oracle (rows a3-a6), through the C ABI.

Full element-by-element comparison on spaces the oracle finishes in seconds
(several CTAs, ragged column counts, nvec that splits across launches), and at
the full norb=16, 3,000 x 3,000 size on sampled rows in the launch
configuration the bench times (FP64, 3 vectors)."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_sigma_close
from tbsci_inputs import WORKLOADS, random_vectors, selected_strings, synth_hamiltonian

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


def _case(tb, ctx, n, na, nb, acnt, bcnt, seed, ecore=0.0):
    h, eri, _ = synth_hamiltonian(n, seed=seed)
    asel = None if acnt is None else selected_strings(n, na, acnt, seed + 1)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, seed + 2)
    sp = tb.Space(ctx, n, na, nb, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    assert (sp.la, sp.lb) == (osp.la, osp.lb)
    return sp, osp, h, eri


CASES = [
    # n, na, nb, alpha count, beta count, nvec
    (6, 3, 3, None, None, 1),
    (8, 4, 4, None, None, 3),
    (8, 4, 3, 40, None, 2),
    (10, 5, 5, 120, 257, 5),     # 257 columns: a ragged tail past one 256-thread sweep
    (10, 3, 5, None, 90, 4),
    (12, 6, 6, 300, 300, 1),
    (9, 1, 0, None, None, 2),    # one alpha electron, no beta: H = h
    (7, 7, 2, None, None, 1),    # fully occupied alpha string
    (14, 7, 7, 700, 650, 3),
]


@pytest.mark.parametrize("n,na,nb,acnt,bcnt,nvec", CASES)
def test_sigma_f64_full_parity(tb, ctx, n, na, nb, acnt, bcnt, nvec):
    import torch
    sp, osp, h, eri = _case(tb, ctx, n, na, nb, acnt, bcnt, seed=100 + n, ecore=0.25)
    C = random_vectors(nvec, sp.la, sp.lb, seed=n)
    s = sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    ref, bound = oracle.sigma(osp, h, eri, 0.25, C, with_bound=True)
    assert_sigma_close(s.reshape(nvec, -1), ref, bound)
    sp.close()


def test_sigma_f32_parity(tb, ctx):
    import torch
    sp, osp, h, eri = _case(tb, ctx, 12, 6, 6, 300, 280, seed=7)
    C = random_vectors(2, sp.la, sp.lb, seed=8)
    s = sp.sigma(torch.from_numpy(C).float().cuda()).double().cpu().numpy().reshape(2, -1)
    # FP32 inputs: compare against the oracle applied to the same rounded vector
    C32 = C.astype(np.float32).astype(np.float64)
    ref, bound = oracle.sigma(osp, h, eri, 0.0, C32, with_bound=True)
    # FP32 products and sums: |d| <= 64 * 2^-24 * (|H||c|) per element
    assert_sigma_close(s, ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    sp.close()


def test_diagonal_parity(tb, ctx):
    sp, osp, h, eri = _case(tb, ctx, 10, 5, 4, 100, None, seed=9)
    d = sp.diagonal().cpu().numpy()
    ref = oracle.diagonal(osp, h, eri, 0.0)
    assert np.max(np.abs(d - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    sp.close()


def test_sigma_host_equals_device_and_deterministic(tb, ctx):
    import torch
    sp, osp, h, eri = _case(tb, ctx, 10, 5, 5, 150, 150, seed=10)
    C = random_vectors(2, sp.la, sp.lb, seed=11)
    s1 = sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    s2 = sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    s3 = sp.sigma_host(C)
    assert np.array_equal(s1, s2) and np.array_equal(s1, s3)
    sp.close()


def test_sigma_host_pipelined_groups(tb, ctx):
    """After tuning (at most 4 vectors per launch group), 5 host vectors pass
    through in several groups with overlapped copies, the last one ragged: the
    result equals the device evaluation bit for bit, pinned or pageable."""
    import torch
    sp, osp, h, eri = _case(tb, ctx, 12, 6, 6, 300, 280, seed=12)
    C = random_vectors(5, sp.la, sp.lb, seed=13)
    Cd = torch.from_numpy(C).cuda()
    out = torch.empty_like(Cd)
    tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, Cd[:4], out[:4], 4, tb.TBSCI_F64)
    assert 1 <= sp.counts()["tuned_nv"][0] <= 4
    want = sp.sigma(Cd).cpu().numpy()
    assert np.array_equal(sp.sigma_host(C), want)
    pinned = torch.from_numpy(C).pin_memory()
    pinned_out = torch.empty_like(pinned).pin_memory()
    tb.tbsci_sigma_host(ctx.handle, sp.ham, sp.ta, sp.tb, pinned.numpy(), pinned_out.numpy(), 5)
    assert np.array_equal(pinned_out.numpy(), want)
    sp.close()


def test_fci8_sigma(tb, ctx):
    import torch
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta)
    C = random_vectors(1, sp.la, sp.lb, seed=wl.seed_vec)
    s = sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    ref, bound = oracle.sigma(osp, h, eri, ecore, C, with_bound=True)
    assert_sigma_close(s.reshape(1, -1), ref, bound)
    sp.close()


def test_sel16_sigma_sampled_rows_full_size(tb, ctx):
    """norb=16, 3,000 x 3,000 selected strings (9.0M determinants), FP64, 3
    vectors in one call, autotuned first: the launch configuration the bench
    times for this workload. 4,000 seeded rows (whole rows of the first and last
    alpha strings included) are recomputed by the oracle."""
    import torch
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, bsel)
    assert sp.ndet == 9_000_000
    C = random_vectors(3, sp.la, sp.lb, seed=wl.seed_vec)
    Cd = torch.from_numpy(C).cuda()
    tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, Cd, torch.empty_like(Cd), 3, tb.TBSCI_F64)
    s = sp.sigma(Cd).cpu().numpy().reshape(3, -1)
    rng = np.random.default_rng(wl.seed_vec)
    rows = np.unique(np.concatenate([rng.choice(sp.ndet, 3000, replace=False), np.arange(500),
                                     np.arange(sp.ndet - 500, sp.ndet)]))
    ref, bound = oracle.sigma(osp, h, eri, ecore, C.reshape(3, -1), rows=rows, with_bound=True)
    assert_sigma_close(s[:, rows], ref, bound)
    sp.close()


def test_sigma_edge_cases(tb, ctx):
    import torch
    h, eri, _ = synth_hamiltonian(6, seed=12)
    # empty selection: nothing to do, no error
    sp = tb.Space(ctx, 6, 3, 3, h, eri, alpha=np.zeros(0, dtype=np.uint64))
    assert sp.ndet == 0
    c = torch.zeros((1, 0, sp.lb), dtype=torch.float64, device="cuda")
    tb.tbsci_sigma(ctx.handle, sp.ham, sp.ta, sp.tb, c, torch.zeros_like(c), 1)
    sp.close()
    # a single determinant: sigma = H_00 c
    sp, osp, h, eri = _case(tb, ctx, 6, 3, 3, 1, 1, seed=13)
    C = np.array([[[1.5]]])
    s = sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
    assert abs(s[0, 0, 0] - 1.5 * oracle.diagonal(osp, h, eri, 0.0)[0]) < 1e-12
    sp.close()


def test_invalid_arguments(tb, ctx):
    import torch
    h, eri, _ = synth_hamiltonian(5, seed=14)
    bad = h.copy()
    bad[0, 1] += 1e-6
    with pytest.raises(tb.B.TbsciError):
        tb.tbsci_hamiltonian_create(ctx.handle, bad, eri)
    e2 = eri.copy()
    e2[0, 1, 2, 3] += 1e-6
    with pytest.raises(tb.B.TbsciError):
        tb.tbsci_hamiltonian_create(ctx.handle, h, e2)
    sp = tb.Space(ctx, 5, 2, 2, h, eri)
    c = torch.zeros((1, sp.la, sp.lb), dtype=torch.float64, device="cuda")
    with pytest.raises(tb.B.TbsciError):
        tb.tbsci_sigma(ctx.handle, sp.ham, sp.ta, sp.tb, c, c, 1)  # aliasing
    with pytest.raises(tb.B.TbsciError):
        tb.tbsci_sigma(ctx.handle, sp.ham, sp.ta, sp.tb, c, torch.zeros_like(c), 0)
    # tables without doubles cannot drive sigma
    s = tb.tbsci_build_strings(ctx.handle, 5, 2, None)
    t = tb.tbsci_build_excitation_tables(ctx.handle, s, tb.TBSCI_TABLES_SINGLES_ONLY)
    with pytest.raises(tb.B.TbsciError):
        tb.tbsci_prepare(ctx.handle, sp.ham, t, t)
    tb.tbsci_tables_destroy(t)
    tb.tbsci_strings_destroy(s)
    sp.close()


@pytest.mark.parametrize("n,dtype", [(18, "f64"), (18, "f32"), (19, "f64"), (19, "f32")])
def test_sigma_rows_longer_than_shared_memory(tb, ctx, n, dtype):
    """Full beta string spaces of norb 18 and 19 with 9 beta electrons (48,620 and
    92,378 strings: 389 KB and 739 KB per FP64 row) and 4 selected alpha strings:
    c rows and sigma accumulators that do not fit in shared memory are read and
    accumulated in global memory. 500 sampled rows against the oracle."""
    import torch
    na = nb = 9
    h, eri, _ = synth_hamiltonian(n, seed=300 + n)
    asel = selected_strings(n, na, 4, 301 + n)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.5, alpha=asel)
    osp = oracle.make_space(n, na, nb, asel, None)
    assert sp.lb == math.comb(n, nb)
    C = random_vectors(2, sp.la, sp.lb, seed=n)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ct = torch.from_numpy(C).to(tdt).cuda()
    s = sp.sigma(Ct).double().cpu().numpy().reshape(2, -1)
    rows = np.sort(np.random.default_rng(n).choice(sp.ndet, 500, replace=False))
    Cref = Ct.double().cpu().numpy().reshape(2, -1)  # the oracle sees the vector the kernel saw
    ref, bound = oracle.sigma(osp, h, eri, 0.5, Cref, rows=rows, with_bound=True)
    if dtype == "f64":
        assert_sigma_close(s[:, rows], ref, bound)
    else:
        assert_sigma_close(s[:, rows], ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    sp.close()


@pytest.mark.parametrize("name,dtype,tune", [("fci16", "f64", False), ("fci16", "f32", False),
                                             ("sel24", "f32", False), ("sel24", "f64", True)])
def test_large_configs_sigma_sampled_rows(tb, ctx, name, dtype, tune):
    """norb=16 full string space (12,870^2 = 165.6M determinants) and norb=24,
    40,000 x 40,000 selected strings (1.6B determinants), one vector: 600 seeded
    rows recomputed by the oracle. FP32 runs compare against the oracle applied
    to the FP32-rounded vector, within FP32 accumulation error. The FP64 run at
    norb 24 is the bench's headline launch: autotuned first, then timed shape."""
    import torch
    wl = WORKLOADS[name]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, bsel)
    rng = np.random.default_rng(wl.seed_vec)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    # the vector is generated on the device (1.6B determinants); the sampled rows'
    # neighbourhoods are read back from it for the oracle
    g = torch.Generator(device="cuda").manual_seed(wl.seed_vec)
    C = torch.randn((1, sp.la, sp.lb), generator=g, device="cuda", dtype=torch.float32).to(tdt)
    if tune:
        S = torch.empty_like(C)
        sdt = tb.TBSCI_F64 if dtype == "f64" else tb.TBSCI_F32
        assert tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, S, 1, sdt) > 0
        assert sp.counts()["tuned_nv"][0 if dtype == "f64" else 1] >= 1
        S = sp.sigma(C, S)
    else:
        S = sp.sigma(C)
    rows = np.sort(rng.choice(sp.ndet, 600, replace=False))
    got = S.reshape(-1)[torch.from_numpy(rows).cuda()].double().cpu().numpy()[None]
    del S
    Ch = C.reshape(-1).double().cpu().numpy() if sp.ndet <= 200_000_000 else None
    if Ch is None:
        # only the coupled entries are needed: gather them through the oracle's row structure
        cols = [oracle.row(osp, h, eri, ecore, int(K))[0] for K in rows]
        allc = np.unique(np.concatenate(cols))
        vals = C.reshape(-1)[torch.from_numpy(allc).cuda()].double().cpu().numpy()
        Ch = np.zeros(1)  # placeholder for clarity; sigma is formed from the gathered entries below
        ref = np.zeros((1, len(rows)))
        bound = np.zeros((1, len(rows)))
        lookup = dict(zip(allc.tolist(), vals.tolist()))
        for i, K in enumerate(rows):
            c, v = oracle.row(osp, h, eri, ecore, int(K))
            cv = np.array([lookup[x] for x in c.tolist()])
            ref[0, i] = float(np.dot(v, cv))
            bound[0, i] = float(np.dot(np.abs(v), np.abs(cv)))
    else:
        ref, bound = oracle.sigma(osp, h, eri, ecore, Ch[None], rows=rows, with_bound=True)
    if dtype == "f64":
        assert_sigma_close(got, ref, bound)
    else:
        assert_sigma_close(got, ref, bound, rel=64 * 2.0 ** -24, norm_rel=1e-5)
    del C
    sp.close()
    torch.cuda.empty_cache()


def test_autotune_keeps_results_bitwise(tb, ctx):
    """The autotuner picks a launch shape by timing; every shape sums each column
    in the same order, so sigma is bit-identical before and after tuning."""
    import torch
    sp, osp, h, eri = _case(tb, ctx, 12, 6, 6, 400, 380, seed=17)
    for dt, tdt in ((tb.TBSCI_F64, torch.float64), (tb.TBSCI_F32, torch.float32)):
        C = torch.from_numpy(random_vectors(3, sp.la, sp.lb, seed=18)).to(tdt).cuda()
        before = sp.sigma(C).cpu().numpy()
        out = torch.empty_like(C)
        ms = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, out, 3, dt)
        assert ms > 0
        assert np.array_equal(out.cpu().numpy(), before)
        assert np.array_equal(sp.sigma(C).cpu().numpy(), before)
    sp.close()


def test_autotune_on_row_sample_keeps_results_bitwise(tb, ctx):
    """norb 16 full space in FP32 (one sigma takes well over 100 ms): the tuner
    times shapes on a sample of alpha rows, including the shared-memory use, and
    sigma stays bit-identical before tuning, after it, and with the chosen shape."""
    import torch
    wl = WORKLOADS["fci16"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    g = torch.Generator(device="cuda").manual_seed(7)
    C = torch.randn((1, sp.la, sp.lb), generator=g, device="cuda", dtype=torch.float32)
    before = sp.sigma(C)
    out = torch.empty_like(C)
    ms = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, out, 1, tb.TBSCI_F32)
    assert ms > 0
    assert torch.equal(out, before)
    assert torch.equal(sp.sigma(C), before)
    cnt = sp.counts()
    assert cnt["tuned_threads"][1] in (128, 256, 512) and cnt["tuned_nv"][1] == 1
    assert cnt["tuned_stage"][1] in (0, 1, 2)
    del C, out, before
    sp.close()
    torch.cuda.empty_cache()


def test_tune_cache_roundtrip(tb, ctx, tmp_path):
    """A tuned shape is recorded under (norb, l_alpha, l_beta), saved as text, and
    a same-shaped space with another Hamiltonian on a fresh context that loads
    the file starts with that shape; sigma there still matches the oracle.
    Malformed files are rejected whole."""
    import torch
    n, na, nb = 12, 6, 6
    asel, bsel = selected_strings(n, na, 300, 1201), selected_strings(n, nb, 280, 1202)
    h, eri, _ = synth_hamiltonian(n, seed=1203)
    sp = tb.Space(ctx, n, na, nb, h, eri, alpha=asel, beta=bsel)
    C = torch.from_numpy(random_vectors(3, sp.la, sp.lb, seed=1204)).cuda()
    tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, torch.empty_like(C), 3, tb.TBSCI_F64)
    tuned = sp.counts()
    assert tuned["tuned_nv"][0] >= 1 and tb.tbsci_tune_cache_size(ctx.handle) >= 1
    path = tmp_path / "tune.txt"
    tb.tbsci_tune_cache_save(ctx.handle, str(path))
    lines = path.read_text().splitlines()
    assert lines[0] == "tbsci-tune 1"
    row = [x for x in lines[1:] if x.split()[:3] == [str(n), str(sp.la), str(sp.lb)]]
    assert len(row) == 1
    assert [int(v) for v in row[0].split()[3:6]] == [tuned["tuned_threads"][0], tuned["tuned_nv"][0],
                                                     tuned["tuned_stage"][0]]
    ctx2 = tb.Context(0)
    for bad in ("", "tbsci-tune 1\n12 300 280 512 9 0 0 0 0 0 0\n", "other 1\n", "tbsci-tune 1\n12 300\n"):
        p = tmp_path / "bad.txt"
        p.write_text(bad)
        with pytest.raises(tb.B.TbsciError) as err:
            tb.tbsci_tune_cache_load(ctx2.handle, str(p))
        assert err.value.status == tb.TBSCI_EINVAL
    assert tb.tbsci_tune_cache_size(ctx2.handle) == 0
    tb.tbsci_tune_cache_load(ctx2.handle, str(path))
    h2, eri2, _ = synth_hamiltonian(n, seed=1205)
    sp2 = tb.Space(ctx2, n, na, nb, h2, eri2, 0.3, alpha=asel, beta=bsel)
    got = sp2.counts()
    for key in ("tuned_threads", "tuned_nv", "tuned_stage"):
        assert got[key][0] == tuned[key][0], key
    osp = oracle.make_space(n, na, nb, asel, bsel)
    C2 = random_vectors(3, sp2.la, sp2.lb, seed=1206)
    s2 = sp2.sigma(torch.from_numpy(C2).cuda()).cpu().numpy().reshape(3, -1)
    ref, bound = oracle.sigma(osp, h2, eri2, 0.3, C2, with_bound=True)
    assert_sigma_close(s2, ref, bound)
    sp2.close()
    ctx2.close()
    sp.close()


def test_sigma_host_recovers_from_a_failed_allocation(tb, ctx):
    """tbsci_sigma_host with more vectors than the device can hold: its device
    buffers cannot be allocated, the call returns ENOMEM without touching the host
    arrays, and the next call of a normal size allocates again and gives the
    device result."""
    import torch
    sp, osp, h, eri = _case(tb, ctx, 10, 5, 5, 120, 130, seed=19)
    C = random_vectors(1, sp.la, sp.lb, seed=20)
    out = np.empty_like(C)
    lib = tb.B.load()
    huge = (1 << 31) - 1  # ~ 2^31 vectors of 15,600 determinants: 267 TB
    st = lib.tbsci_sigma_host(ctx.handle, sp.ham, sp.ta, sp.tb, tb.B._ptr(C), tb.B._ptr(out), huge)
    assert st == tb.TBSCI_ENOMEM, st
    assert np.array_equal(sp.sigma_host(C), sp.sigma(torch.from_numpy(C).cuda()).cpu().numpy())
    sp.close()
