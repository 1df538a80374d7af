"""GPU Davidson (row a7) vs dense diagonalisation and the stored oracle energies."""
import os

import numpy as np
import pytest

import oracle
from tbsci_inputs import WORKLOADS, random_vectors, selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


@pytest.fixture(scope="module")
def ctx(tb):
    c = tb.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_fci8_golden(tb, ctx, mixed):
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    ref = np.loadtxt(os.path.join(GOLDEN, "fci8_energies.txt"))
    e, info = sp.davidson(3, mixed=mixed)
    assert info["converged"]
    assert np.max(np.abs(e - ref[:3])) < 1e-8, (e, ref[:3])
    if mixed:
        assert info["nsigma_f32"] > 0 and info["nsigma"] > info["nsigma_f32"]
    sp.close()


def test_small_selected_vs_dense(tb, ctx):
    n, na, nb = 8, 4, 3
    h, eri, _ = synth_hamiltonian(n, seed=41)
    asel = selected_strings(n, na, 50, 42)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel)
    osp = oracle.make_space(n, na, nb, asel, None)
    H = oracle.hamiltonian_dense(osp, h, eri, 0.1)
    w, U = np.linalg.eigh(H)
    e, info, X = sp.davidson(4, want_vectors=True, max_subspace=16)
    assert info["converged"]
    assert np.max(np.abs(e - w[:4])) < 1e-8
    X = X.cpu().numpy().reshape(4, -1)
    for k in range(4):
        r = H @ X[k] - e[k] * X[k]
        assert np.linalg.norm(r) < 2e-5
        assert abs(np.linalg.norm(X[k]) - 1.0) < 1e-10
    sp.close()


def test_sel16_eigenpairs_sampled(tb, ctx):
    """norb=16, 3,000 x 3,000 (9.0M determinants), 3 roots, FP64: every returned
    pair satisfies H x = E x on 1,500 oracle-recomputed rows, and the GPU's
    residual norms are below the stopping threshold."""
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    e, info, X = sp.davidson(3, want_vectors=True)
    assert info["converged"], info
    X = X.cpu().numpy().reshape(3, -1)
    osp = oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, bsel)
    rng = np.random.default_rng(1)
    big = np.argsort(-np.abs(X[0]))[:500]
    rows = np.unique(np.concatenate([rng.choice(sp.ndet, 1000, replace=False), big]))
    hx = oracle.sigma(osp, h, eri, ecore, X, rows=rows)
    for k in range(3):
        assert np.max(np.abs(hx[k] - e[k] * X[k, rows])) < 1e-5
        assert info["residual"][k] < 1e-5
    assert e[0] <= e[1] <= e[2]
    sp.close()


def test_sel16_mixed_matches_fp64(tb, ctx):
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    e64, i64 = sp.davidson(3)
    e32, i32 = sp.davidson(3, mixed=True)
    assert i64["converged"] and i32["converged"]
    assert np.max(np.abs(e64 - e32)) < 1e-8
    sp.close()


@pytest.mark.parametrize("mixed", [0, 1])
def test_transpose_antisymmetric_ground_state(tb, ctx, mixed):
    """Identical alpha/beta sets, lowest state antisymmetric under the transpose,
    lowest diagonal entry closed-shell (norb 6, 3+3, seed 12): FP64 and mixed
    Davidson both reach the dense lowest eigenvalues."""
    n, N = 6, 3
    h, eri, _ = synth_hamiltonian(n, seed=12)
    osp = oracle.make_space(n, N, N)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(osp, h, eri, 0.0))
    sp = tb.Space(ctx, n, N, N, h, eri)
    for nroots in (1, 2, 3):
        e, info = sp.davidson(nroots, mixed=mixed)
        assert info["converged"]
        assert np.max(np.abs(e - w[:nroots])) < 1e-8, (nroots, e, w[:nroots])
    sp.close()


@pytest.mark.parametrize("mixed", [1, 2])
def test_fp32_basis_vs_dense(tb, ctx, mixed):
    """FP32-stored basis in the low-precision phase (Rayleigh problem solved against
    the measured overlap of the stored basis), then FP64 refinement on a smaller
    FP64 basis: the dense eigenvalues to 1e-8 Eh, H x = E x and unit norm for
    every returned vector. The low-precision phase runs for over a hundred
    iterations with 4 corrections each, so the FP32 basis is thick-restarted
    many times."""
    n, na, nb = 8, 4, 3
    h, eri, _ = synth_hamiltonian(n, seed=41)
    asel = selected_strings(n, na, 50, 42)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel)
    osp = oracle.make_space(n, na, nb, asel, None)
    H = oracle.hamiltonian_dense(osp, h, eri, 0.1)
    w = np.linalg.eigvalsh(H)
    e, info, X = sp.davidson(4, want_vectors=True, mixed=mixed, basis_f32=True, max_subspace=16)
    assert info["converged"], info
    assert info["nsigma_f32"] > 0 and info["nsigma"] > info["nsigma_f32"]
    assert np.max(np.abs(e - w[:4])) < 1e-8, (e, w[:4])
    X = X.cpu().numpy().reshape(4, -1)
    for k in range(4):
        assert np.linalg.norm(H @ X[k] - e[k] * X[k]) < 2e-5
        assert abs(np.linalg.norm(X[k]) - 1.0) < 1e-10
    sp.close()


def test_fp32_basis_fci8_golden(tb, ctx):
    wl = WORKLOADS["fci8"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore)
    ref = np.loadtxt(os.path.join(GOLDEN, "fci8_energies.txt"))
    e, info = sp.davidson(3, mixed=1, basis_f32=True)
    assert info["converged"]
    assert np.max(np.abs(e - ref[:3])) < 1e-8, (e, ref[:3])
    sp.close()


def test_fp32_basis_sel16_matches_fp64(tb, ctx):
    """norb=16, 3,000 x 3,000 (9.0M determinants), 3 roots: the FP32 basis with
    FP64 refinement reaches the FP64-basis energies to 1e-8 Eh."""
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    asel, bsel = wl.alpha_selection(), wl.beta_selection()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=bsel)
    e64, i64 = sp.davidson(3)
    e32, i32 = sp.davidson(3, mixed=1, basis_f32=True)
    assert i64["converged"] and i32["converged"]
    assert np.max(np.abs(e64 - e32)) < 1e-8, (e64, e32)
    sp.close()


def test_fp32_basis_argument_checks(tb, ctx):
    n, na, nb = 6, 3, 3
    h, eri, _ = synth_hamiltonian(n, seed=5)
    sp = tb.Space(ctx, n, na, nb, h, eri)
    for kw in ({"basis_f32": True},  # needs a low-precision phase
               {"basis_f32": True, "mixed": 1, "max_subspace": 8, "max_subspace_refine": 9},
               {"basis_f32": True, "mixed": 1, "max_subspace": 8, "max_subspace_refine": 2}):
        with pytest.raises(tb.B.TbsciError) as err:
            sp.davidson(2, **kw)
        assert err.value.status == tb.TBSCI_EINVAL, kw
    sp.close()


def test_restart_with_fewer_free_slots_than_roots(tb, ctx):
    """max_subspace 12 with 4 roots keeps 10 Ritz vectors at each restart, leaving
    two free slots for four corrections: the lowest unconverged roots' take them,
    and all four dense eigenvalues are still reached."""
    n, na, nb = 8, 4, 3
    h, eri, _ = synth_hamiltonian(n, seed=41)
    asel = selected_strings(n, na, 50, 42)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel)
    osp = oracle.make_space(n, na, nb, asel, None)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(osp, h, eri, 0.1))
    e, info = sp.davidson(4, max_subspace=12, restart_keep=10)
    assert info["converged"], info
    assert np.max(np.abs(e - w[:4])) < 1e-8, (e, w[:4])
    sp.close()


def _sel12_space(tb, ctx):
    """norb=12, 6+6 electrons, 250 x 260 selected strings (65,000 determinants,
    distinct alpha and beta sets): the space of tests/golden/sel12_energies.txt."""
    h, eri, ecore = synth_hamiltonian(12, seed=4012)
    a = selected_strings(12, 6, 250, 4013)
    b = selected_strings(12, 6, 260, 4014)
    return tb.Space(ctx, 12, 6, 6, h, eri, ecore, alpha=a, beta=b)


@pytest.mark.parametrize("mixed,basis_f32", [(0, False), (1, False), (2, False), (1, True)])
def test_sel12_golden_beyond_dense(tb, ctx, mixed, basis_f32):
    """65,000 determinants, 3 roots: FP64, FP32-sigma mixed, split-TF32 tensor-core
    mixed and FP32-basis solves all reach the stored oracle energies (oracle
    Davidson, cross-checked by ARPACK Lanczos on the oracle sigma) to 1e-8 Eh."""
    ref = np.loadtxt(os.path.join(GOLDEN, "sel12_energies.txt"))
    sp = _sel12_space(tb, ctx)
    assert sp.ndet == 65_000
    e, info = sp.davidson(3, mixed=mixed, basis_f32=basis_f32)
    assert info["converged"], info
    assert np.max(np.abs(e - ref)) < 1e-8, (e, ref)
    if mixed:
        assert info["nsigma_f32"] > 0
    sp.close()


def test_sel16_lowest_roots_self_consistency(tb, ctx):
    """Self-consistency check (no independent reference exists at 9.0M
    determinants): the 3 roots of the bench's workload equal the lowest 3 of a
    6-root solve, so the 3-root solve did not converge to higher states."""
    wl = WORKLOADS["sel16"]
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=wl.alpha_selection(),
                  beta=wl.beta_selection())
    e3, i3 = sp.davidson(3)
    e6, i6 = sp.davidson(6)
    assert i3["converged"] and i6["converged"]
    assert np.all(np.diff(e6) >= -1e-10)
    assert np.max(np.abs(e3 - e6[:3])) < 1e-8, (e3, e6)
    sp.close()


def test_context_options_budget_default_mode_and_tune_file(tb, tmp_path):
    """tbsci_create_ex: objects are counted against hbm_budget (a space that does
    not fit is refused with ENOMEM and nothing stays counted; closing a space
    returns its bytes); tbsci_davidson without options runs in the context's
    default mixed mode and reports the precision used and the FP64-refinement
    delta; the tune-cache file is written back by tbsci_destroy."""
    import ctypes
    n, na, nb = 8, 4, 3
    h, eri, _ = synth_hamiltonian(n, seed=41)
    asel = selected_strings(n, na, 50, 42)
    small = tb.Context(0, hbm_budget=64 << 10)
    with pytest.raises(tb.B.TbsciError) as err:
        tb.Space(small, 12, 6, 6, *synth_hamiltonian(12, seed=3)[:2])
    assert err.value.status == tb.TBSCI_ENOMEM
    assert tb.tbsci_hbm_used(small.handle) == 0
    small.close()
    path = tmp_path / "tune.txt"
    ctx = tb.Context(0, hbm_budget=1 << 30, default_mixed=1, tune_cache=str(path))
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel)
    used = tb.tbsci_hbm_used(ctx.handle)
    assert used > 0
    lib = tb.B.load()
    e = np.zeros(2)
    info = tb.B.DavidsonInfo()
    st = lib.tbsci_davidson(ctx.handle, sp.ham, sp.ta, sp.tb, 2, None, tb.B._ptr(e), None, ctypes.byref(info))
    assert st == tb.TBSCI_OK
    d = info.as_dict()
    assert d["precision"] == tb.TBSCI_F32 and d["nsigma_f32"] > 0
    assert np.allclose(np.array(d["refine_delta"][:2]), e - np.array(d["energy_f32"][:2]), atol=1e-14)
    assert max(abs(x) for x in d["refine_delta"][:2]) < 1e-3
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(oracle.make_space(n, na, nb, asel, None), h, eri, 0.1))
    assert np.max(np.abs(e - w[:2])) < 1e-8
    e64, i64 = sp.davidson(2)
    assert i64["precision"] == tb.TBSCI_F64 and i64["refine_delta"][:2] == [0.0, 0.0]
    assert tb.tbsci_hbm_used(ctx.handle) == used  # the solves' vectors were given back
    sp.close()
    assert tb.tbsci_hbm_used(ctx.handle) == 0
    ctx.close()
    assert path.read_text().startswith("tbsci-tune 1")
