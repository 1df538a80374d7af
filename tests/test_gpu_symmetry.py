"""Point-group symmetry blocking (Sec. II.A): with D2h-labelled integrals H is
block diagonal by determinant irrep. The GPU symmetry blocks (pruned spaces of
one irrep) are compared with the oracle's blocks, and the lowest eigenvalues of
the full space are the lowest of the blocks' eigenvalues together."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_sigma_close
from tbsci_inputs import orbital_irreps, selected_strings, synth_hamiltonian_symmetric

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


@pytest.mark.parametrize("n,na,nb,acnt,bcnt", [(8, 4, 4, None, None), (10, 5, 4, 150, None), (12, 6, 6, 300, 280)])
def test_symmetry_block_sigma_matches_the_oracle(tb, ctx, n, na, nb, acnt, bcnt):
    import torch
    g = orbital_irreps(n, seed=950 + n)
    h, eri, _ = synth_hamiltonian_symmetric(n, 951 + n, g)
    asel = None if acnt is None else selected_strings(n, na, acnt, 952 + n)
    bsel = None if bcnt is None else selected_strings(n, nb, bcnt, 953 + n)
    sp = tb.Space(ctx, n, na, nb, h, eri, 0.1, alpha=asel, beta=bsel)
    osp = oracle.make_space(n, na, nb, asel, bsel)
    total = 0
    for t in range(8):
        blk = sp.symmetry_block(g, t)
        ops = oracle.symmetry_space(osp, g, t)
        assert blk.ndet == ops.ndet
        total += blk.ndet
        if blk.ndet == 0:
            blk.close()
            continue
        C = np.random.default_rng(t).standard_normal((1, blk.ndet))
        s = blk.sigma(torch.from_numpy(C).cuda()).cpu().numpy()
        ref, bound = oracle.sigma_pruned(ops, h, eri, 0.1, C, with_bound=True)
        assert_sigma_close(s, ref, bound)
        blk.close()
    assert total == sp.ndet
    sp.close()


def test_blocks_together_give_the_dense_spectrum(tb, ctx):
    """norb 8, 4+4, all 70 x 70 strings with D2h labels: the lowest eigenvalues
    of the eight symmetry blocks (GPU Davidson per block) are eigenvalues of the
    dense H of the whole space, and the lowest 4 of them together are its lowest
    4 (to 1e-8 Eh)."""
    n, N = 8, 4
    g = orbital_irreps(n, seed=955)
    h, eri, _ = synth_hamiltonian_symmetric(n, 956, g)
    w = np.linalg.eigvalsh(oracle.hamiltonian_dense(oracle.make_space(n, N, N), h, eri, 0.0))
    sp = tb.Space(ctx, n, N, N, h, eri)
    block_e = []
    for t in range(8):
        blk = sp.symmetry_block(g, t)
        assert blk.ndet >= 64  # each block of this space is large enough for a 4-root solve
        e, info = blk.davidson(4)
        assert info["converged"]
        for x in e:
            assert np.min(np.abs(w - x)) < 1e-8
        block_e.extend(list(e))
        blk.close()
    assert np.max(np.abs(np.sort(block_e)[:4] - w[:4])) < 1e-8, (np.sort(block_e)[:4], w[:4])
    sp.close()


def test_full_space_solve_lies_in_the_blocks(tb, ctx):
    """norb 12, 6+6, all 924 x 924 strings (853,776 determinants) with D2h labels.
    H never couples two blocks, so Davidson on the whole space stays in the
    symmetry sectors of its guess: every root it returns is an eigenvalue of one
    block, and the lowest block energy is at or below its lowest root (it can
    miss a sector, which is why solves run block by block). A vector supported on
    one block stays in it under H."""
    import torch
    n, N = 12, 6
    g = orbital_irreps(n, seed=960)
    h, eri, _ = synth_hamiltonian_symmetric(n, 961, g)
    sp = tb.Space(ctx, n, N, N, h, eri)
    e_full, info = sp.davidson(3)
    assert info["converged"]
    block_e = []
    for t in range(8):
        blk = sp.symmetry_block(g, t)
        if blk.ndet >= 8:
            e, i = blk.davidson(6)
            assert i["converged"]
            block_e.extend(e.tolist())
        blk.close()
    block_e = np.array(block_e)
    assert np.min(block_e) <= e_full[0] + 1e-10
    for x in e_full:
        assert np.min(np.abs(block_e - x)) < 1e-8, (x, np.sort(block_e)[:8])
    # H keeps a one-block vector inside its block
    osp = oracle.make_space(n, N, N)
    ga = np.array([oracle.string_irrep(s, g) for s in osp.sa])
    irr = ga[:, None] ^ ga[None, :]
    v = torch.zeros((1, sp.la, sp.lb), dtype=torch.float64, device="cuda")
    mask = torch.from_numpy(irr == 5).cuda()
    v[0][mask] = torch.randn(int(mask.sum()), dtype=torch.float64, device="cuda")
    s = sp.sigma(v)
    assert float(torch.max(torch.abs(s[0][~mask]))) == 0.0
    sp.close()


def test_symmetry_block_errors(tb, ctx):
    n = 6
    g = orbital_irreps(n, seed=970)
    h, eri, _ = synth_hamiltonian_symmetric(n, 971, g)
    sp = tb.Space(ctx, n, 3, 3, h, eri)
    for labels, target in ((g, 8), (g, -1), (np.full(n, 9), 0)):
        with pytest.raises(tb.B.TbsciError) as err:
            sp.symmetry_block(labels, target)
        assert err.value.status == tb.TBSCI_EINVAL
    sp.close()
