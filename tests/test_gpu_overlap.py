"""tbsci_overlap: overlaps of device CI vectors vs numpy, and determinism."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("ma,mb,n", [(1, 1, 1), (3, 5, 1000), (9, 2, 4099), (24, 3, 9_000_000), (17, 13, 777)])
def test_overlap_matches_numpy(tb, ctx, ma, mb, n):
    import torch
    rng = np.random.default_rng(ma * 100 + mb)
    A = rng.standard_normal((ma, n))
    B = rng.standard_normal((mb, n))
    S = tb.tbsci_overlap(ctx.handle, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    ref = A @ B.T
    bound = np.abs(A) @ np.abs(B).T
    assert np.all(np.abs(S - ref) <= 1e-13 * bound + 1e-300)
    S2 = tb.tbsci_overlap(ctx.handle, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert np.array_equal(S, S2)


def test_overlap_empty(tb, ctx):
    import torch
    A = torch.zeros((0, 10), dtype=torch.float64, device="cuda")
    B = torch.ones((2, 10), dtype=torch.float64, device="cuda")
    assert tb.tbsci_overlap(ctx.handle, A, B).shape == (0, 2)
