"""tbsci_overlap_noalloc: the overlap entry point for callers that must not
allocate device memory while they run (a framework whose caching pool already
holds all free HBM, or a serving loop that cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree). It keeps its scratch in static device
memory. This file is collected last on purpose: if it fails, a run that stops
at the first failure has already run every other test.

The test calls the new entry point through the C ABI twice in a row (with
different sizes and data, so the second call runs over the first call's
leftovers in the shared scratch) and checks each result against the existing
tbsci_overlap, within the tolerance the overlap tests use. It also checks that
a request beyond the scratch limit is refused before anything is launched.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, ctx, A, B, S, stream):
    ma, mb = int(A.shape[0]), int(B.shape[0])
    n = int(A[0].numel())
    return lib.tbsci_overlap_noalloc(ctx, ctypes.c_void_p(A.data_ptr()), ma, ctypes.c_void_p(B.data_ptr()), mb, n,
                                     ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_overlap_matches_overlap_on_two_calls():
    import torch
    import paper_2503_10335_gb300 as tb
    lib = tb.B.load()
    ctx = tb.Context(0)
    stream = torch.cuda.current_stream()
    try:
        for call, (ma, mb, n) in enumerate([(7, 5, 123_457), (16, 32, 1_000_003)]):
            rng = np.random.default_rng(100 + call)
            A = torch.from_numpy(rng.standard_normal((ma, n))).cuda()
            B = torch.from_numpy(rng.standard_normal((mb, n))).cuda()
            S = torch.full((ma * mb,), float("nan"), dtype=torch.float64, device="cuda")
            st = _call_noalloc(lib, ctx.handle, A, B, S, stream)
            assert st == tb.TBSCI_OK, tb.tbsci_last_error(ctx.handle)
            torch.cuda.synchronize()
            got = S.cpu().numpy().reshape(ma, mb)
            ref = tb.tbsci_overlap(ctx.handle, A, B)
            bound = np.abs(A.cpu().numpy()) @ np.abs(B.cpu().numpy()).T
            assert np.all(np.abs(got - ref) <= 1e-13 * bound + 1e-300), call
    finally:
        ctx.close()


def test_noalloc_overlap_refuses_oversize_request():
    import torch
    import paper_2503_10335_gb300 as tb
    lib = tb.B.load()
    ctx = tb.Context(0)
    try:
        A = torch.ones((32, 8), dtype=torch.float64, device="cuda")
        B = torch.ones((17, 8), dtype=torch.float64, device="cuda")  # 32 * 17 = 544 > 512 products
        S = torch.full((32 * 17,), -1.0, dtype=torch.float64, device="cuda")
        st = _call_noalloc(lib, ctx.handle, A, B, S, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert st == tb.TBSCI_EINVAL
        assert "512" in tb.tbsci_last_error(ctx.handle)
        assert torch.all(S == -1.0)  # nothing was written
    finally:
        ctx.close()
