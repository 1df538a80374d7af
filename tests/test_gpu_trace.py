"""Kernel trace: while tracing is on, every sigma-path launch is bracketed by
two CUDA events on its stream and read back as (kernel, ms), oldest first;
nothing is recorded while it is off, and a read drains what it returns."""
import numpy as np
import pytest

from tbsci_inputs import selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


def test_trace_of_the_fused_kernel(tb):
    import torch
    ctx = tb.Context(0)
    h, eri, _ = synth_hamiltonian(8, seed=71)
    sp = tb.Space(ctx, 8, 4, 4, h, eri)
    C = torch.randn((1, sp.la, sp.lb), dtype=torch.float64, device="cuda")
    assert tb.tbsci_trace_read(ctx.handle) == ([], 0)
    sp.sigma(C)  # not traced
    tb.tbsci_trace_enable(ctx.handle, True)
    for _ in range(3):
        sp.sigma(C)
    tb.tbsci_trace_enable(ctx.handle, False)
    sp.sigma(C)
    entries, dropped = tb.tbsci_trace_read(ctx.handle)
    assert [k for k, _ in entries] == ["k_sigma"] * 3 and dropped == 0
    assert all(ms > 0.0 for _, ms in entries)
    assert tb.tbsci_trace_read(ctx.handle) == ([], 0)
    sp.close()
    ctx.close()


def test_trace_of_the_split_path(tb, tmp_path):
    """A space pinned to the split path (stage 3) launches, per vector: the
    transpose and beta-double product, the row kernel, the combine and the
    alpha-double product, in that order; their times sum to about the sigma."""
    import torch
    n, na, nb = 10, 5, 5
    asel, bsel = selected_strings(n, na, 120, 73), selected_strings(n, nb, 200, 74)
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n%d %d %d 512 1 3 0 0 0 0 0\n" % (n, len(asel), len(bsel)))
    ctx = tb.Context(0)
    tb.tbsci_tune_cache_load(ctx.handle, str(path))
    h, eri, _ = synth_hamiltonian(n, seed=72)
    sp = tb.Space(ctx, n, na, nb, h, eri, alpha=asel, beta=bsel)
    assert sp.counts()["tuned_stage"][0] == 3
    C = torch.randn((2, sp.la, sp.lb), dtype=torch.float64, device="cuda")
    sp.sigma(C)
    torch.cuda.synchronize()
    tb.tbsci_trace_enable(ctx.handle, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sp.sigma(C)
    ev1.record()
    torch.cuda.synchronize()
    tb.tbsci_trace_enable(ctx.handle, False)
    entries, _ = tb.tbsci_trace_read(ctx.handle)
    one = ["k_transpose", "k_dbl_spmm_beta", "k_sigma_parts", "k_combine", "k_dbl_spmm_alpha"]
    assert [k for k, _ in entries] == one * 2
    total = sum(ms for _, ms in entries)
    assert 0.0 < total <= ev0.elapsed_time(ev1) * 1.05 + 0.05
    sp.close()
    ctx.close()
