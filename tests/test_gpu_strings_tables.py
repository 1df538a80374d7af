"""GPU string sets and excitation tables vs the oracle: bit-exact (rows a1, a2)."""
import math
import os

import numpy as np
import pytest

import oracle
from tbsci_inputs import WORKLOADS, selected_strings

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


@pytest.mark.parametrize("n,N", [(1, 0), (1, 1), (5, 0), (8, 4), (12, 5), (16, 8), (20, 3), (24, 12), (64, 1),
                                 (64, 63), (64, 64), (40, 2)])
def test_full_strings_bit_exact(tb, ctx, n, N):
    s = tb.tbsci_build_strings(ctx.handle, n, N, None)
    try:
        got = tb.tbsci_strings_export(ctx.handle, s)
    finally:
        tb.tbsci_strings_destroy(s)
    ref = oracle.fci_strings(n, N)
    assert got.dtype == np.uint64 and np.array_equal(got, ref)


@pytest.mark.parametrize("n,N,cnt,seed", [(8, 4, 40, 1), (16, 8, 3000, 2002), (24, 12, 40000, 2004),
                                          (10, 5, 1, 3), (10, 5, 0, 3)])
def test_selected_strings_sorted(tb, ctx, n, N, cnt, seed):
    sel = selected_strings(n, N, cnt, seed) if cnt else np.zeros(0, dtype=np.uint64)
    s = tb.tbsci_build_strings(ctx.handle, n, N, sel)
    try:
        got = tb.tbsci_strings_export(ctx.handle, s)
    finally:
        tb.tbsci_strings_destroy(s)
    st, ref = oracle.sort_validate(n, N, sel)
    assert st == 0 and np.array_equal(got, ref)


@pytest.mark.parametrize("bad,why", [([0b11, 0b11], "duplicate"), ([0b111], "electron count"),
                                     ([0b1000001], "at or above norb")])
def test_selected_strings_rejected(tb, ctx, bad, why):
    with pytest.raises(tb.B.TbsciError) as ei:
        tb.tbsci_build_strings(ctx.handle, 6, 2, np.array(bad, dtype=np.uint64))
    assert ei.value.status == tb.TBSCI_EINVAL and why in str(ei.value)


def _tables(tb, ctx, n, N, sel, flags=0):
    s = tb.tbsci_build_strings(ctx.handle, n, N, sel)
    l = tb.tbsci_strings_count(s)
    t = tb.tbsci_build_excitation_tables(ctx.handle, s, flags)
    strs = tb.tbsci_strings_export(ctx.handle, s)
    tb.tbsci_strings_destroy(s)
    return t, l, strs


@pytest.mark.parametrize("n,N,cnt,seed", [(6, 3, None, 0), (8, 4, None, 0), (10, 5, 60, 11), (12, 4, 200, 12),
                                          (16, 8, 3000, 2002), (16, 8, None, 0), (7, 0, None, 0), (7, 7, None, 0),
                                          (9, 1, None, 0)])
def test_tables_bit_exact(tb, ctx, n, N, cnt, seed):
    sel = None if cnt is None else selected_strings(n, N, cnt, seed)
    t, l, strs = _tables(tb, ctx, n, N, sel)
    try:
        off1, e1, off2, e2 = tb.tbsci_tables_export(ctx.handle, t, l)
    finally:
        tb.tbsci_tables_destroy(t)
    r1 = oracle.links_single(n, strs)
    assert np.array_equal(off1, r1[0])
    assert np.array_equal(e1["target"], r1[1]) and np.array_equal(e1["sign"], r1[2])
    assert np.array_equal(e1["p"], r1[3]) and np.array_equal(e1["q"], r1[4])
    r2 = oracle.links_double(n, strs)
    assert np.array_equal(off2, r2[0])
    for name, ref in zip(["target", "sign", "p", "r", "q", "s"], r2[1:]):
        assert np.array_equal(e2[name], ref), name
    if cnt is None:
        assert off1[-1] == math.comb(n, N) * N * (n - N)
        assert off2[-1] == math.comb(n, N) * math.comb(N, 2) * math.comb(n - N, 2)


def test_table6_single_link_counts(tb, ctx):
    """Paper Table VI (Sec. III.C): BETA_SINGLE_LINK entry counts of the four FCI
    benchmark spaces, reproduced by the device table build (count pass)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "table6_single_links.txt")
    rows = []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            name, n, nb, entries, gb = line.split()
            rows.append((name, int(n), int(nb), int(entries)))
    for name, n, nb, entries in rows:
        s = tb.tbsci_build_strings(ctx.handle, n, nb, None)
        t = tb.tbsci_build_excitation_tables(ctx.handle, s, tb.TBSCI_TABLES_SINGLES_ONLY | tb.TBSCI_TABLES_COUNT_ONLY)
        n1, n2 = tb.tbsci_tables_counts(t)
        tb.tbsci_tables_destroy(t)
        tb.tbsci_strings_destroy(s)
        assert n1 == entries, name
        assert n2 == 0


def test_table6_stored_entries_smallest(tb, ctx):
    """CN cc-pVTZ row of Table VI (58 orbitals, 4 beta electrons): the stored
    single links, checked for count, reciprocity and sign against masked loops
    on a sample of rows."""
    s = tb.tbsci_build_strings(ctx.handle, 58, 4, None)
    l = tb.tbsci_strings_count(s)
    t = tb.tbsci_build_excitation_tables(ctx.handle, s, tb.TBSCI_TABLES_SINGLES_ONLY)
    strs = tb.tbsci_strings_export(ctx.handle, s)
    off1, e1, _, _ = tb.tbsci_tables_export(ctx.handle, t, l, doubles=False)
    tb.tbsci_tables_destroy(t)
    tb.tbsci_strings_destroy(s)
    assert off1[-1] == 91642320
    rng = np.random.default_rng(0)
    for J in rng.choice(l, 200, replace=False):
        src = int(strs[J])
        for k in range(off1[J], off1[J + 1]):
            e = e1[k]
            p, q = int(e["p"]), int(e["q"])
            tgt = (src & ~(1 << q)) | (1 << p)
            assert int(strs[e["target"]]) == tgt
            lo, hi = min(p, q), max(p, q)
            between = sum((src >> x) & 1 for x in range(lo + 1, hi))
            assert int(e["sign"]) == (-1) ** between
