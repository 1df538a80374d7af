"""Serving (row a8): continuous batching of many solves through tbsci_submit /
tbsci_poll. Each result must equal the same request solved alone (and the
oracle's dense eigenvalues for the small ones), whatever else ran beside it."""
import time

import numpy as np
import pytest

import oracle
from tbsci_inputs import selected_strings, synth_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import paper_2503_10335_gb300 as tb
    return tb


def _requests(seed=0, n=10):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        norb = int(rng.choice([6, 7, 8, 9, 10]))
        na = norb // 2
        nb = int(rng.integers(max(1, na - 1), na + 1))
        h, eri, _ = synth_hamiltonian(norb, seed=int(rng.integers(1 << 30)))
        cnt = int(rng.integers(8, 60))
        asel = selected_strings(norb, na, cnt, int(rng.integers(1 << 30)))
        bsel = None if i % 3 == 0 else selected_strings(norb, nb, cnt + 5, int(rng.integers(1 << 30)))
        out.append(dict(norb=norb, nalpha=na, nbeta=nb, h=h, eri=eri, ecore=0.1 * i, alpha=asel, beta=bsel,
                        nroots=1 + i % 3, mixed=bool(i % 2)))
    return out


def _solve_all(srv, reqs, stagger=0.0):
    tickets = []
    for r in reqs:
        tickets.append(srv.submit(**r))
        if stagger:
            time.sleep(stagger)
    res = []
    for t in tickets:
        st, d = srv.poll(t, timeout_ms=120000)
        assert st == 0, st
        res.append(d)
    return res


def test_results_same_alone_and_in_the_mix(tb):
    reqs = _requests(1, 10)
    srv = tb.Server(0)
    try:
        mixed_res = _solve_all(srv, reqs, stagger=0.002)
        alone = []
        for r in reqs:
            alone.append(_solve_all(srv, [r])[0])
    finally:
        srv.close()
    for r, a, b in zip(reqs, mixed_res, alone):
        assert a["status"] == 0 and b["status"] == 0
        assert np.max(np.abs(np.array(a["energies"]) - np.array(b["energies"]))) < 1e-8
        osp = oracle.make_space(r["norb"], r["nalpha"], r["nbeta"], r["alpha"], r["beta"])
        if osp.ndet <= 2500:
            w = np.linalg.eigvalsh(oracle.hamiltonian_dense(osp, r["h"], r["eri"], r["ecore"]))[:r["nroots"]]
            assert np.max(np.abs(np.array(a["energies"]) - w)) < 1e-8
        assert a["t_submit"] <= a["t_admit"] <= a["t_first_sigma"] <= a["t_done"]


def test_budget_admission_serialises_and_oversize_is_refused(tb):
    reqs = _requests(2, 4)
    srv = tb.Server(0, hbm_budget=1)  # nothing fits: every request is refused
    try:
        for d in _solve_all(srv, reqs[:2]):
            assert d["status"] == tb.TBSCI_ENOMEM
    finally:
        srv.close()
    # one solve at a time still gives every result
    srv = tb.Server(0, max_active=1)
    try:
        res = _solve_all(srv, reqs)
        assert all(d["status"] == 0 for d in res)
        # with one slot, admissions follow completions
        for prev, nxt in zip(res, res[1:]):
            assert nxt["t_admit"] >= prev["t_done"] - 1e-3
    finally:
        srv.close()


def test_unfused_sigma_gives_the_same_results(tb):
    reqs = _requests(3, 6)
    a = tb.Server(0)
    b = tb.Server(0, fuse_sigma=-1)
    try:
        ra = _solve_all(a, reqs)
        rb = _solve_all(b, reqs)
    finally:
        a.close()
        b.close()
    for x, y in zip(ra, rb):
        assert np.max(np.abs(np.array(x["energies"]) - np.array(y["energies"]))) < 1e-8


def test_poll_timeout_queue_limit_and_injected_failure(tb):
    reqs = _requests(4, 3)
    srv = tb.Server(0, max_queue=1, fail_admission_at=2)
    try:
        t1 = srv.submit(**reqs[0])
        # unknown ticket
        st, _ = srv.poll(999999, timeout_ms=0)
        assert st == tb.TBSCI_EINVAL
        st, d = srv.poll(t1, timeout_ms=60000)
        assert st == 0 and d["status"] == 0
        t2 = srv.submit(**reqs[1])   # second admission: the injected allocation failure
        st, d = srv.poll(t2, timeout_ms=60000)
        assert st == 0 and d["status"] == tb.TBSCI_ENOMEM
        t3 = srv.submit(**reqs[2])
        st, d = srv.poll(t3, timeout_ms=60000)
        assert st == 0 and d["status"] == 0
    finally:
        srv.close()


def test_server_with_tune_cache(tb, tmp_path):
    """A server created with a tune cache file serves solves as before (the file
    only changes launch shapes); an unreadable cache file is refused at creation."""
    with pytest.raises(tb.B.TbsciError):
        tb.Server(0, tune_cache=str(tmp_path / "missing.txt"))
    path = tmp_path / "tune.txt"
    path.write_text("tbsci-tune 1\n8 40 45 128 1 0 256 1 1 0 0\n")
    reqs = _requests(4, 4)
    srv = tb.Server(0, tune_cache=str(path))
    plain = tb.Server(0)
    try:
        ra = _solve_all(srv, reqs)
        rb = _solve_all(plain, reqs)
    finally:
        srv.close()
        plain.close()
    for x, y in zip(ra, rb):
        assert np.max(np.abs(np.array(x["energies"]) - np.array(y["energies"]))) < 1e-8


def test_large_job_same_alone_and_in_the_mix(tb):
    """Two requests above the batching threshold (2^20 determinant-vectors: full
    norb 12, 6+6 space, 853,776 determinants x 2 roots, one FP64 and one mixed)
    launch their sigma on their own streams while small solves ride in the
    batched launches beside them. Each result equals the same request solved
    alone on the server and the blocking tbsci_davidson solve, to 1e-8 Eh."""
    small = _requests(5, 8)
    h, eri, _ = synth_hamiltonian(12, seed=5012)
    big = [dict(norb=12, nalpha=6, nbeta=6, h=h, eri=eri, ecore=0.0, alpha=None, beta=None, nroots=2,
                mixed=m) for m in (False, True)]
    reqs = small[:3] + [big[0]] + small[3:6] + [big[1]] + small[6:]
    srv = tb.Server(0)
    try:
        mixed_res = _solve_all(srv, reqs, stagger=0.01)
        alone = [_solve_all(srv, [r])[0] for r in reqs]
    finally:
        srv.close()
    for r, a, b in zip(reqs, mixed_res, alone):
        assert a["status"] == 0 and b["status"] == 0
        assert np.max(np.abs(np.array(a["energies"]) - np.array(b["energies"]))) < 1e-8
    ctx = tb.Context(0)
    sp = tb.Space(ctx, 12, 6, 6, h, eri, 0.0)
    assert sp.ndet * 2 > (1 << 20)
    e, info = sp.davidson(2)
    assert info["converged"]
    for k in (3, 7):
        assert np.max(np.abs(np.array(mixed_res[k]["energies"]) - e)) < 1e-8, (k, mixed_res[k], e)
    sp.close()
    ctx.close()


def test_tensor_core_mixed_requests_in_the_mix(tb):
    """Requests whose low-precision phase uses the tensor-core sigma types (2:
    split TF32, 3: BF16) ride beside FP64 and FP32-sigma requests in the same
    server; each result equals the dense eigenvalues to 1e-8 Eh after the FP64
    refinement. A mode outside 0..3 is refused at submit."""
    reqs = _requests(6, 8)
    for i, r in enumerate(reqs):
        r["mixed"] = i % 4
    srv = tb.Server(0)
    try:
        with pytest.raises(tb.B.TbsciError):
            srv.submit(**dict(reqs[0], mixed=4))
        res = _solve_all(srv, reqs, stagger=0.002)
    finally:
        srv.close()
    for r, d in zip(reqs, res):
        assert d["status"] == 0
        osp = oracle.make_space(r["norb"], r["nalpha"], r["nbeta"], r["alpha"], r["beta"])
        w = np.linalg.eigvalsh(oracle.hamiltonian_dense(osp, r["h"], r["eri"], r["ecore"]))[:r["nroots"]]
        assert np.max(np.abs(np.array(d["energies"]) - w)) < 1e-8, (r["mixed"], d["energies"], w)
        if r["mixed"]:
            assert d["nsigma_f32"] > 0
