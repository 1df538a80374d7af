"""ctypes binding of libtbsci (include/tbsci.h): argument marshalling only.

Every function named ``tbsci_*`` here calls the C entry point of the same name;
all computation runs in the library's CUDA kernels. Device arrays are torch
tensors (their ``data_ptr()`` is passed), streams are torch CUDA streams. The
binding raises ``TbsciError`` on any non-OK status and ``RuntimeError`` when the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtbsci.so")

TBSCI_OK, TBSCI_EINVAL, TBSCI_ENOMEM, TBSCI_ECUDA, TBSCI_ENOCONV, TBSCI_EAGAIN, TBSCI_ETIMEOUT, TBSCI_EBUSY = range(8)
TBSCI_F64, TBSCI_F32, TBSCI_F32_TC_TF32, TBSCI_F32_TC_BF16 = 0, 1, 2, 3
TBSCI_TABLES_SINGLES_ONLY, TBSCI_TABLES_COUNT_ONLY = 1, 2

# exported names declared in include/tbsci.h
EXPORTS = [
    "tbsci_create", "tbsci_destroy", "tbsci_last_error", "tbsci_status_string",
    "tbsci_build_strings", "tbsci_strings_count", "tbsci_strings_export", "tbsci_strings_destroy",
    "tbsci_build_excitation_tables", "tbsci_tables_counts", "tbsci_tables_export", "tbsci_tables_destroy",
    "tbsci_hamiltonian_create", "tbsci_hamiltonian_destroy", "tbsci_prepare", "tbsci_sigma",
    "tbsci_sigma_host", "tbsci_diagonal", "tbsci_sigma_counts_get", "tbsci_davidson", "tbsci_overlap",
    "tbsci_overlap_noalloc", "tbsci_server_create", "tbsci_submit", "tbsci_poll", "tbsci_server_load",
    "tbsci_server_destroy", "tbsci_sigma_autotune", "tbsci_tune_cache_save", "tbsci_tune_cache_load",
    "tbsci_tune_cache_size", "tbsci_create_ex", "tbsci_hbm_used",
    "tbsci_pruned_create", "tbsci_pruned_count", "tbsci_pruned_destroy", "tbsci_sigma_pruned",
    "tbsci_diagonal_pruned", "tbsci_davidson_pruned", "tbsci_string_weights", "tbsci_select_by_weight",
    "tbsci_coefficient_histogram", "tbsci_pruned_create_symmetry", "tbsci_trace_enable", "tbsci_trace_read",
]


class SingleLink(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int32), ("sign", ctypes.c_int8), ("p", ctypes.c_uint8),
                ("q", ctypes.c_uint8), ("pad", ctypes.c_uint8)]


class DoubleLink(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int32), ("sign", ctypes.c_int8), ("p", ctypes.c_uint8),
                ("r", ctypes.c_uint8), ("q", ctypes.c_uint8), ("s", ctypes.c_uint8),
                ("pad", ctypes.c_uint8 * 3)]


SINGLE_DTYPE = np.dtype([("target", "<i4"), ("sign", "i1"), ("p", "u1"), ("q", "u1"), ("pad", "u1")])
DOUBLE_DTYPE = np.dtype([("target", "<i4"), ("sign", "i1"), ("p", "u1"), ("r", "u1"), ("q", "u1"),
                         ("s", "u1"), ("pad", "u1", (3,))])
assert SINGLE_DTYPE.itemsize == 8 and DOUBLE_DTYPE.itemsize == 12


class TraceEntry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char_p), ("ms", ctypes.c_double)]


class SigmaCounts(ctypes.Structure):
    _fields_ = [("ndet", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nnz_aa", ctypes.c_int64),
                ("nnz_bb", ctypes.c_int64), ("nnz_ab", ctypes.c_int64), ("bytes_tables", ctypes.c_int64),
                ("tuned_threads", ctypes.c_int32 * 2), ("tuned_nv", ctypes.c_int32 * 2),
                ("tuned_stage", ctypes.c_int32 * 2), ("tuned_rest", ctypes.c_int32 * 2)]


class DavidsonOpts(ctypes.Structure):
    _fields_ = [("max_subspace", ctypes.c_int), ("restart_keep", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol_energy", ctypes.c_double),
                ("tol_residual", ctypes.c_double), ("mixed", ctypes.c_int),
                ("tol_mixed_residual", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("basis_f32", ctypes.c_int), ("max_subspace_refine", ctypes.c_int)]


class DavidsonInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("nsigma", ctypes.c_int),
                ("nsigma_f32", ctypes.c_int), ("iterations_f32", ctypes.c_int),
                ("residual", ctypes.c_double * 8), ("energy_f32", ctypes.c_double * 8),
                ("seconds_total", ctypes.c_double), ("seconds_sigma", ctypes.c_double),
                ("seconds_sigma_f32", ctypes.c_double), ("precision", ctypes.c_int),
                ("refine_delta", ctypes.c_double * 8)]

    def as_dict(self):
        return dict(iterations=self.iterations, converged=bool(self.converged), nsigma=self.nsigma,
                    nsigma_f32=self.nsigma_f32, iterations_f32=self.iterations_f32,
                    residual=list(self.residual), energy_f32=list(self.energy_f32),
                    seconds_total=self.seconds_total, seconds_sigma=self.seconds_sigma,
                    seconds_sigma_f32=self.seconds_sigma_f32, precision=self.precision,
                    refine_delta=list(self.refine_delta))


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("default_mixed", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("fuse_sigma", ctypes.c_int), ("fail_admission_at", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p)]


class Request(ctypes.Structure):
    _fields_ = [("norb", ctypes.c_int), ("nalpha", ctypes.c_int), ("nbeta", ctypes.c_int),
                ("h", ctypes.c_void_p), ("eri", ctypes.c_void_p), ("ecore", ctypes.c_double),
                ("alpha", ctypes.c_void_p), ("n_alpha", ctypes.c_int64), ("beta", ctypes.c_void_p),
                ("n_beta", ctypes.c_int64), ("nroots", ctypes.c_int), ("mixed", ctypes.c_int),
                ("tol_energy", ctypes.c_double), ("tol_residual", ctypes.c_double), ("max_iter", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nroots", ctypes.c_int), ("energies", ctypes.c_double * 8),
                ("residual", ctypes.c_double * 8), ("iterations", ctypes.c_int), ("nsigma", ctypes.c_int),
                ("nsigma_f32", ctypes.c_int), ("ndet", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_first_sigma", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        n = self.nroots
        return dict(status=self.status, energies=list(self.energies[:n]), residual=list(self.residual[:n]),
                    iterations=self.iterations, nsigma=self.nsigma, nsigma_f32=self.nsigma_f32, ndet=self.ndet,
                    t_submit=self.t_submit, t_admit=self.t_admit, t_first_sigma=self.t_first_sigma,
                    t_done=self.t_done)


class TbsciError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tbsci status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load(path: str | None = None):
    """Loads libtbsci.so (raises if it has not been built). An explicit ``path``
    loads that file without caching it."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libtbsci.so is not built (%s); run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "tbsci_create": ([I, PP], I),
        "tbsci_create_ex": ([ctypes.POINTER(Options), PP], I),
        "tbsci_hbm_used": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
        "tbsci_trace_enable": ([P, I], I),
        "tbsci_trace_read": ([P, ctypes.POINTER(TraceEntry), I64, ctypes.POINTER(I64), ctypes.POINTER(I64)], I),
        "tbsci_string_weights": ([P, P, P, P, P, P, P], I),
        "tbsci_select_by_weight": ([P, P, P, P, D, P, ctypes.POINTER(I64), P, ctypes.POINTER(I64), P], I),
        "tbsci_coefficient_histogram": ([P, P, I64, P, I, P, P], I),
        "tbsci_pruned_create": ([P, P, P, P, P, PP], I),
        "tbsci_pruned_create_symmetry": ([P, P, P, P, I, PP], I),
        "tbsci_pruned_count": ([P, ctypes.POINTER(I64)], I),
        "tbsci_pruned_destroy": ([P], None),
        "tbsci_sigma_pruned": ([P, P, P, P, P, P, P, I, I, P], I),
        "tbsci_diagonal_pruned": ([P, P, P, P, P, P, P], I),
        "tbsci_davidson_pruned": ([P, P, P, P, P, I, ctypes.POINTER(DavidsonOpts), P, P,
                                   ctypes.POINTER(DavidsonInfo)], I),
        "tbsci_destroy": ([P], None),
        "tbsci_last_error": ([P], ctypes.c_char_p),
        "tbsci_status_string": ([I], ctypes.c_char_p),
        "tbsci_build_strings": ([P, I, I, P, I64, PP], I),
        "tbsci_strings_count": ([P, ctypes.POINTER(I64)], I),
        "tbsci_strings_export": ([P, P, P], I),
        "tbsci_strings_destroy": ([P], None),
        "tbsci_build_excitation_tables": ([P, P, I, PP], I),
        "tbsci_tables_counts": ([P, ctypes.POINTER(I64), ctypes.POINTER(I64)], I),
        "tbsci_tables_export": ([P, P, P, P, P, P], I),
        "tbsci_tables_destroy": ([P], None),
        "tbsci_hamiltonian_create": ([P, I, P, P, D, PP], I),
        "tbsci_hamiltonian_destroy": ([P], None),
        "tbsci_prepare": ([P, P, P, P], I),
        "tbsci_sigma": ([P, P, P, P, P, P, I, I, P], I),
        "tbsci_sigma_host": ([P, P, P, P, P, P, I], I),
        "tbsci_diagonal": ([P, P, P, P, P, P], I),
        "tbsci_sigma_counts_get": ([P, P, P, P, ctypes.POINTER(SigmaCounts)], I),
        "tbsci_davidson": ([P, P, P, P, I, ctypes.POINTER(DavidsonOpts), P, P, ctypes.POINTER(DavidsonInfo)], I),
        "tbsci_overlap": ([P, P, I, P, I, I64, P, P], I),
        "tbsci_overlap_noalloc": ([P, P, I, P, I, I64, P, P], I),
        "tbsci_server_create": ([ctypes.POINTER(ServerOpts), PP], I),
        "tbsci_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], I),
        "tbsci_poll": ([P, ctypes.c_uint64, I, ctypes.POINTER(Result)], I),
        "tbsci_server_load": ([P, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "tbsci_server_destroy": ([P], None),
        "tbsci_sigma_autotune": ([P, P, P, P, P, P, I, I, P, ctypes.POINTER(D)], I),
        "tbsci_tune_cache_save": ([P, ctypes.c_char_p], I),
        "tbsci_tune_cache_load": ([P, ctypes.c_char_p], I),
        "tbsci_tune_cache_size": ([P, ctypes.POINTER(I64)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(ctx, st):
    if st != TBSCI_OK:
        msg = load().tbsci_last_error(ctx).decode() if ctx else ""
        raise TbsciError(st, msg)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- handles

def tbsci_create(device: int = 0):
    h = ctypes.c_void_p()
    st = load().tbsci_create(device, ctypes.byref(h))
    if st != TBSCI_OK:
        raise TbsciError(st, "tbsci_create(%d) failed" % device)
    return h


def tbsci_create_ex(device: int = 0, hbm_budget: int = 0, default_mixed: int = 0, tune_cache=None):
    o = Options(device, hbm_budget, default_mixed, None if tune_cache is None else os.fsencode(tune_cache))
    h = ctypes.c_void_p()
    st = load().tbsci_create_ex(ctypes.byref(o), ctypes.byref(h))
    if st != TBSCI_OK:
        raise TbsciError(st, "tbsci_create_ex(device %d) failed" % device)
    return h


def tbsci_hbm_used(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, load().tbsci_hbm_used(ctx, ctypes.byref(n)))
    return n.value


def tbsci_destroy(ctx):
    load().tbsci_destroy(ctx)


def tbsci_trace_enable(ctx, on: bool) -> None:
    _check(ctx, load().tbsci_trace_enable(ctx, 1 if on else 0))


def tbsci_trace_read(ctx, chunk: int = 4096):
    """Drains the kernel trace: ([(kernel, ms), ...] oldest first, entries dropped)."""
    out, dropped = [], 0
    buf = (TraceEntry * chunk)()
    while True:
        n, d = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(ctx, load().tbsci_trace_read(ctx, buf, chunk, ctypes.byref(n), ctypes.byref(d)))
        dropped += d.value
        out.extend((buf[i].kernel.decode(), buf[i].ms) for i in range(n.value))
        if n.value < chunk:
            return out, dropped


def tbsci_last_error(ctx) -> str:
    return load().tbsci_last_error(ctx).decode()


def tbsci_build_strings(ctx, norb: int, nelec: int, selected=None):
    out = ctypes.c_void_p()
    if selected is None:
        st = load().tbsci_build_strings(ctx, norb, nelec, None, 0, ctypes.byref(out))
    else:
        sel = np.ascontiguousarray(np.asarray(selected, dtype=np.uint64))
        st = load().tbsci_build_strings(ctx, norb, nelec, _ptr(sel), len(sel), ctypes.byref(out))
    _check(ctx, st)
    return out


def tbsci_strings_count(s) -> int:
    c = ctypes.c_int64()
    st = load().tbsci_strings_count(s, ctypes.byref(c))
    if st:
        raise TbsciError(st, "strings_count")
    return c.value


def tbsci_strings_export(ctx, s) -> np.ndarray:
    out = np.zeros(tbsci_strings_count(s), dtype=np.uint64)
    _check(ctx, load().tbsci_strings_export(ctx, s, _ptr(out)))
    return out


def tbsci_strings_destroy(s):
    load().tbsci_strings_destroy(s)


def tbsci_build_excitation_tables(ctx, strings, flags: int = 0):
    out = ctypes.c_void_p()
    _check(ctx, load().tbsci_build_excitation_tables(ctx, strings, flags, ctypes.byref(out)))
    return out


def tbsci_tables_counts(t):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    st = load().tbsci_tables_counts(t, ctypes.byref(a), ctypes.byref(b))
    if st:
        raise TbsciError(st, "tables_counts")
    return a.value, b.value


def tbsci_tables_export(ctx, t, nrows: int, singles=True, doubles=True):
    """Returns ``(off1, ent1, off2, ent2)`` as numpy arrays (structured entries)."""
    n1, n2 = tbsci_tables_counts(t)
    off1 = np.zeros(nrows + 1, dtype=np.int64)
    off2 = np.zeros(nrows + 1, dtype=np.int64) if doubles else None
    e1 = np.zeros(n1, dtype=SINGLE_DTYPE) if singles else None
    e2 = np.zeros(n2, dtype=DOUBLE_DTYPE) if doubles else None
    _check(ctx, load().tbsci_tables_export(ctx, t, _ptr(off1), _ptr(e1), _ptr(off2), _ptr(e2)))
    return off1, e1, off2, e2


def tbsci_tables_destroy(t):
    load().tbsci_tables_destroy(t)


def tbsci_hamiltonian_create(ctx, h, eri, ecore: float = 0.0):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    n = h.shape[0]
    out = ctypes.c_void_p()
    _check(ctx, load().tbsci_hamiltonian_create(ctx, n, _ptr(h), _ptr(eri), float(ecore), ctypes.byref(out)))
    return out


def tbsci_hamiltonian_destroy(ham):
    load().tbsci_hamiltonian_destroy(ham)


def tbsci_prepare(ctx, ham, ta, tb):
    _check(ctx, load().tbsci_prepare(ctx, ham, ta, tb))


def tbsci_sigma(ctx, ham, ta, tb, c, sigma, nvec: int, dtype: int = TBSCI_F64, stream=None):
    """sigma <- H c on device tensors [nvec][la][lb] (F64 or F32)."""
    _check(ctx, load().tbsci_sigma(ctx, ham, ta, tb, _ptr(c), _ptr(sigma), int(nvec), int(dtype), _stream(stream)))


def tbsci_sigma_autotune(ctx, ham, ta, tb, c, sigma, nvec: int, dtype: int = TBSCI_F64, stream=None) -> float:
    """Tunes the sigma launch shape on (c, sigma); returns the chosen shape's time in ms."""
    ms = ctypes.c_double()
    _check(ctx, load().tbsci_sigma_autotune(ctx, ham, ta, tb, _ptr(c), _ptr(sigma), int(nvec), int(dtype),
                                            _stream(stream), ctypes.byref(ms)))
    return ms.value


def tbsci_tune_cache_save(ctx, path):
    """Writes the context's autotune cache (shapes keyed by norb, l_alpha, l_beta) to ``path``."""
    _check(ctx, load().tbsci_tune_cache_save(ctx, os.fsencode(path)))


def tbsci_tune_cache_load(ctx, path):
    """Merges an autotune cache file into the context; applies to spaces prepared afterwards."""
    _check(ctx, load().tbsci_tune_cache_load(ctx, os.fsencode(path)))


def tbsci_tune_cache_size(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().tbsci_tune_cache_size(ctx, ctypes.byref(n)))
    return n.value


def tbsci_sigma_host(ctx, ham, ta, tb, c: np.ndarray, sigma: np.ndarray, nvec: int):
    """sigma <- H c with host FP64 arrays (copies inside the call)."""
    assert c.dtype == np.float64 and sigma.dtype == np.float64
    assert c.flags.c_contiguous and sigma.flags.c_contiguous
    _check(ctx, load().tbsci_sigma_host(ctx, ham, ta, tb, _ptr(c), _ptr(sigma), int(nvec)))


def tbsci_diagonal(ctx, ham, ta, tb, diag, stream=None):
    _check(ctx, load().tbsci_diagonal(ctx, ham, ta, tb, _ptr(diag), _stream(stream)))


def tbsci_sigma_counts_get(ctx, ham, ta, tb) -> dict:
    c = SigmaCounts()
    _check(ctx, load().tbsci_sigma_counts_get(ctx, ham, ta, tb, ctypes.byref(c)))
    d = {k: getattr(c, k) for k, _ in SigmaCounts._fields_}
    d["tuned_threads"] = list(c.tuned_threads)
    d["tuned_nv"] = list(c.tuned_nv)
    d["tuned_stage"] = list(c.tuned_stage)
    d["tuned_rest"] = list(c.tuned_rest)
    return d


def tbsci_davidson(ctx, ham, ta, tb, nroots: int, vecs=None, max_subspace=0, max_iter=0, tol_energy=0.0,
                   tol_residual=0.0, mixed=False, tol_mixed_residual=0.0, stream=None, check=True,
                   restart_keep=0, basis_f32=False, max_subspace_refine=0):
    """Lowest ``nroots`` energies (numpy) and the info dict; ``vecs`` (device FP64
    tensor [nroots][la][lb]) receives the eigenvectors when given."""
    o = DavidsonOpts(max_subspace, restart_keep, max_iter, tol_energy, tol_residual, int(mixed),
                     tol_mixed_residual,
                     None if stream is None else _stream(stream).value, int(basis_f32), max_subspace_refine)
    e = np.zeros(nroots)
    info = DavidsonInfo()
    st = load().tbsci_davidson(ctx, ham, ta, tb, nroots, ctypes.byref(o), _ptr(e), _ptr(vecs), ctypes.byref(info))
    if check or st not in (TBSCI_OK, TBSCI_ENOCONV):
        _check(ctx, st)
    d = info.as_dict()
    d["status"] = st
    return e, d


def tbsci_string_weights(ctx, ta, tb, c, la: int, lb: int, stream=None):
    """(W_a [la], W_b [lb]) numpy arrays for the FP64 device vector c."""
    wa, wb = np.zeros(la), np.zeros(lb)
    _check(ctx, load().tbsci_string_weights(ctx, ta, tb, _ptr(c), _ptr(wa), _ptr(wb), _stream(stream)))
    return wa, wb


def tbsci_select_by_weight(ctx, ta, tb, c, delta: float, la: int, lb: int, stream=None):
    """(kept alpha strings, kept beta strings) as uint64 numpy arrays."""
    sa, sb = np.zeros(la, dtype=np.uint64), np.zeros(lb, dtype=np.uint64)
    na, nb = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().tbsci_select_by_weight(ctx, ta, tb, _ptr(c), float(delta), _ptr(sa), ctypes.byref(na),
                                              _ptr(sb), ctypes.byref(nb), _stream(stream)))
    return sa[:na.value].copy(), sb[:nb.value].copy()


def tbsci_coefficient_histogram(ctx, x, edges, stream=None) -> np.ndarray:
    """Counts [len(edges) + 1] of |x| per bin of the ascending edges."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    counts = np.zeros(len(e) + 1, dtype=np.int64)
    _check(ctx, load().tbsci_coefficient_histogram(ctx, _ptr(x), int(x.numel()), _ptr(e), len(e), _ptr(counts),
                                                   _stream(stream)))
    return counts


def tbsci_pruned_create(ctx, ta, tb, off, cols):
    """Pruned space from host CSR arrays (off [la + 1], cols [off[la]])."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(ctx, load().tbsci_pruned_create(ctx, ta, tb, _ptr(off), _ptr(cols) if len(cols) else None,
                                           ctypes.byref(out)))
    return out


def tbsci_pruned_create_symmetry(ctx, ta, tb, orb_irrep, target: int):
    """Symmetry block of irrep ``target`` (orbital labels 0..7, XOR products)."""
    g = np.ascontiguousarray(orb_irrep, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(ctx, load().tbsci_pruned_create_symmetry(ctx, ta, tb, _ptr(g), int(target), ctypes.byref(out)))
    return out


def tbsci_pruned_count(pr) -> int:
    n = ctypes.c_int64()
    st = load().tbsci_pruned_count(pr, ctypes.byref(n))
    if st:
        raise TbsciError(st, "pruned_count")
    return n.value


def tbsci_pruned_destroy(pr):
    load().tbsci_pruned_destroy(pr)


def tbsci_sigma_pruned(ctx, ham, ta, tb, pr, c, sigma, nvec: int, dtype: int = TBSCI_F64, stream=None):
    _check(ctx, load().tbsci_sigma_pruned(ctx, ham, ta, tb, pr, _ptr(c), _ptr(sigma), int(nvec), int(dtype),
                                          _stream(stream)))


def tbsci_diagonal_pruned(ctx, ham, ta, tb, pr, diag, stream=None):
    _check(ctx, load().tbsci_diagonal_pruned(ctx, ham, ta, tb, pr, _ptr(diag), _stream(stream)))


def tbsci_davidson_pruned(ctx, ham, ta, tb, pr, nroots: int, vecs=None, max_subspace=0, max_iter=0,
                          tol_energy=0.0, tol_residual=0.0, mixed=False, tol_mixed_residual=0.0, stream=None,
                          check=True, restart_keep=0, basis_f32=False, max_subspace_refine=0):
    """tbsci_davidson on a pruned space; ``vecs``: device FP64 [nroots][ndet] or None."""
    o = DavidsonOpts(max_subspace, restart_keep, max_iter, tol_energy, tol_residual, int(mixed),
                     tol_mixed_residual,
                     None if stream is None else _stream(stream).value, int(basis_f32), max_subspace_refine)
    e = np.zeros(nroots)
    info = DavidsonInfo()
    st = load().tbsci_davidson_pruned(ctx, ham, ta, tb, pr, nroots, ctypes.byref(o), _ptr(e), _ptr(vecs),
                                      ctypes.byref(info))
    if check or st not in (TBSCI_OK, TBSCI_ENOCONV):
        _check(ctx, st)
    d = info.as_dict()
    d["status"] = st
    return e, d


def tbsci_overlap(ctx, A, B, stream=None) -> np.ndarray:
    """S[i, j] = <A_i | B_j> for FP64 device tensors A [ma, ...] and B [mb, ...]
    with the same number of elements per vector; returns a numpy [ma, mb]."""
    ma, mb = int(A.shape[0]), int(B.shape[0])
    na = A.numel() // ma if ma else None
    nb = B.numel() // mb if mb else None
    assert na is None or nb is None or na == nb, "vectors of different length"
    n = int(na if na is not None else (nb or 0))
    S = np.zeros((ma, mb))
    _check(ctx, load().tbsci_overlap(ctx, _ptr(A), ma, _ptr(B), mb, n, _ptr(S), _stream(stream)))
    return S


# ---------------------------------------------------------------- serving

def tbsci_server_create(device=0, hbm_budget=0, max_active=0, max_queue=0, fuse_sigma=0, fail_admission_at=0,
                        tune_cache=None):
    o = ServerOpts(device, hbm_budget, max_active, max_queue, fuse_sigma, fail_admission_at,
                   None if tune_cache is None else os.fsencode(tune_cache))
    out = ctypes.c_void_p()
    st = load().tbsci_server_create(ctypes.byref(o), ctypes.byref(out))
    if st != TBSCI_OK:
        raise TbsciError(st, "tbsci_server_create failed")
    return out


def tbsci_submit(srv, norb, nalpha, nbeta, h, eri, ecore=0.0, alpha=None, beta=None, nroots=1, mixed=False,
                 tol_energy=0.0, tol_residual=0.0, max_iter=0):
    """Queues one solve; returns ``(status, ticket)`` (status EAGAIN when the queue is full).
    ``mixed``: False / 0 FP64, True / 1 FP32 sigma, 2 split-TF32 and 3 BF16
    tensor-core sigma, each then FP64 refinement."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.uint64)
    b = None if beta is None else np.ascontiguousarray(beta, dtype=np.uint64)
    r = Request(norb, nalpha, nbeta, h.ctypes.data, eri.ctypes.data, float(ecore),
                None if a is None else a.ctypes.data, 0 if a is None else len(a),
                None if b is None else b.ctypes.data, 0 if b is None else len(b),
                nroots, int(mixed), tol_energy, tol_residual, max_iter)
    t = ctypes.c_uint64()
    st = load().tbsci_submit(srv, ctypes.byref(r), ctypes.byref(t))
    return st, t.value


def tbsci_poll(srv, ticket, timeout_ms=-1):
    """``(status, result dict or None)``; status ETIMEOUT when not finished in time."""
    res = Result()
    st = load().tbsci_poll(srv, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(res))
    return st, (res.as_dict() if st == TBSCI_OK else None)


def tbsci_server_load(srv):
    q, a = ctypes.c_int(), ctypes.c_int()
    load().tbsci_server_load(srv, ctypes.byref(q), ctypes.byref(a))
    return q.value, a.value


def tbsci_server_destroy(srv):
    load().tbsci_server_destroy(srv)
