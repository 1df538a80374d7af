"""GB300 TBSCI: sigma = H.c over a tensor-product bitstring space and the
Davidson solver that drives it (arXiv 2503.10335, Sec. II), on one GPU.

The compute path is libtbsci.so (CUDA for sm_103a, C ABI in include/tbsci.h);
this package only marshals arguments to it. ``Space`` bundles the handles of
one problem (strings, link tables, Hamiltonian) for convenience.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B

# the C entry points (same names) and status / dtype constants
for _n in dir(B):
    if _n.startswith(("tbsci_", "TBSCI_")):
        globals()[_n] = getattr(B, _n)
del _n

__all__ = ["Context", "Space", "Pruned", "Server", "B"] + [n for n in dir(B) if n.startswith(("tbsci_", "TBSCI_"))]


class Context:
    """A libtbsci context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, default_mixed: int = 0, tune_cache=None):
        if hbm_budget or default_mixed or tune_cache is not None:
            self.handle = B.tbsci_create_ex(device, hbm_budget, default_mixed, tune_cache)
        else:
            self.handle = B.tbsci_create(device)
        self.device = device

    def close(self):
        if self.handle is not None:
            B.tbsci_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Space:
    """One TPB problem: alpha/beta string sets (selected or full), their link
    tables, and a Hamiltonian. ``alpha`` / ``beta``: host uint64 arrays or None
    for the full string space."""

    def __init__(self, ctx: Context, norb, nalpha, nbeta, h, eri, ecore=0.0, alpha=None, beta=None,
                 prepare=True):
        self.ctx = ctx
        c = ctx.handle
        self.norb, self.nalpha, self.nbeta = int(norb), int(nalpha), int(nbeta)
        self._handles = []
        try:
            self._build(c, norb, nalpha, nbeta, h, eri, ecore, alpha, beta, prepare)
        except Exception:
            self.close()  # frees what was made before the failing call
            raise

    def _build(self, c, norb, nalpha, nbeta, h, eri, ecore, alpha, beta, prepare):
        self.sa = B.tbsci_build_strings(c, norb, nalpha, alpha)
        self._handles.append((B.tbsci_strings_destroy, self.sa))
        self.sb = B.tbsci_build_strings(c, norb, nbeta, beta)
        self._handles.append((B.tbsci_strings_destroy, self.sb))
        self.ta = B.tbsci_build_excitation_tables(c, self.sa, 0)
        self._handles.append((B.tbsci_tables_destroy, self.ta))
        self.tb = B.tbsci_build_excitation_tables(c, self.sb, 0)
        self._handles.append((B.tbsci_tables_destroy, self.tb))
        self.ham = B.tbsci_hamiltonian_create(c, h, eri, ecore)
        self._handles.append((B.tbsci_hamiltonian_destroy, self.ham))
        self.la = B.tbsci_strings_count(self.sa)
        self.lb = B.tbsci_strings_count(self.sb)
        self.ndet = self.la * self.lb
        if prepare:
            B.tbsci_prepare(c, self.ham, self.ta, self.tb)

    def strings(self):
        return B.tbsci_strings_export(self.ctx.handle, self.sa), B.tbsci_strings_export(self.ctx.handle, self.sb)

    def sigma(self, c, out=None, stream=None, dtype=None):
        """sigma = H c for a device tensor ``c`` [nvec, la, lb]: float64 -> TBSCI_F64,
        float32 -> TBSCI_F32 unless ``dtype`` names a tensor-core mode
        (TBSCI_F32_TC_TF32 / TBSCI_F32_TC_BF16, float32 tensors)."""
        import torch
        nvec = c.shape[0] if c.dim() == 3 else 1
        assert c.is_cuda and c.is_contiguous() and c.numel() == nvec * self.ndet
        if out is None:
            out = torch.empty_like(c)
        if dtype is None:
            dtype = B.TBSCI_F64 if c.dtype == torch.float64 else B.TBSCI_F32
        assert (c.dtype == torch.float64) == (dtype == B.TBSCI_F64)
        B.tbsci_sigma(self.ctx.handle, self.ham, self.ta, self.tb, c, out, nvec, dtype, stream)
        return out

    def sigma_host(self, c: np.ndarray) -> np.ndarray:
        c = np.ascontiguousarray(c, dtype=np.float64)
        nvec = c.shape[0] if c.ndim == 3 else 1
        out = np.empty_like(c)
        B.tbsci_sigma_host(self.ctx.handle, self.ham, self.ta, self.tb, c, out, nvec)
        return out

    def diagonal(self, stream=None):
        import torch
        d = torch.empty(self.ndet, dtype=torch.float64, device="cuda:%d" % self.ctx.device)
        B.tbsci_diagonal(self.ctx.handle, self.ham, self.ta, self.tb, d, stream)
        return d

    def counts(self) -> dict:
        return B.tbsci_sigma_counts_get(self.ctx.handle, self.ham, self.ta, self.tb)

    def davidson(self, nroots, want_vectors=False, **kw):
        import torch
        vecs = None
        if want_vectors:
            vecs = torch.empty((nroots, self.la, self.lb), dtype=torch.float64,
                               device="cuda:%d" % self.ctx.device)
        e, info = B.tbsci_davidson(self.ctx.handle, self.ham, self.ta, self.tb, nroots, vecs=vecs, **kw)
        return (e, info, vecs) if want_vectors else (e, info)

    def string_weights(self, c):
        """(W_a, W_b) of the FP64 device vector c [la, lb] (Sec. III.B)."""
        return B.tbsci_string_weights(self.ctx.handle, self.ta, self.tb, c, self.la, self.lb)

    def select_by_weight(self, c, delta):
        """The alpha and beta strings whose weight in c is at least delta times the
        largest (the HF string's) weight (Sec. III.B): the next space's strings."""
        return B.tbsci_select_by_weight(self.ctx.handle, self.ta, self.tb, c, delta, self.la, self.lb)

    def coefficient_histogram(self, c, c_hf, lo=-12, hi=0, per_decade=1):
        """Counts of |c_K / c_HF| per logarithmic bin from 10^lo to 10^hi (Fig. 3):
        returns (bin edges of the ratio, counts incl. the under- and overflow bins)."""
        ratios = 10.0 ** (np.arange(lo * per_decade, hi * per_decade + 1) / per_decade)
        counts = B.tbsci_coefficient_histogram(self.ctx.handle, c, ratios * abs(float(c_hf)))
        return ratios, counts

    def prune(self, off, cols):
        """The pruned space D_TBSCI of this space: per alpha string w the ascending
        beta indices cols[off[w]:off[w + 1]]."""
        return Pruned(self, off, cols)

    def symmetry_block(self, orb_irrep, target):
        """The determinants of irrep ``target`` (abelian point group, labels 0..7)."""
        return Pruned(self, None, None, handle=B.tbsci_pruned_create_symmetry(self.ctx.handle, self.ta, self.tb,
                                                                              orb_irrep, target))

    def close(self):
        for fn, h in reversed(self._handles):
            fn(h)
        self._handles = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pruned:
    """A pruned TBSCI space inside a ``Space`` (compressed vectors [nvec, ndet])."""

    def __init__(self, space: Space, off, cols, handle=None):
        self.space = space
        self.handle = handle if handle is not None else B.tbsci_pruned_create(space.ctx.handle, space.ta, space.tb,
                                                                               off, cols)
        self.ndet = B.tbsci_pruned_count(self.handle)

    def sigma(self, c, out=None, stream=None, dtype=None):
        import torch
        nvec = c.shape[0] if c.dim() == 2 else 1
        assert c.is_cuda and c.is_contiguous() and c.numel() == nvec * self.ndet
        if out is None:
            out = torch.empty_like(c)
        if dtype is None:
            dtype = B.TBSCI_F64 if c.dtype == torch.float64 else B.TBSCI_F32
        sp = self.space
        B.tbsci_sigma_pruned(sp.ctx.handle, sp.ham, sp.ta, sp.tb, self.handle, c, out, nvec, dtype, stream)
        return out

    def diagonal(self, stream=None):
        import torch
        sp = self.space
        d = torch.empty(self.ndet, dtype=torch.float64, device="cuda:%d" % sp.ctx.device)
        B.tbsci_diagonal_pruned(sp.ctx.handle, sp.ham, sp.ta, sp.tb, self.handle, d, stream)
        return d

    def davidson(self, nroots, want_vectors=False, **kw):
        import torch
        sp = self.space
        vecs = None
        if want_vectors:
            vecs = torch.empty((nroots, self.ndet), dtype=torch.float64, device="cuda:%d" % sp.ctx.device)
        e, info = B.tbsci_davidson_pruned(sp.ctx.handle, sp.ham, sp.ta, sp.tb, self.handle, nroots, vecs=vecs, **kw)
        return (e, info, vecs) if want_vectors else (e, info)

    def close(self):
        if self.handle is not None:
            B.tbsci_pruned_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (tbsci_server_*): submit solves from any thread, poll results."""

    def __init__(self, device=0, hbm_budget=0, max_active=0, max_queue=0, fuse_sigma=0, fail_admission_at=0,
                 tune_cache=None):
        self.handle = B.tbsci_server_create(device, hbm_budget, max_active, max_queue, fuse_sigma,
                                            fail_admission_at, tune_cache)

    def submit(self, norb, nalpha, nbeta, h, eri, ecore=0.0, alpha=None, beta=None, nroots=1, mixed=False, **kw):
        st, ticket = B.tbsci_submit(self.handle, norb, nalpha, nbeta, h, eri, ecore, alpha, beta, nroots, mixed, **kw)
        if st != B.TBSCI_OK:
            raise B.TbsciError(st, "tbsci_submit")
        return ticket

    def poll(self, ticket, timeout_ms=-1):
        return B.tbsci_poll(self.handle, ticket, timeout_ms)

    def load(self):
        return B.tbsci_server_load(self.handle)

    def close(self):
        if self.handle is not None:
            B.tbsci_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
