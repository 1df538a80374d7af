"""Shared helpers of the GPU parity tests (comparison rules, fixtures' data)."""
import numpy as np


def assert_sigma_close(s_gpu, s_ref, bound, rel=1e-12, norm_rel=1e-12):
    """Elementwise |d| <= rel * (|H||c|)_I + 1e-300 and normwise
    ||d|| <= norm_rel * ||sigma_ref|| (summation order differs, so sigma is not
    compared bit for bit)."""
    s_gpu = np.asarray(s_gpu).reshape(s_ref.shape)
    d = np.abs(s_gpu - s_ref)
    ratio = d / (bound + 1e-300)
    worst = float(ratio.max()) if ratio.size else 0.0
    assert np.all(d <= rel * bound + 1e-300), "elementwise: worst |d|/(|H||c|) = %.3e" % worst
    nr = np.linalg.norm(s_ref)
    if nr > 0:
        assert np.linalg.norm(s_gpu - s_ref) <= norm_rel * nr, "normwise %.3e" % (np.linalg.norm(s_gpu - s_ref) / nr)
    return worst
