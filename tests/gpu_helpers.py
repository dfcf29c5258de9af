"""Shared helpers of the GPU parity tests: layout conversion between the CUDA
library's row-grouped block storage and the oracle's column layout, and the
block error metric (max over blocks of |dB|_max / |B_ref|_max)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA GPU not available")
    return torch


def to_oracle_layout(vals, recv, nt):
    """vals[R, slot] (R = receiving row, slot = source face among the 3 others)
    -> blocks[J = 4t+f, k] (k-th destination face f' != f ascending)."""
    vals = np.asarray(vals, dtype=np.float64)
    t = np.repeat(np.arange(nt), 12)
    f = np.tile(np.repeat(np.arange(4), 3), nt)
    fp = np.tile(np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]).reshape(-1), nt)
    R = recv[4 * t + fp]
    slot = f - (f > fp)
    return vals[R, slot].reshape(4 * nt, 3, vals.shape[2], vals.shape[3])


def block_rel_err(a, b):
    a = np.asarray(a).reshape(-1, a.shape[-2] * a.shape[-1])
    b = np.asarray(b).reshape(-1, b.shape[-2] * b.shape[-1])
    den = np.abs(b).max(axis=1)
    return np.abs(a - b).max(axis=1) / den
