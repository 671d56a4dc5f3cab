"""Shared helpers of the GPU tests: mechanism handles, state transfer and
the error measures the parity bars are written in."""
import os

import numpy as np
import pytest

from paper_2411_02640_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.environ.get("KX_CACHE_DIR", os.path.join(ROOT, ".kxcache"))
MECHDIR = os.path.join(ROOT, ".kxcache", "mech")

_handles = {}


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def mechanism(name, **opts):
    from paper_2411_02640_gb300 import kx
    key = (name, tuple(sorted(opts.items())))
    if key not in _handles:
        path = synth.mechanism_file(name, MECHDIR)
        _handles[key] = kx.Mechanism(path, cache_dir=CACHE, **opts)
    return _handles[key]


def oracle(name, nthreads=None):
    import oracle as ora
    return ora.Oracle(synth.mechanism_file(name, MECHDIR), nthreads=nthreads or min(16, os.cpu_count() or 1))


def to_device(torch, T, p, Y, ld=None):
    n = T.shape[0]
    ld = ld or n
    Td = torch.tensor(T, dtype=torch.float64, device="cuda")
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    Yd = torch.zeros((Y.shape[0], ld), dtype=torch.float64, device="cuda")
    Yd[:, :n] = torch.tensor(Y, dtype=torch.float64, device="cuda")
    return Td, pd, Yd


def wdot_error(W, w_gpu, w_ora):
    """Per point: max_k W_k |dw_k| / max_k W_k |w_k| (the per-point scale)."""
    num = np.max(W[:, None] * np.abs(w_gpu - w_ora), axis=0)
    den = np.max(W[:, None] * np.abs(w_ora), axis=0)
    return num / np.where(den > 0, den, 1.0)
