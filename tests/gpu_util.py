"""Helpers for the GPU parity tests."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def rel_err(got, ref, floor=1e-3):
    """max |got - ref| / max(|ref|, floor): the relative error with a floor for
    kernel values near 0 (straight lines with <a,b> < 0 give J_0, which can
    cross 0)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()
