"""Helpers for the GPU parity tests (CUDA path vs oracle)."""
from __future__ import annotations

import numpy as np


def require_cuda():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_err(gpu, ref, mask, floor_rel=1.0):
    """Per-voxel error measure of the parity rule: |g - r| / max(|r|, s_v), s_v = max_v |r_v|."""
    g = gpu[:, mask]
    r = ref[:, mask]
    s = np.max(np.abs(r), axis=1, keepdims=True) * floor_rel
    s = np.where(s == 0, 1.0, s)
    return np.abs(g - r) / np.maximum(np.abs(r), s)


def assert_parity(gpu, ref, mask, tol=1e-12, what=""):
    e = rel_err(gpu, ref, mask)
    worst = float(e.max()) if e.size else 0.0
    assert np.all(np.isfinite(gpu[:, mask])), f"{what}: non-finite GPU values"
    assert worst <= tol, f"{what}: max relative error {worst:.3e} > {tol:.1e}"
    return worst
