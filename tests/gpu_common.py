"""Helpers of the GPU parity tests (the CUDA path against the oracle)."""
from __future__ import annotations

import numpy as np

import oracle as orc
import qs3_inputs as qi


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def lib_basis(spec, nd, K=None):
    import paper_2107_00872_gb300 as qs3
    return qs3.Basis(spec, nd, K)


def olat(spec) -> orc.Lattice:
    return orc.Lattice(**spec.as_dict())


def to_dev(x: np.ndarray, dtype):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def tol_hphi(phi: np.ndarray, fp32: bool, row_weight: float = 16.0) -> float:
    """Element-wise bound for |psi_gpu - psi_oracle|: fp64 keeps the product
    within 1e-12 |phi| (spec bound, scaled by the largest row weight of
    H, at most ~16 here); fp32 rows accumulate up to ~30 terms in fp32 with
    fp32 matrix elements, so 2e-6 |phi|_inf per unit row weight."""
    m = float(np.max(np.abs(phi))) if phi.size else 1.0
    return (2e-6 if fp32 else 1e-12) * m * row_weight


def gaussian(seed, d, complex_):
    return qi.gaussian_start(seed, d, complex_)
