"""The 10x10x10 cube at N_down = 4 (41.4 M rows per momentum sector; Sec.
"Energy-dispersion relation", Alg. 10): thick-restart Lanczos on Gamma and a
generic momentum of the k-path with the stored-term H Phi, fp32 H Phi +
fp64 recurrences + binary64 refinement.  The oracle cannot solve these
sectors; they are pinned by the binary64 residual |H v - E v| <= 1e-9 |E| of
every returned pair (the oracle's sampled rows of the same product are
compared in test_gpu_fullsize.py), by agreement with the plain binary64 run
at Gamma, and by SU(2): the isotropic model's N_down = 4 sector contains every
N_down = 3 level of the same momentum, so its lowest level is not above the
N_down = 3 one."""
from __future__ import annotations

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import lib_basis, torch_cuda

pytestmark = pytest.mark.gpu


def test_cubic10_nd4_trl_gamma_and_generic_k():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.cubic(10)
    Ks = [(0, 0, 0), (1, 0, 0)]
    b = lib_basis(spec, 4, Ks)
    assert b.dims == [41_417_998, 41_417_000]
    b.store_terms(1)
    o = qs3.SolveOpts(n_eig=2, n_keep=8, n_max=32, max_iter=4000, eps=1e-10, precision="f32", refine_tol=1e-9,
                      seed=11)
    e, v, info = b.trlanczos(o, vectors=False)
    assert info["status"] == "QS3_OK" and info["refine_iterations"] > 0
    assert info["max_residual"] <= 1e-9 * float(np.max(np.abs(e)))
    # plain binary64 at Gamma only
    g = lib_basis(spec, 4, Ks[:1])
    g.store_terms(1)
    e64, _, i64 = g.trlanczos(qs3.SolveOpts(n_eig=2, n_keep=8, n_max=32, max_iter=4000, eps=1e-10, seed=11),
                              vectors=False)
    assert i64["status"] == "QS3_OK"
    assert abs(e[0, 0] - e64[0, 0]) <= 1e-9 * abs(e64[0, 0])
    # SU(2): the lowest N_down = 4 level lies at or below the N_down = 3 one (same K)
    b3 = lib_basis(spec, 3, Ks)
    e3, _, i3 = b3.trlanczos(qs3.SolveOpts(n_eig=1, n_keep=8, n_max=32, max_iter=4000, eps=1e-12, seed=3),
                             vectors=False)
    assert i3["status"] == "QS3_OK"
    assert np.all(e[:, 0] <= e3[:, 0] + 1e-9 * np.abs(e3[:, 0]))
