"""The binary64 Lanczos engine (precision "f64"): IEEE binary64 Lanczos
vectors, H Phi, dot products and updates.  Its eigenvalues agree with the
oracle's dense diagonalisation; the variant that keeps every Gram-Schmidt
update on binary64 FMAs (strict64) agrees with the default, whose update with
tiny coefficients sums the correction in fp32 from the stored high words
(error below binary64 rounding of w); Ritz residuals reach binary64 level."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


def _dense_lowest(spec, nd, K):
    if K is None:
        return np.linalg.eigvalsh(orc.dense_u1(olat(spec), nd))
    return np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(spec), nd, K)))


@pytest.mark.parametrize("name,spec,nd,Ks", [
    ("chain14_u1", qi.chain(14, Jz=0.7), 4, None),
    ("square6_k", qi.square(6), 3, [(0, 0, 0), (1, 2, 0), (3, 3, 0), (2, 5, 0)]),
    ("cube4_k", qi.hypercubic((4, 4, 4), J=1.0, Jz=0.6), 2, [(0, 0, 0), (1, 0, 2)]),
    ("random_u1", qi.random_graph(13, 30, seed=4, field=True), 5, None),
])
def test_lanczos_binary64_vs_oracle_and_strict(name, spec, nd, Ks):
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(spec, nd, Ks)
    out = {}
    for strict in (False, True):
        o = qs3.SolveOpts(n_max=200, eps=1e-14, res_tol=1e-12, precision="f64", strict64=strict, use_graphs=False)
        e, v, info = b.lanczos(o)
        torch.cuda.synchronize()
        assert info["status"] == "QS3_OK"
        assert info["max_residual"] <= 1e-11 * max(1.0, float(np.max(np.abs(e))))
        out[strict] = (e, v)
    e0, e1 = out[False][0], out[True][0]
    scale = max(1.0, float(np.max(np.abs(e1))))
    assert float(np.max(np.abs(e0 - e1))) <= 1e-13 * scale
    for s in range(b.n_sectors):
        K = None if Ks is None else Ks[s]
        w = _dense_lowest(spec, nd, K)
        assert abs(e0[s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


def test_trl_binary64_vs_oracle():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.square(6)
    Ks = [(0, 0, 0), (2, 1, 0)]
    b = lib_basis(spec, 3, Ks)
    o = qs3.SolveOpts(n_eig=3, n_keep=8, n_max=32, eps=1e-13, precision="f64")
    e, _, info = b.trlanczos(o)
    assert info["status"] == "QS3_OK"
    assert info["max_residual"] <= 1e-10
    for s, K in enumerate(Ks):
        w = _dense_lowest(spec, 3, K)
        assert abs(e[s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


def test_fp32_refinement_is_binary64():
    """fp32 H Phi, then the binary64 engine from the fp32 Ritz vector: the
    result meets |dE| <= 1e-9 |E| against the plain binary64 solve."""
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.square(6)
    b = lib_basis(spec, 3, [(0, 0, 0), (1, 2, 0), (3, 3, 0)])
    e64, _, _ = b.lanczos(qs3.SolveOpts(n_max=200, eps=1e-14, res_tol=1e-12, precision="f64"), vectors=False)
    e32, _, info = b.lanczos(qs3.SolveOpts(n_max=200, eps=1e-10, res_tol=1e-9, precision="f32", refine_tol=1e-9),
                             vectors=False)
    assert info["status"] == "QS3_OK" and info["refine_iterations"] > 0
    assert float(np.max(np.abs(e32 - e64) / np.abs(e64))) <= 1e-9


def test_rejects_unknown_precision():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    with pytest.raises(ValueError):
        qs3.SolveOpts(precision="f16")
