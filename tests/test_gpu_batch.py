"""GPU parity of the batched uneven-instance solver: many independent bases
(chains, squares, cubes, with and without momentum, different N_down and
anisotropy) solved concurrently, against the oracle's dense matrices and
against the same instances solved one by one."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


def _instances():
    """Small seeded uneven mix (dimensions 20..~2000) the oracle can diagonalise."""
    rng = np.random.default_rng(77)
    out = []
    specs = [((12, 1, 1), 3), ((10, 1, 1), 4), ((4, 4, 1), 3), ((5, 4, 1), 3), ((3, 3, 3), 2), ((3, 3, 2), 3),
             ((14, 1, 1), 2), ((6, 5, 1), 2), ((4, 3, 1), 4), ((16, 1, 1), 3)]
    for i, (dims, nd) in enumerate(specs):
        delta = float(rng.uniform(0.5, 1.5))
        spec = qi.hypercubic(dims, J=1.0, Jz=delta)
        K = None
        if i % 2 == 1:
            K = tuple(int(rng.integers(0, dims[a])) for a in range(3))
        out.append((spec, nd, K))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_solve_uneven_instances(prec):
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    inst = _instances()
    bases = [lib_basis(spec, nd, None if K is None else [K]) for spec, nd, K in inst]
    opts = qs3.SolveOpts(n_max=200, eps=1e-14, res_tol=1e-11, precision=prec, refine_tol=1e-9)
    ev, infos, status = qs3.batch_solve(bases, opts, max_concurrent=4)
    assert status == "QS3_OK", (status, infos)
    for (spec, nd, K), e, info in zip(inst, ev, infos):
        if K is None:
            w = np.linalg.eigvalsh(orc.dense_u1(olat(spec), nd))
        else:
            sec = orc.mk_list(olat(spec), nd, K)
            w = np.linalg.eigvalsh(orc.dense_k(sec))
        tol = 1e-11 if prec == "f64" else 1e-9
        assert abs(e[0] - w[0]) <= tol * max(1.0, abs(w[0])), (spec.name, nd, K, e[0], w[0])
    # the same instances one by one give the same eigenvalues
    for b, e in zip(bases[:4], ev[:4]):
        e1, _, _ = b.lanczos(opts, vectors=False)
        assert abs(e1[0, 0] - e[0]) <= 1e-12 * max(1.0, abs(e[0]))


def test_batch_solve_reports_errors():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.chain(8), 2)
    with pytest.raises(qs3.QS3Error):
        qs3.batch_solve([b], qs3.SolveOpts(n_max=1))
