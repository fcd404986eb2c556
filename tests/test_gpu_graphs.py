"""CUDA-graph replay of the fp64 Lanczos step (qs3_solve_opts.use_graphs):
the replayed step runs the same kernels with the step index read on the
device, so eigenvalues, iteration counts and vectors must be identical to the
directly launched solve, for Lanczos, thick-restart Lanczos and the batch
solver (whose worker threads capture concurrently)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


def _opts(graphs, **kw):
    import paper_2107_00872_gb300 as qs3
    base = dict(n_max=120, eps=1e-14, res_tol=1e-12)
    base.setdefault("precision", "f64")
    base.update(kw)
    return qs3.SolveOpts(use_graphs=graphs, **base)


@pytest.mark.parametrize("prec", ["f64", "df"])
@pytest.mark.parametrize("name,spec,nd,K", [
    ("chain16_u1", qi.chain(16), 3, None),
    ("square6_k", qi.square(6), 3, [(0, 0, 0), (1, 2, 0), (3, 3, 0)]),
    ("cube4_k", qi.hypercubic((4, 4, 4), J=1.0, Jz=0.6), 2, [(0, 0, 0), (1, 0, 2)]),
])
def test_lanczos_graphs_identical(name, spec, nd, K, prec):
    torch = torch_cuda()
    b = lib_basis(spec, nd, K)
    e0, v0, i0 = b.lanczos(_opts(False, precision=prec))
    e1, v1, i1 = b.lanczos(_opts(True, precision=prec))
    torch.cuda.synchronize()
    assert i0["status"] == i1["status"] == "QS3_OK"
    assert i1["hphi_graph_calls"] > 0 and i0["hphi_graph_calls"] == 0
    assert i0["iterations"] == i1["iterations"]
    np.testing.assert_array_equal(e0, e1)
    assert torch.equal(v0, v1)
    # and the oracle's dense spectrum
    for s in range(b.n_sectors):
        if K is None:
            w = np.linalg.eigvalsh(orc.dense_u1(olat(spec), nd))
        else:
            w = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(spec), nd, K[s])))
        assert abs(e1[s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


@pytest.mark.parametrize("prec", ["f64", "df"])
def test_trl_graphs_identical(prec):
    torch = torch_cuda()
    spec = qi.square(6)
    b = lib_basis(spec, 3, [(0, 0, 0), (2, 1, 0)])
    kw = dict(n_eig=3, n_keep=6, n_max=24, eps=1e-12, precision=prec)
    e0, v0, i0 = b.trlanczos(_opts(False, **kw))
    e1, v1, i1 = b.trlanczos(_opts(True, **kw))
    torch.cuda.synchronize()
    assert i1["hphi_graph_calls"] > 0
    assert i0["iterations"] == i1["iterations"] and i0["restarts"] == i1["restarts"]
    np.testing.assert_array_equal(e0, e1)
    assert torch.equal(v0, v1)


def test_batch_graphs_identical():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    bases = [lib_basis(qi.chain(n), 3) for n in (12, 13, 14, 15, 16, 17)]
    bases += [lib_basis(qi.square(5), 3, [(1, 0, 0)]), lib_basis(qi.square(4), 4, [(0, 0, 0)])]
    ev0, inf0, st0 = qs3.batch_solve(bases, _opts(False), max_concurrent=4)
    ev1, inf1, st1 = qs3.batch_solve(bases, _opts(True), max_concurrent=4)
    assert st0 == st1 == "QS3_OK"
    for a, b_, i0, i1 in zip(ev0, ev1, inf0, inf1):
        np.testing.assert_array_equal(a, b_)
        assert i0["iterations"] == i1["iterations"]
