"""The bounded waits of the copy-ring dot pass (k_dotb).  With the host-side
injection qs3_inject_wait_timeout its copy warp issues no copies: every
consumer warp's wait on its first stage gives up after one second, the
kernel sets the error flag, writes zero partials for the vectors it could
not multiply and returns, and the call reports QS3_ERR_TIMEOUT.  No fault,
trap or endless wait is involved: the context stays usable and the next
calls give the same bits as before the injection."""
from __future__ import annotations

import time

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TIMEOUT = -7


def test_gs_dots_wait_timeout():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.square(6), 3, [(0, 0, 0), (1, 0, 0)])
    b.tuning(dot_vectors64=8)
    D = b.total_dim
    V = np.stack([gaussian(20 + j, D, True) for j in range(4)])
    w = gaussian(30, D, True)
    Vd, wd = to_dev(V, torch.complex128), to_dev(w, torch.complex128)
    ref = b.gs_dots(Vd, wd)
    assert qs3.inject_wait_timeout(1) == 0
    t0 = time.perf_counter()
    with pytest.raises(qs3.QS3Error) as ei:
        b.gs_dots(Vd, wd)
    assert ei.value.status == TIMEOUT
    assert time.perf_counter() - t0 < 60
    assert qs3.inject_wait_timeout(0) == 0          # the injection was used
    np.testing.assert_array_equal(b.gs_dots(Vd, wd), ref)


def test_solve_wait_timeout():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.square(6), 3, [(0, 0, 0)])
    b.tuning(dot_vectors64=8)
    o = qs3.SolveOpts(n_max=40, eps=1e-14, res_tol=1e-12, use_graphs=False, precision="f64")
    e_ref, _, _ = b.lanczos(o, vectors=False)
    qs3.inject_wait_timeout(1)
    with pytest.raises(qs3.QS3Error) as ei:
        b.lanczos(o, vectors=False)
    assert ei.value.status == TIMEOUT
    assert qs3.inject_wait_timeout(0) == 0
    e, _, _ = b.lanczos(o, vectors=False)
    np.testing.assert_array_equal(e, e_ref)
