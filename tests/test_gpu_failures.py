"""Failure paths on the GPU without a GPU fault: an allocation failure
injected on the host (qs3_inject_alloc_failure) at every allocation of a
basis build and of a solve returns QS3_ERR_OOM, releases what the call had
allocated, and leaves the library usable: the same solve succeeds right after
with the same result."""
from __future__ import annotations

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import torch_cuda

pytestmark = pytest.mark.gpu

OOM = -4


@pytest.mark.parametrize("prec", ["f64", "f32", "df"])
def test_injected_oom_at_every_allocation(prec):
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.square(4)
    Ks = [(0, 0, 0), (1, 2, 0)]
    o = qs3.SolveOpts(n_max=60, eps=1e-12, res_tol=1e-10, precision=prec)
    ref, _, _ = qs3.Basis(spec, 3, Ks).lanczos(o)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fails = 0
    for after in range(400):
        qs3.inject_alloc_failure(after)
        try:
            b = qs3.Basis(spec, 3, Ks)
            e, _, _ = b.lanczos(o)
        except qs3.QS3Error as err:
            assert err.status == OOM, err
            fails += 1
            continue
        finally:
            qs3.inject_alloc_failure(-1)
        np.testing.assert_array_equal(e, ref)
        break
    else:
        pytest.fail("the solve never completed")
    assert fails > 5
    torch.cuda.synchronize()
    # nothing leaked beyond allocator granularity
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    e, _, info = qs3.Basis(spec, 3, Ks).lanczos(o)
    np.testing.assert_array_equal(e, ref)
