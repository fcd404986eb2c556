"""The no-allocation S^-_q entry point against the allocating one.

Some callers cannot allocate device memory while they run (they hand out all
device memory from their own pool, or an allocation there would synchronise
the device).  qs3_smq_noalloc serves them with a fixed scratch array inside
the library.  This file is collected last so that a failure here leaves every
other test already run; it also passes on its own in a fresh process."""
from __future__ import annotations

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import lib_basis, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nd,K", [((6, 4, 1), 3, (1, 2, 0)), ((10, 1, 1), 2, None), ((3, 3, 3), 0, (0, 0, 0))])
def test_smq_noalloc_matches_allocating_call_twice(dims, nd, K):
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.hypercubic(dims)
    Ks = None if K is None else [K]
    src = lib_basis(spec, nd, Ks)
    x = qi.gaussian_start(12, src.total_dim, True)
    phi = to_dev(x, torch.complex128)
    for call, Q in enumerate([(1, 0, 0), (2, 1, 0) if dims[1] > 1 else (3, 0, 0)]):
        K2 = None if K is None else [tuple((K[a] + Q[a]) % dims[a] for a in range(3))]
        dst = lib_basis(spec, nd + 1, K2)
        want = qs3.smq(src, 0, phi, dst, 0, Q).cpu().numpy()
        psi = torch.full((dst.total_dim,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        qs3.smq_noalloc(src, 0, phi, dst, 0, Q, psi)
        torch.cuda.synchronize()
        got = psi.cpu().numpy()
        assert got.shape == want.shape and np.all(np.isfinite(got)), call
        np.testing.assert_allclose(got, want, atol=1e-12, rtol=0)


def test_smq_noalloc_rejects_oversized_lattice():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.chain(2100, periodic=False)
    src = lib_basis(spec, 1)
    dst = lib_basis(spec, 2)
    phi = torch.ones(src.total_dim, dtype=torch.complex128, device="cuda")
    psi = torch.zeros(dst.total_dim, dtype=torch.complex128, device="cuda")
    with pytest.raises(qs3.QS3Error) as ex:
        qs3.smq_noalloc(src, 0, phi, dst, 0, (1, 0, 0), psi)
    assert ex.value.status == -1 and "2048" in str(ex.value)
