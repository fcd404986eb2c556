"""The representative table of k-sector H Phi (qs3_basis_rep_table): the
tabulated representative search must give exactly the same H Phi as the
search of Alg. 7 it replaces, on lattices with non-trivial stabilisers and at
the full size of the 10x10, N_down = 4 workload, and both against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, tol_hphi, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    # (name, dims, N_down): chains whose N_down divides N have periodic states
    ("chain12_nd3", (12, 1, 1), 3),
    ("chain8_nd4", (8, 1, 1), 4),
    ("square4_nd4", (4, 4, 1), 4),
    ("square6x4_nd3", (6, 4, 1), 3),
    ("cube3_nd3", (3, 3, 3), 3),
    ("cube4x3x2_nd2", (4, 3, 2), 2),
]


def _hphi_both(b, phi):
    torch = torch_cuda()
    assert b.rep_table(-1), "the table is built by default for small lattices"
    with_table = b.hphi(phi)
    b.rep_table(0)
    assert not b.rep_table(-1)
    search = b.hphi(phi)
    assert b.rep_table(1)
    again = b.hphi(phi)
    torch.cuda.synchronize()
    return with_table, search, again


@pytest.mark.parametrize("name,dims,nd", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_table_equals_search(name, dims, nd, dt):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=0.7)
    K = qi.all_k(dims)
    b = lib_basis(spec, nd, K)
    phi_h = gaussian(11, b.total_dim, True)
    phi = to_dev(phi_h, torch.complex128 if dt == "c128" else torch.complex64)
    t, s, t2 = _hphi_both(b, phi)
    # same terms, same order, same arithmetic: identical bits
    assert torch.equal(t, s)
    assert torch.equal(t, t2)
    # and the oracle's Alg. 9 on every sector
    out = t.cpu().numpy().astype(np.complex128)
    for i, k in enumerate(K):
        sec = orc.mk_list(olat(spec), nd, k)
        lo, hi = b.offsets[i], b.offsets[i + 1]
        ref = orc.hphi_k(sec, phi_h[lo:hi])
        tol = tol_hphi(phi_h[lo:hi], dt == "c64")
        assert np.max(np.abs(out[lo:hi] - ref), initial=0.0) <= tol, (name, k)


def test_table_full_size_square10_nd4():
    torch = torch_cuda()
    spec = qi.square(10)
    b = lib_basis(spec, 4, qi.all_k((10, 10, 1)))
    assert b.total_dim == 3921225
    phi = to_dev(gaussian(5, b.total_dim, True), torch.complex128)
    t, s, _ = _hphi_both(b, phi)
    assert torch.equal(t, s)


def test_table_errors():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    u1 = lib_basis(qi.chain(10), 3)
    assert not u1.rep_table(-1)
    with pytest.raises(qs3.QS3Error):
        u1.rep_table(1)
    kb = lib_basis(qi.chain(10), 3, [(0, 0, 0)])
    with pytest.raises(qs3.QS3Error):
        kb.rep_table(2)
    assert kb.rep_table(-1)
