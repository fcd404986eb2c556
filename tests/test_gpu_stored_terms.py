"""Stored-term H Phi (qs3_basis_store_terms): the enumerated terms replayed as
a gather SpMV must give the matrix-free product bit for bit in complex128
(same terms, order and arithmetic), whether they were enumerated through the
representative table or the representative search, and agree with the
oracle's Alg. 9; solvers on a basis with stored terms return the same
eigenvalues."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, tol_hphi, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ("chain12_nd3", (12, 1, 1), 3, 1.0),
    ("chain8_nd4", (8, 1, 1), 4, 0.6),
    ("square4_nd3", (4, 4, 1), 3, 1.0),
    ("square5x4_nd4", (5, 4, 1), 4, 1.2),
    ("cube3_nd3", (3, 3, 3), 3, 0.8),
]


@pytest.mark.parametrize("table", [True, False], ids=["table", "search"])
@pytest.mark.parametrize("name,dims,nd,anis", CASES, ids=[c[0] for c in CASES])
def test_stored_equals_matrix_free(name, dims, nd, anis, table):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=anis)
    Ks = qi.all_k(dims)
    b = lib_basis(spec, nd, Ks)
    if not table:
        b.rep_table(0)
    x = gaussian(21, b.total_dim, True)
    phi = to_dev(x, torch.complex128)
    ref = b.hphi(phi)
    ref64 = b.hphi(phi.to(torch.complex64))
    nbytes = b.store_terms(1)
    assert nbytes > 0 and b.store_terms(-1) == nbytes
    got = b.hphi(phi)
    got64 = b.hphi(phi.to(torch.complex64))
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    tol32 = tol_hphi(x, True)
    assert float((got64.to(torch.complex128) - ref64.to(torch.complex128)).abs().max()) <= tol32
    out = got.cpu().numpy()
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), nd, K)
        lo, hi = b.offsets[s], b.offsets[s + 1]
        if hi > lo:
            assert np.max(np.abs(out[lo:hi] - orc.hphi_k(sec, x[lo:hi]))) <= tol_hphi(x[lo:hi], False), K
    assert b.store_terms(0) == 0
    again = b.hphi(phi)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)


def test_stored_full_size_square10_nd4():
    torch = torch_cuda()
    b = lib_basis(qi.square(10), 4, qi.all_k((10, 10, 1)))
    phi = to_dev(gaussian(8, b.total_dim, True), torch.complex128)
    ref = b.hphi(phi)
    nbytes = b.store_terms(1)
    # 8 bytes per off-diagonal term, 16 per row
    assert nbytes == 8 * (b.nnz() - b.total_dim) + 8 * (b.total_dim + 1) + 8 * b.total_dim
    got = b.hphi(phi)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_stored_terms_in_lanczos():
    """Stored terms give the binary64 FMA product bit for bit, so a strict64
    solve (FMA products throughout) is identical with and without them; the
    default solve (integer products on the matrix-free path) agrees within
    rounding."""
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.square(6), 3, [(0, 0, 0), (1, 2, 0), (3, 3, 0)])
    o = qs3.SolveOpts(n_max=120, eps=1e-14, res_tol=1e-12, strict64=True)
    od = qs3.SolveOpts(n_max=120, eps=1e-14, res_tol=1e-12)
    e0, _, i0 = b.lanczos(o, vectors=False)
    ed, _, _ = b.lanczos(od, vectors=False)
    b.store_terms(1)
    e1, _, i1 = b.lanczos(o, vectors=False)
    np.testing.assert_array_equal(e0, e1)
    assert i0["iterations"] == i1["iterations"]
    assert float(np.max(np.abs(ed - e0))) <= 1e-13 * float(np.max(np.abs(e0)))


def test_stored_terms_errors():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    u1 = lib_basis(qi.chain(10), 3)
    with pytest.raises(qs3.QS3Error):
        u1.store_terms(1)
    k = lib_basis(qi.chain(10), 3, [(0, 0, 0)])
    with pytest.raises(qs3.QS3Error):
        k.store_terms(2)
    assert k.store_terms(-1) == 0
