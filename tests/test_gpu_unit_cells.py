"""Lattices with several spins per unit cell (the extension the paper's
Summary names for kagome-type lattices): the translation group moves cells,
every spin keeps its place in its cell.  On honeycomb and kagome clusters the
device-built sectors equal the oracle's Alg. 5-6 bit for bit (ranks, |Stab|,
dimensions against the character sum over the cell group), H Phi agrees
element by element with the oracle's Alg. 9 (with the representative table
and with the search, complex128, complex64 and double-float), stored terms
reproduce the matrix-free product bit for bit, and the lowest eigenvalue of
every sector agrees with the oracle's dense diagonalisation."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins
from tests.gpu_common import gaussian, lib_basis, olat, to_dev, tol_hphi, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [("honeycomb3x2", qi.honeycomb(3, 2), 3), ("kagome2x2", qi.kagome(2, 2, Jz=0.6), 3),
         ("kagome2x2", qi.kagome(2, 2), 4), ("honeycomb3x3", qi.honeycomb(3, 3, Jz=1.2), 4),
         ("kagome3x2", qi.kagome(3, 2), 3)]


@pytest.mark.parametrize("name,spec,nd", CASES)
def test_sectors_bit_exact_and_hphi(name, spec, nd):
    torch = torch_cuda()
    Ks = qi.all_k(spec.L)
    b = lib_basis(spec, nd, Ks)
    lat = olat(spec)
    for table in (True, False):
        if not table:
            b.rep_table(0)
        for s, K in enumerate(Ks):
            sec = orc.mk_list(lat, nd, K)
            assert b.dims[s] == sec.dim == pins.sector_dim_closed_form(spec.L, nd, K, spec.n_sub)
            if sec.dim == 0:
                continue
            r, st = b.ranks(s)
            np.testing.assert_array_equal(r, sec.rank0)
            np.testing.assert_array_equal(st, sec.stab)
        x = gaussian(7, b.total_dim, True)
        got = b.hphi(to_dev(x, torch.complex128)).cpu().numpy()
        got64 = b.hphi(to_dev(x, torch.complex64)).cpu().numpy()
        for s, K in enumerate(Ks):
            o0, o1 = b.offsets[s], b.offsets[s + 1]
            if o1 == o0:
                continue
            want = orc.hphi_k(orc.mk_list(lat, nd, K), x[o0:o1])
            assert float(np.max(np.abs(got[o0:o1] - want))) <= tol_hphi(x[o0:o1], False)
            assert float(np.max(np.abs(got64[o0:o1] - want))) <= tol_hphi(x[o0:o1], True)


def test_double_float_and_stored_terms_on_cells():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.kagome(3, 2)
    Ks = qi.all_k(spec.L)
    b = lib_basis(spec, 4, Ks)
    x = to_dev(gaussian(9, b.total_dim, True), torch.complex128)
    ref = b.hphi(x)
    df = b.hphi_df(qs3.split_df(x))
    assert float((df - ref).abs().max()) <= 1e-13 * float(x.abs().max()) * 16
    b.store_terms(1)
    st = b.hphi(x)
    assert torch.equal(st, ref)


@pytest.mark.parametrize("name,spec,nd", CASES[:4])
def test_lowest_eigenvalues_on_cells(name, spec, nd):
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    Ks = qi.all_k(spec.L)
    b = lib_basis(spec, nd, Ks)
    e, _, info = b.lanczos(qs3.SolveOpts(n_max=200, eps=1e-14, res_tol=1e-12), vectors=False)
    assert info["status"] == "QS3_OK"
    lat = olat(spec)
    for s, K in enumerate(Ks):
        sec = orc.mk_list(lat, nd, K)
        if sec.dim == 0:
            continue
        w = np.linalg.eigvalsh(orc.dense_k(sec))
        assert abs(e[s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


def test_cell_lattice_limits():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.kagome(2, 2)
    b = lib_basis(spec, 3, [(0, 0, 0)])
    dst = lib_basis(spec, 4, [(0, 0, 0)])
    x = to_dev(gaussian(1, b.total_dim, True), torch.complex128)
    with pytest.raises(qs3.QS3Error):
        b.correlations(x, 0, pairs=[(0, 1)])
    with pytest.raises(qs3.QS3Error):
        qs3.smq(b, 0, x, dst, 0, (0, 0, 0))
