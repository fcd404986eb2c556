"""Triangular-lattice samples (periodic Lx x Ly clusters, six neighbours): the
translation group is that of the square cluster and only the bonds change, so
the same basis build, representative search / table and H Phi apply.  Checked
against the oracle: bit-exact sectors, H Phi rows, lowest eigenvalues."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, tol_hphi, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [((4, 4), 2), ((4, 4), 3), ((6, 3), 3), ((5, 5), 2)]


@pytest.mark.parametrize("shape,nd", SHAPES, ids=[f"{s[0]}x{s[1]}_nd{n}" for s, n in SHAPES])
def test_triangular_sectors_and_hphi(shape, nd):
    torch = torch_cuda()
    Lx, Ly = shape
    spec = qi.triangular(Lx, Ly, J=1.0, Jz=0.9)
    lat = olat(spec)
    Ks = qi.all_k((Lx, Ly, 1))
    b = lib_basis(spec, nd, Ks)
    x = gaussian(31, b.total_dim, True)
    phi = to_dev(x, torch.complex128)
    got = b.hphi(phi)
    b.rep_table(0)
    got_search = b.hphi(phi)
    torch.cuda.synchronize()
    assert torch.equal(got, got_search)
    out = got.cpu().numpy()
    for s, K in enumerate(Ks):
        sec = orc.mk_list(lat, nd, K)
        r, st = b.ranks(s)
        np.testing.assert_array_equal(r, sec.rank0)
        np.testing.assert_array_equal(st.astype(np.int64), sec.stab)
        lo, hi = b.offsets[s], b.offsets[s + 1]
        if hi > lo:
            assert np.max(np.abs(out[lo:hi] - orc.hphi_k(sec, x[lo:hi]))) <= tol_hphi(x[lo:hi], False), K


def test_triangular_lowest_eigenvalues():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    Lx, Ly, nd = 4, 4, 3
    spec = qi.triangular(Lx, Ly, J=1.0, Jz=1.0)
    lat = olat(spec)
    Ks = qi.all_k((Lx, Ly, 1))
    b = lib_basis(spec, nd, Ks)
    e, _, info = b.lanczos(qs3.SolveOpts(n_max=150, eps=1e-14, res_tol=1e-12), vectors=False)
    assert info["status"] == "QS3_OK"
    lowest = []
    for s, K in enumerate(Ks):
        w = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(lat, nd, K)))
        assert abs(e[s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0])), K
        lowest.append(w[0])
    # the momentum sectors together hold the U(1) ground state
    assert abs(min(lowest) - np.linalg.eigvalsh(orc.dense_u1(lat, nd))[0]) < 1e-11
