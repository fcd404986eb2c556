"""Full diagonalisation of a sector (qs3_full_diag, the paper's ALG = 3) and
the thermal averages of Eq. (ens) (qs3_thermal): eigenvalues against the
dense diagonalisation of the oracle's Alg. 4 / Alg. 8 matrices, eigenvectors
by their residual through H Phi and their orthonormality, and Eq. (ens) over
all sectors of a small chain against the oracle and the full 2^N trace."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nd,anis", [((10, 1, 1), 3, 0.7), ((4, 3, 1), 3, 1.0), ((3, 3, 2), 2, 1.3)])
def test_full_diag_k_sectors(dims, nd, anis):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=anis)
    lat = olat(spec)
    Ks = qi.all_k(dims)[:4]
    b = lib_basis(spec, nd, Ks)
    for s, K in enumerate(Ks):
        want = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(lat, nd, K)))
        ev, V = b.full_diag(s, vectors=True)
        scale = max(1.0, float(np.max(np.abs(want)))) if len(want) else 1.0
        np.testing.assert_allclose(ev, want, atol=1e-12 * scale * 10)
        if len(ev) == 0:
            continue
        # orthonormal columns, and H v = E v through the matrix-free product
        G = V.conj().T @ V
        assert float((G - torch.eye(len(ev), dtype=G.dtype, device=G.device)).abs().max()) < 1e-11
        full = torch.zeros(b.total_dim, dtype=torch.complex128, device="cuda")
        for nu in (0, len(ev) // 2, len(ev) - 1):
            full.zero_()
            full[b.offsets[s]:b.offsets[s + 1]] = V[:, nu]
            hv = b.hphi(full)[b.offsets[s]:b.offsets[s + 1]]
            assert float((hv - ev[nu] * V[:, nu]).abs().max()) < 1e-11 * scale


def test_full_diag_u1():
    torch_cuda()
    spec = qi.chain(11, J=1.0, Jz=0.5)
    b = lib_basis(spec, 3)
    ev, _ = b.full_diag(0)
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(orc.dense_u1(olat(spec), 3)), atol=1e-11)


def test_thermal_over_all_sectors():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.chain(8, J=1.0, Jz=0.6)
    E, mz = [], []
    for nd in range(9):
        b = lib_basis(spec, nd, qi.all_k((8, 1, 1)))
        for s in range(b.n_sectors):
            if b.dims[s]:
                lv = b.full_diag(s)[0]
                E.append(lv)
                mz.append(np.full(len(lv), 4.0 - nd))        # S^z_total = N/2 - N_down
    E, mz = np.concatenate(E), np.concatenate(mz)
    assert len(E) == 256
    beta = np.array([0.05, 0.5, 2.0, 30.0])
    logz, eavg = qs3.thermal(E, beta)
    lz_o, ea_o = orc.thermal(E, None, beta)
    np.testing.assert_allclose(logz, lz_o, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(eavg, ea_o, rtol=1e-12, atol=1e-12)
    Ef = np.linalg.eigvalsh(pins.kron_hamiltonian(spec))
    for i, bt in enumerate(beta):
        w = np.exp(-bt * Ef)
        assert abs(logz[i] - np.log(w.sum())) < 1e-10
        assert abs(eavg[i] - (w * Ef).sum() / w.sum()) < 1e-10
    # the thermal magnetisation from the sector labels
    _, m_avg = qs3.thermal(E, beta, A=mz)
    _, m_o = orc.thermal(E, mz, beta)
    np.testing.assert_allclose(m_avg, m_o, atol=1e-12)


def test_full_diag_limits():
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.square(10), 4, [(1, 0, 0)])
    assert b.dims[0] > 16384
    with pytest.raises(qs3.QS3Error):
        b.full_diag(0)
    with pytest.raises(qs3.QS3Error):
        qs3.thermal(np.array([]), [1.0])
