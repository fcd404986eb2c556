"""GPU parity: basis construction (bit-exact) and H Phi (fp64 / fp32) against
the oracle, through the C ABI."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins
from tests.gpu_common import gaussian, lib_basis, olat, to_dev, tol_hphi, torch_cuda

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------- U(1) H Phi

U1_CASES = [
    ("chain16_nd3", lambda: qi.chain(16), 3),                       # the 16-site chain workload
    ("random14_nd4", lambda: qi.random_graph(14, 30, 9), 4),         # random couplings + site field
    ("open12x12_nd3", lambda: qi.disordered_open_square(12, seed=5), 3),  # small disordered open square
    ("chain9_nd1", lambda: qi.chain(9, J=0.7, Jz=1.3), 1),
    ("chain8_nd8", lambda: qi.chain(8), 8),                         # fully down: no hops
    ("chain10_nd0", lambda: qi.chain(10), 0),                       # vacuum
]


@pytest.mark.parametrize("name,mk,nd", U1_CASES, ids=[c[0] for c in U1_CASES])
@pytest.mark.parametrize("dt", ["f64", "f32", "c128", "c64"])
def test_hphi_u1_parity(name, mk, nd, dt):
    torch = torch_cuda()
    spec = mk()
    B = lib_basis(spec, nd)
    D = comb(spec.n_sites, nd)
    assert B.total_dim == D and B.dims == [D]
    cplx = dt.startswith("c")
    x = gaussian(17, D, cplx)
    want = orc.hphi_u1(olat(spec), nd, x.astype(np.complex128))
    tdt = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128, "c64": torch.complex64}[dt]
    phi = to_dev(x, tdt)
    psi = B.hphi(phi)
    got = psi.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - (want if cplx else want.real)))
    assert err <= tol_hphi(x, dt in ("f32", "c64")), err


def test_hphi_u1_nnz():
    spec = qi.disordered_open_square(5, seed=2)
    B = lib_basis(spec, 3)
    H = orc.dense_u1(olat(spec), 3)
    assert B.nnz() == int(np.count_nonzero(H))


# ------------------------------------------------------- k-sector basis

K_CASES = [
    ("chain12_nd3", (12, 1, 1), 3, 1.0),
    ("chain12_nd4", (12, 1, 1), 4, 0.6),
    ("sq4x3_nd3", (4, 3, 1), 3, 1.0),
    ("sq5x4_nd4", (5, 4, 1), 4, 1.2),
    ("cub3x3x2_nd3", (3, 3, 2), 3, 0.8),
    ("sq6x6_nd3", (6, 6, 1), 3, 1.0),
    ("cub3x3x3_nd4", (3, 3, 3), 4, 1.0),
    ("chain7_nd7", (7, 1, 1), 7, 1.0),
    ("chain9_nd1", (9, 1, 1), 1, 1.0),
]


def _sectors(dims):
    ks = qi.all_k(dims)
    return ks if len(ks) <= 12 else ks[:: max(1, len(ks) // 10)]


@pytest.mark.parametrize("name,dims,nd,anis", K_CASES, ids=[c[0] for c in K_CASES])
def test_k_basis_bit_exact(name, dims, nd, anis):
    spec = qi.hypercubic(dims, J=1.0, Jz=anis)
    Ks = qi.all_k(dims)
    B = lib_basis(spec, nd, Ks)
    assert sum(B.dims) == comb(spec.n_sites, nd)
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), nd, K)
        r, st = B.ranks(s)
        assert B.dims[s] == sec.dim == pins.sector_dim_closed_form(dims, nd, K)
        np.testing.assert_array_equal(r, sec.rank0)
        np.testing.assert_array_equal(st.astype(np.int64), sec.stab)


@pytest.mark.parametrize("name,dims,nd,anis", K_CASES, ids=[c[0] for c in K_CASES])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_hphi_k_parity_batched(name, dims, nd, anis, dt):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=anis)
    Ks = _sectors(dims)
    B = lib_basis(spec, nd, Ks)
    x = gaussian(23, B.total_dim, True)
    phi = to_dev(x, torch.complex128 if dt == "c128" else torch.complex64)
    got = B.hphi(phi).cpu().numpy().astype(np.complex128)
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), nd, K)
        a, b = B.offsets[s], B.offsets[s + 1]
        want = orc.hphi_k(sec, x[a:b])
        err = np.max(np.abs(got[a:b] - want)) if b > a else 0.0
        assert err <= tol_hphi(x[a:b], dt == "c64"), (K, err)


def test_hphi_k_multi_tile_square8():
    """8x8 square lattice, N_down = 4: sectors of ~10^4 rows (many tiles)."""
    torch = torch_cuda()
    spec = qi.square(8)
    Ks = [(0, 0, 0), (1, 3, 0), (4, 4, 0)]
    B = lib_basis(spec, 4, Ks)
    x = gaussian(5, B.total_dim, True)
    got = B.hphi(to_dev(x, torch.complex128)).cpu().numpy()
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), 4, K)
        a, b = B.offsets[s], B.offsets[s + 1]
        assert b - a == sec.dim > 5000
        r, _ = B.ranks(s)
        np.testing.assert_array_equal(r, sec.rank0)
        assert np.max(np.abs(got[a:b] - orc.hphi_k(sec, x[a:b]))) <= tol_hphi(x[a:b], False)


def test_k_dims_large_closed_forms():
    """Sector sizes of the paper's systems, built on the device: the 6x6x6
    N_down = 5 k = 0 sector quoted in the paper, and every momentum sector of
    the 10x10 square lattice at N_down = 4."""
    B = lib_basis(qi.cubic(6), 5, [(0, 0, 0)])
    assert B.dims == [17313563]
    ks = qi.all_k((10, 10, 1))
    B = lib_basis(qi.square(10), 4, ks)
    assert sum(B.dims) == comb(100, 4)
    for s in range(0, 100, 7):
        assert B.dims[s] == pins.sector_dim_closed_form((10, 10, 1), 4, ks[s])
    r, st = B.ranks(0)
    assert np.all(np.diff(r.astype(np.int64)) > 0)
