"""GPU parity at the full sizes of the benchmark workloads, on sampled rows
the oracle computes one by one (Alg. 9 for U(1) rows; for momentum sectors,
one row of Alg. 9 with Alg. 7 / Alg. 5 applied to every hop target, which
needs no representative list), plus exact properties: closed-form sector
dimensions, validity of sampled representatives, sum rules."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins
from tests.gpu_common import lib_basis, olat, to_dev, tol_hphi, torch_cuda

pytestmark = pytest.mark.gpu


def _check_k_rows(spec, nd, K, B, s, x, got, rows, fp32):
    lat = olat(spec)
    r, st = B.ranks(s)
    a, b = B.offsets[s], B.offsets[s + 1]
    xs, gs = x[a:b], got[a:b]
    tol = tol_hphi(xs, fp32)
    for row in rows:
        rep1 = int(r[row]) + 1
        res = orc.row_terms_k(lat, nd, K, rep1)
        assert res is not None, "GPU representative is not a compatible representative"
        dg, tgt, cf = res
        assert int(st[row]) * spec.n_sites == round(orc.check_state(lat, nd, K, rep1))
        idx = np.searchsorted(r, tgt.astype(np.uint64) - np.uint64(1))
        assert np.all(idx < len(r)) and np.all(r[np.minimum(idx, len(r) - 1)] == tgt - 1), "target missing from sigma"
        want = dg * xs[row] + np.sum(cf * xs[idx])
        assert abs(gs[row] - want) <= tol, (row, gs[row], want)


def test_disordered_open_square_32x32_full_u1():
    """Config 4: open 32x32 square, random XXZ couplings and site field,
    N_down = 3, dim 178,433,024; fp64 and fp32 H Phi on sampled rows."""
    torch = torch_cuda()
    spec = qi.disordered_open_square(32)
    B = lib_basis(spec, 3)
    D = comb(1024, 3)
    assert B.total_dim == D == 178433024
    rng = np.random.default_rng(11)
    x = rng.standard_normal(D)
    rows = np.concatenate([[0, 1, D - 1], rng.integers(0, D, 400)])
    want = orc.hphi_u1_rows(olat(spec), 3, x, rows).real
    for dt in (torch.float64, torch.float32):
        xd = to_dev(x, dt)
        got = B.hphi(xd)
        g = got[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        assert np.max(np.abs(g - want)) <= tol_hphi(x, dt == torch.float32)
        del xd, got
    # local magnetisation of a state: sum_i <s^z_i> = N/2 - N_down exactly
    xd = to_dev(x / np.linalg.norm(x), torch.float64)
    out = B.correlations(xd, 0, local=True)
    assert abs(out["sz"].sum() - (512 - 3)) < 1e-9
    assert np.all(np.abs(out["sz"]) <= 0.5 + 1e-12)


def _apply(B, x, dt):
    """H x through qs3_hphi as complex128, complex64 or double-float (C128DF)."""
    import paper_2107_00872_gb300 as qs3
    torch = torch_cuda()
    if dt == "c128df":
        return B.hphi_df(qs3.split_df(to_dev(x, torch.complex128))).cpu().numpy()
    return B.hphi(to_dev(x, torch.complex128 if dt == "c128" else torch.complex64)).cpu().numpy().astype(complex)


@pytest.mark.parametrize("dt", ["c128", "c128df", "c64"])
def test_cubic10_nd4_gamma_sector_full(dt):
    """Config 3's largest sector: 10x10x10, N_down = 4, k = 0: the dimension
    equals the character-sum closed form, sampled representatives are valid,
    sampled H Phi rows match the oracle."""
    torch = torch_cuda()
    spec = qi.cubic(10)
    K = (0, 0, 0)
    B = lib_basis(spec, 4, [K])
    d = B.dims[0]
    assert d == pins.sector_dim_closed_form((10, 10, 10), 4, K)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    got = _apply(B, x, dt)
    rows = np.concatenate([[0, d - 1], rng.integers(0, d, 60)])
    _check_k_rows(spec, 4, K, B, 0, x, got, rows, dt == "c64")


def test_cubic10_nd3_kpath_sectors():
    """Config 3 at N_down = 3: the 28 distinct sectors of the k-path in one
    batched basis; dimensions by closed form, sampled rows of three sectors."""
    torch = torch_cuda()
    spec = qi.cubic(10)
    path = qi.cubic_kpath(10)
    Ks = list(dict.fromkeys(path))
    assert len(path) == 31 and len(Ks) == 28
    B = lib_basis(spec, 3, Ks)
    for s, K in enumerate(Ks):
        assert B.dims[s] == pins.sector_dim_closed_form((10, 10, 10), 3, K)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(B.total_dim) + 1j * rng.standard_normal(B.total_dim)
    got = B.hphi(to_dev(x, torch.complex128)).cpu().numpy()
    for s in (0, 7, 20):
        rows = rng.integers(0, B.dims[s], 40)
        _check_k_rows(spec, 3, Ks[s], B, s, x, got, rows, False)


@pytest.mark.parametrize("dt", ["c128", "c128df"])
def test_square10_nd4_all_sectors_batched_rows(dt):
    """Config 2: all 100 sectors of the 10x10 square lattice at N_down = 4 in
    one batched H Phi (complex128 and double-float); sampled rows of several
    sectors."""
    torch_cuda()
    spec = qi.square(10)
    Ks = qi.all_k((10, 10, 1))
    B = lib_basis(spec, 4, Ks)
    assert sum(B.dims) == comb(100, 4)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(B.total_dim) + 1j * rng.standard_normal(B.total_dim)
    got = _apply(B, x, dt)
    for s in (0, 1, 11, 55, 99):
        rows = np.concatenate([[0, B.dims[s] - 1], rng.integers(0, B.dims[s], 50)])
        _check_k_rows(spec, 4, Ks[s], B, s, x, got, rows, False)


def test_cubic6_nd5_paper_workload_rows():
    """The paper's OpenMP benchmark workload: 6x6x6, N_down = 5, k = 0
    (dimension 17,313,563 quoted in the paper); sampled rows."""
    torch = torch_cuda()
    spec = qi.cubic(6)
    B = lib_basis(spec, 5, [(0, 0, 0)])
    assert B.dims == [17313563]
    rng = np.random.default_rng(1)
    d = B.dims[0]
    x = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    got = B.hphi(to_dev(x, torch.complex128)).cpu().numpy()
    _check_k_rows(spec, 5, (0, 0, 0), B, 0, x, got, rng.integers(0, d, 40), False)
