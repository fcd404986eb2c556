"""GPU parity of S^+_q and S^z_q (qs3_sq_apply, the paper's spsmsz = 1 and 3)
and of their continued-fraction structure factors (qs3_dsf_op) against the
oracle: the operators applied by definition in the full U(1) basis and folded
onto the target sector, and the exact spectral sum of the target sector once
the Lanczos run has exhausted its Krylov space."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SP, SM, SZ = 1, 2, 3
TOL = 1e-12


def qs3mod():
    import paper_2107_00872_gb300 as qs3
    return qs3


def _dn(op):
    return -1 if op == SP else (1 if op == SM else 0)


@pytest.mark.parametrize("op", [SP, SZ])
@pytest.mark.parametrize("dims,nd", [((8, 1, 1), 3), ((4, 3, 1), 2), ((3, 2, 2), 2), ((6, 1, 1), 1)])
def test_sq_apply_k_against_oracle(op, dims, nd):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=0.8)
    lat = olat(spec)
    for K in qi.all_k(dims)[:3]:
        src = lib_basis(spec, nd, [K])
        osrc = orc.mk_list(lat, nd, K)
        if osrc.dim == 0:
            continue
        x = gaussian(13, osrc.dim, True)
        for Q in qi.all_k(dims)[:4]:
            K2 = tuple((K[a] + Q[a]) % dims[a] for a in range(3))
            dst = lib_basis(spec, nd + _dn(op), [K2])
            odst = orc.mk_list(lat, nd + _dn(op), K2)
            got = qs3mod().sq_apply(op, src, 0, to_dev(x, torch.complex128), dst, 0, Q).cpu().numpy()
            want = orc.sq_apply_k(osrc, x, op, Q, odst)
            assert got.shape == want.shape
            assert np.max(np.abs(got - want), initial=0.0) <= TOL * max(1.0, np.max(np.abs(x))) * 8, (K, Q)


@pytest.mark.parametrize("op", [SP, SZ, SM])
def test_sq_apply_u1_against_oracle(op):
    torch = torch_cuda()
    N, nd = 10, 3
    spec = qi.chain(N)
    src = lib_basis(spec, nd)
    dst = lib_basis(spec, nd + _dn(op))
    x = gaussian(17, src.total_dim, True)
    for q in (0, 3, 7):
        got = qs3mod().sq_apply(op, src, 0, to_dev(x, torch.complex128), dst, 0, (q, 0, 0)).cpu().numpy()
        want = orc.sq_apply_u1(N, nd, op, x, (q, 0, 0), (N, 1, 1))
        np.testing.assert_allclose(got, want, atol=TOL * 8)


def test_sq_apply_vacuum_edges():
    """S^+ from one down spin to the vacuum, S^z on the vacuum, both bases."""
    torch = torch_cuda()
    dims = (4, 3, 1)
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    N = spec.n_sites
    for K in [(0, 0, 0), (1, 2, 0)]:
        one = lib_basis(spec, 1, [K])
        x = gaussian(3, one.total_dim, True)
        Q = tuple((-K[a]) % dims[a] for a in range(3))
        vac = lib_basis(spec, 0, [(0, 0, 0)])
        got = qs3mod().sq_apply(SP, one, 0, to_dev(x, torch.complex128), vac, 0, Q).cpu().numpy()
        want = orc.sq_apply_k(orc.mk_list(lat, 1, K), x, SP, Q, orc.mk_list(lat, 0, (0, 0, 0)))
        np.testing.assert_allclose(got, want, atol=TOL * 8)
    vac = lib_basis(spec, 0, [(0, 0, 0)])
    got = qs3mod().sq_apply(SZ, vac, 0, to_dev(np.ones(1, np.complex128), torch.complex128), vac, 0,
                            (0, 0, 0)).cpu().numpy()
    np.testing.assert_allclose(got, [(N / 2) / np.sqrt(N)], atol=TOL)
    u1 = lib_basis(qi.chain(9), 1)
    vu = lib_basis(qi.chain(9), 0)
    x = gaussian(5, 9, True)
    got = qs3mod().sq_apply(SP, u1, 0, to_dev(x, torch.complex128), vu, 0, (2, 0, 0)).cpu().numpy()
    np.testing.assert_allclose(got, orc.sq_apply_u1(9, 1, SP, x, (2, 0, 0), (9, 1, 1)), atol=TOL * 8)


def _ground(spec, nd, dims):
    lat = olat(spec)
    best = None
    for K in qi.all_k(dims):
        sec = orc.mk_list(lat, nd, K)
        if sec.dim == 0:
            continue
        e, v = np.linalg.eigh(orc.dense_k(sec))
        if best is None or e[0] < best[0] - 1e-10:
            best = (e[0], v[:, 0], sec)
    return best


@pytest.mark.parametrize("op", [SZ, SP])
def test_dsf_op_against_exact_spectral_sum(op):
    """n_iter exceeds every target sector's dimension, so the continued
    fraction equals the exact sum of Lorentzians over the target sector."""
    torch = torch_cuda()
    dims, nd = (4, 3, 1), 3
    spec = qi.hypercubic(dims, J=1.0, Jz=1.2)
    lat = olat(spec)
    N = spec.n_sites
    E0, phi, sec = _ground(spec, nd, dims)
    Qs = qi.all_k(dims)
    K2s = [tuple((sec.K[a] + Q[a]) % dims[a] for a in range(3)) for Q in Qs]
    Bs = lib_basis(spec, nd, [sec.K])
    Bd = lib_basis(spec, nd + _dn(op), K2s)
    n_iter = max(Bd.dims) + 2
    omega = np.linspace(-2.0, 8.0, 501)
    h, eta = 1.5, 0.05
    s, al, be, n2 = qs3mod().dsf(Bs, 0, to_dev(phi, torch.complex128), E0, Bd, Qs, n_iter, eta, h, omega, op=op)
    # Parseval over all q: N/4 for S^z, N_down for S^+ (unit ground state)
    assert abs(n2.sum() - (N / 4 if op == SZ else nd)) < 1e-11
    for n, Q in enumerate(Qs):
        dst = orc.mk_list(lat, nd + _dn(op), K2s[n])
        v = orc.sq_apply_k(sec, phi, op, Q, dst)
        assert abs(np.vdot(v, v).real - n2[n]) < 1e-12
        if n2[n] < 1e-14:
            continue
        en, U = np.linalg.eigh(orc.dense_k(dst))
        wgt = np.abs(U.conj().T @ v) ** 2
        shift = h * _dn(op)
        exact = sum(wgt[k] * (eta / np.pi) / ((omega + E0 - shift - en[k]) ** 2 + eta ** 2) for k in range(len(en)))
        peak = max(np.max(exact), 1e-300)
        assert np.max(np.abs(s[n] - exact)) <= 1e-6 * peak, (Q, np.max(np.abs(s[n] - exact)), peak)


def test_dsf_sz_trivial_subtraction():
    """At q = 0, S^z_q phi is (M / sqrt(N)) phi: subtracting the ground state's
    own Lorentzian leaves nothing; other q are unchanged."""
    torch = torch_cuda()
    dims, nd = (4, 3, 1), 2
    spec = qi.hypercubic(dims)
    E0, phi, sec = _ground(spec, nd, dims)
    Qs = [(0, 0, 0), (1, 0, 0)]
    K2s = [tuple((sec.K[a] + Q[a]) % dims[a] for a in range(3)) for Q in Qs]
    Bs = lib_basis(spec, nd, [sec.K])
    Bd = lib_basis(spec, nd, K2s)
    omega = np.linspace(-1.0, 4.0, 301)
    g = to_dev(phi, torch.complex128)
    s0, _, _, n2 = qs3mod().dsf(Bs, 0, g, E0, Bd, Qs, 40, 0.05, 0.0, omega, op=SZ)
    s1, _, _, _ = qs3mod().dsf(Bs, 0, g, E0, Bd, Qs, 40, 0.05, 0.0, omega, op=SZ, subtract_trivial=True)
    N = spec.n_sites
    M = N / 2 - nd
    assert abs(n2[0] - M * M / N) < 1e-10
    assert np.max(np.abs(s1[0])) <= 1e-6 * np.max(s0[0])
    np.testing.assert_array_equal(s1[1], s0[1])
