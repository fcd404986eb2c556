"""GPU parity: two-point functions, S(q), S^-_q phi (Alg. 11) and the
continued-fraction S^-(q, omega) (Eq. cfe) against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins
from tests.gpu_common import lib_basis, olat, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def qs3mod():
    import paper_2107_00872_gb300 as qs3
    return qs3


def grid_q(L):
    return [(2 * np.pi * K[0] / L[0], 2 * np.pi * K[1] / L[1], 2 * np.pi * K[2] / L[2]) for K in qi.all_k(L)]


def sq_from_matrix(M, spec, q):
    """(1/N) sum_{r,r'} e^{iq.(R_r - R_r')} M[r, r'] with lattice coordinates."""
    N = spec.n_sites
    L = spec.L if spec.L != (0, 0, 0) else (N, 1, 1)
    R = np.array([pins.coords(r, L) for r in range(N)], float)
    e = np.exp(1j * R @ np.array(q))
    return float((np.outer(e, e.conj()) * M).sum().real / N)


def test_correlations_u1_chain16_ground_state():
    torch = torch_cuda()
    spec = qi.chain(16)
    B = lib_basis(spec, 3)
    e, vec, info = B.lanczos(qs3mod().SolveOpts(n_max=300))
    phi = vec.cpu().numpy()
    pairs = [(i, j) for i in range(16) for j in range(16)]
    qs = grid_q((16, 1, 1))
    out = B.correlations(vec, 0, pairs=pairs, q=qs, local=True)
    szsz, spsm, sz = orc.corr_u1(16, 3, phi.astype(np.complex128))
    np.testing.assert_allclose(out["szsz"], szsz.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["spsm"], spsm.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["sz"], sz, atol=1e-12)
    for n, q in enumerate(qs):
        assert abs(out["sq_zz"][n] - sq_from_matrix(szsz, spec, q)) < 1e-11
        assert abs(out["sq_pm"][n] - sq_from_matrix(spsm, spec, q)) < 1e-11
    del torch


def test_correlations_u1_random_field():
    torch = torch_cuda()
    spec = qi.random_graph(12, 25, 3)
    B = lib_basis(spec, 4)
    x = qi.gaussian_start(9, B.total_dim, False)
    out = B.correlations(to_dev(x, torch.float64), 0, pairs=[(0, 5), (3, 3), (11, 2)], local=True)
    szsz, spsm, sz = orc.corr_u1(12, 4, (x / np.linalg.norm(x)).astype(np.complex128))
    np.testing.assert_allclose(out["szsz"], [szsz[0, 5], szsz[3, 3], szsz[11, 2]], atol=1e-12)
    np.testing.assert_allclose(out["spsm"], [spsm[0, 5], spsm[3, 3], spsm[11, 2]], atol=1e-12)
    np.testing.assert_allclose(out["sz"], sz, atol=1e-12)


@pytest.mark.parametrize("dims,nd,K", [((4, 3, 1), 3, (1, 2, 0)), ((12, 1, 1), 3, (5, 0, 0)),
                                       ((3, 3, 2), 2, (0, 1, 1))])
def test_correlations_k_sector_equal_site_resolved(dims, nd, K):
    """Translation-symmetrised operators in the sector give the site-resolved
    values of the unfolded state (the state is a translation eigenstate)."""
    torch = torch_cuda()
    spec = qi.hypercubic(dims, Jz=0.8)
    N = spec.n_sites
    B = lib_basis(spec, nd, [K])
    sec = orc.mk_list(olat(spec), nd, K)
    x = qi.gaussian_start(4, sec.dim, True)
    x /= np.linalg.norm(x)
    pairs = [(i, j) for i in range(N) for j in range(N)]
    qs = grid_q(dims)
    out = B.correlations(to_dev(x, torch.complex128), 0, pairs=pairs, q=qs, local=True)
    szsz, spsm, sz = orc.corr_u1(N, nd, orc.unfold(sec, x))
    np.testing.assert_allclose(out["szsz"], szsz.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["spsm"], spsm.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["sz"], sz, atol=1e-12)
    for n, q in enumerate(qs):
        assert abs(out["sq_zz"][n] - sq_from_matrix(szsz, spec, q)) < 1e-11
        assert abs(out["sq_pm"][n] - sq_from_matrix(spsm, spec, q)) < 1e-11


@pytest.mark.parametrize("dims,nd", [((12, 1, 1), 2), ((4, 3, 1), 2), ((3, 3, 2), 1), ((4, 3, 1), 0),
                                     ((5, 4, 1), 3)])
def test_smq_pull_equals_oracle_push(dims, nd):
    torch = torch_cuda()
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    Ks = qi.all_k(dims)[:3] if nd else [(0, 0, 0)]
    for K in Ks:
        src = orc.mk_list(lat, nd, K)
        if src.dim == 0:
            continue
        Bs = lib_basis(spec, nd, [K])
        x = qi.gaussian_start(6, src.dim, True)
        for Q in qi.all_k(dims)[:5]:
            K2 = tuple((K[a] + Q[a]) % dims[a] for a in range(3))
            dst = orc.mk_list(lat, nd + 1, K2)
            Bd = lib_basis(spec, nd + 1, [K2])
            got = qs3mod().smq(Bs, 0, to_dev(x, torch.complex128), Bd, 0, Q).cpu().numpy()
            want = orc.smq(src, x, Q, dst)
            np.testing.assert_allclose(got, want, atol=1e-12)


def test_smq_u1_against_definition():
    torch = torch_cuda()
    spec = qi.chain(10)
    Bs, Bd = lib_basis(spec, 2), lib_basis(spec, 3)
    x = qi.gaussian_start(2, Bs.total_dim, True)
    Q = (3, 0, 0)
    got = qs3mod().smq(Bs, 0, to_dev(x, torch.complex128), Bd, 0, Q).cpu().numpy()
    src = pins.colex_subsets(10, 2)
    dst = {c: k for k, c in enumerate(pins.colex_subsets(10, 3))}
    want = np.zeros(len(dst), complex)
    for k, c in enumerate(src):
        for r in range(10):
            if r not in c:
                want[dst[tuple(sorted(c + (r,)))]] += np.exp(-2j * np.pi * 3 * r / 10) * x[k] / np.sqrt(10)
    np.testing.assert_allclose(got, want, atol=1e-12)


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


@pytest.mark.parametrize("dims,nd,n_iter", [((8, 1, 1), 2, 40), ((4, 3, 1), 2, 30), ((6, 6, 1), 2, 210)])
def test_dsf_batched_against_oracle(dims, nd, n_iter):
    """n_iter is at least the target sector dimension, so the Lanczos run
    exhausts the Krylov space and the continued fraction equals the exact
    spectral sum; late Lanczos coefficients before exhaustion depend on
    rounding (two valid reorthogonalisations differ there), so only the
    first coefficients are compared one by one."""
    torch = torch_cuda()
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    E0, phi, sec = _ground(spec, nd, dims)
    Qs = qi.all_k(dims)
    K2s = [tuple((sec.K[a] + Q[a]) % dims[a] for a in range(3)) for Q in Qs]
    Bs = lib_basis(spec, nd, [sec.K])
    Bd = lib_basis(spec, nd + 1, K2s)
    omega = np.linspace(-1.0, 7.0, 801)
    h, eta = 2.0, 0.05
    s, al, be, n2 = qs3mod().dsf(Bs, 0, to_dev(phi, torch.complex128), E0, Bd, Qs, n_iter, eta, h, omega)
    # static S(q) from the correlations: |S^-_q phi|^2 = S^{+-}(q)  (sum rule route 1)
    corr = Bs.correlations(to_dev(phi, torch.complex128), 0, q=grid_q(dims))
    np.testing.assert_allclose(n2, corr["sq_pm"], atol=1e-12)
    for n, Q in enumerate(Qs):
        dst = orc.mk_list(lat, nd + 1, K2s[n])
        v = orc.smq(sec, phi, Q, dst)
        assert abs(np.vdot(v, v).real - n2[n]) < 1e-12
        if n2[n] < 1e-14:
            continue
        assert dst.dim <= n_iter
        Hd = orc.dense_k(dst)
        a, b, Psi, b0 = orc.lanczos(lambda y: Hd @ y, v, n_iter)
        m = min(len(a), 8)
        np.testing.assert_allclose(al[n, :m], a[:m], atol=1e-10)
        np.testing.assert_allclose(be[n, 1:m], b[:m - 1], atol=1e-10)
        # exact spectral sum from the dense eigendecomposition (Lorentzians of width eta)
        en, U = np.linalg.eigh(Hd)
        wgt = np.abs(U.conj().T @ v) ** 2
        exact = sum(wgt[k] * (eta / np.pi) / ((omega + E0 - h - en[k]) ** 2 + eta ** 2) for k in range(len(en)))
        peak = max(np.max(exact), 1e-300)
        assert np.max(np.abs(s[n] - exact)) <= 1e-6 * peak, (Q, np.max(np.abs(s[n] - exact)), peak)
        ref = orc.continued_fraction(a, b, n2[n], omega, E0, eta, shift=h)
        assert np.max(np.abs(ref - exact)) <= 1e-6 * peak
        # sum rule route 2: the spectral weights of T sum to |S^-_q phi|^2
        mm = int(np.count_nonzero(al[n]))
        T = orc.tridiag(al[n][:mm], be[n][1:mm])
        w, C = np.linalg.eigh(T)
        assert abs(n2[n] * (C[0] ** 2).sum() - n2[n]) < 1e-10
