"""GPU parity: conventional Lanczos and thick-restart Lanczos (Alg. 10),
batched over sectors, fp64 and fp32-with-fp64-refinement, against the
oracle's dense matrices (Alg. 4 / Alg. 8) diagonalised by numpy."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


def opts(**kw):
    import paper_2107_00872_gb300 as qs3
    return qs3.SolveOpts(**kw)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lanczos_chain16_ground_state(prec):
    """16-site periodic Heisenberg chain, N_down = 3 (dim 560), no momentum:
    lowest eigenvalue to 1e-12 relative (fp64) or 1e-9 after fp32 + refinement,
    FP64 residual <= 1e-12 |E|, eigenvector equal to the dense one."""
    torch_cuda()
    spec = qi.chain(16)
    H = orc.dense_u1(olat(spec), 3)
    ev, U = np.linalg.eigh(H)
    B = lib_basis(spec, 3)
    e, vec, info = B.lanczos(opts(n_max=300, eps=1e-14, precision=prec, seed=1))
    assert info["status"] == "QS3_OK", info
    tol = 1e-12 if prec == "f64" else 1e-9
    assert abs(e[0, 0] - ev[0]) <= tol * abs(ev[0]), (e, ev[0])
    # fp64: residual <= 1e-12 |E| (res_tol); fp32 + refinement: |dE| <= 1e-9 |E| needs ~sqrt of that
    assert info["max_residual"] <= (1e-11 if prec == "f64" else 1e-4) * abs(ev[0]), info
    v = vec.cpu().numpy()
    assert abs(abs(np.dot(v, U[:, 0])) - 1.0) < (1e-10 if prec == "f64" else 1e-7)
    if prec == "f32":
        assert info["refine_iterations"] > 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_trl_chain16_lowest_four(prec):
    torch_cuda()
    spec = qi.chain(16, Jz=0.7)
    H = orc.dense_u1(olat(spec), 3)
    ev = np.linalg.eigvalsh(H)
    B = lib_basis(spec, 3)
    e, vecs, info = B.trlanczos(opts(n_eig=4, n_keep=8, n_max=32, max_iter=500, eps=1e-13, precision=prec))
    assert info["status"] == "QS3_OK", info
    tol = 1e-11 if prec == "f64" else 1e-9
    np.testing.assert_allclose(e[0], ev[:4], rtol=0, atol=tol * abs(ev[0]))
    V = vecs.cpu().numpy().reshape(4, -1)
    np.testing.assert_allclose(V @ V.T, np.eye(4), atol=1e-8)


def test_lanczos_batched_k_sectors_square4x4():
    """All 16 momentum sectors of the 4x4 square lattice at N_down = 4 in one
    batched solve; each lowest eigenvalue against the dense Alg. 8 block."""
    torch_cuda()
    spec = qi.square(4, 4, Jz=0.9)
    Ks = qi.all_k((4, 4, 1))
    B = lib_basis(spec, 4, Ks)
    e, vec, info = B.lanczos(opts(n_max=200, eps=1e-14))
    assert info["status"] == "QS3_OK", info
    v = vec.cpu().numpy()
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), 4, K)
        Hk = orc.dense_k(sec)
        w, U = np.linalg.eigh(Hk)
        assert abs(e[s, 0] - w[0]) <= 1e-11 * max(1.0, abs(w[0])), (K, e[s, 0], w[0])
        a, b = B.offsets[s], B.offsets[s + 1]
        r = Hk @ v[a:b] - e[s, 0] * v[a:b]
        assert np.linalg.norm(r) < 1e-9


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_trl_batched_cubic_and_exhausted_sectors(prec):
    """3x3x3 cubic lattice, N_down = 3: 27 sectors, several smaller than N_M
    (the Krylov space is exhausted and the Ritz values are exact)."""
    torch_cuda()
    spec = qi.cubic(3, Jz=1.1)
    Ks = qi.all_k((3, 3, 3))
    B = lib_basis(spec, 3, Ks)
    e, vecs, info = B.trlanczos(opts(n_eig=3, n_keep=6, n_max=24, max_iter=500, eps=1e-13, precision=prec))
    assert info["status"] == "QS3_OK", info
    tol = 1e-10 if prec == "f64" else 1e-9
    for s, K in enumerate(Ks):
        sec = orc.mk_list(olat(spec), 3, K)
        w = np.linalg.eigvalsh(orc.dense_k(sec))
        n = min(3, len(w))
        np.testing.assert_allclose(e[s, :n], w[:n], atol=tol * max(1.0, abs(w[0])))


def test_trl_k_sector_square6x6():
    torch_cuda()
    spec = qi.square(6)
    sec = orc.mk_list(olat(spec), 4, (0, 0, 0))
    w = np.linalg.eigvalsh(orc.dense_k(sec))
    B = lib_basis(spec, 4, [(0, 0, 0), (1, 2, 0)])
    e, _, info = B.trlanczos(opts(n_eig=4, n_keep=8, n_max=32, max_iter=1000, eps=1e-13))
    assert info["status"] == "QS3_OK", info
    np.testing.assert_allclose(e[0], w[:4], atol=1e-10 * abs(w[0]))
    w2 = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(spec), 4, (1, 2, 0))))
    np.testing.assert_allclose(e[1], w2[:4], atol=1e-10 * abs(w2[0]))


def test_solver_option_errors():
    import paper_2107_00872_gb300 as qs3
    B = lib_basis(qi.chain(8), 2)
    with pytest.raises(qs3.QS3Error) as ex:
        B.trlanczos(opts(n_eig=9, n_keep=8, n_max=32))
    assert ex.value.status == -1
    with pytest.raises(qs3.QS3Error) as ex:
        B.lanczos(opts(n_max=1))
    assert ex.value.status == -1


def test_not_converged_status():
    """A too-small iteration limit reports QS3_ERR_NOT_CONVERGED (and the
    current Ritz value)."""
    B = lib_basis(qi.disordered_open_square(8, seed=3), 3)
    e, _, info = B.lanczos(opts(n_max=6, min_iter=2, check_every=2, eps=1e-15))
    assert info["status"] == "QS3_ERR_NOT_CONVERGED"
    assert np.isfinite(e[0, 0])
