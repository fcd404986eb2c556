"""Ground state and local magnetisation of the bond-disordered open square
lattice (J ~ U[0.5, 1.5], Jz = 0.8 J, h_i ~ U[-0.1, 0.1], seeded; Alg. 10 and
Sec. "Calculating expectation values").

- Reduced 8x8 lattice, N_down = 3 (dimension 41,664): thick-restart Lanczos
  with fp32 H Phi + binary64 refinement, and in plain binary64, against the
  oracle's Lanczos ground state (its H Phi is Alg. 9 as printed): E within
  1e-9 |E| and every <s^z_i> within 1e-8.
- Full 32x32 lattice, N_down = 3 (dimension 178,433,024): the refined state's
  binary64 residual |H v - E v| <= 1e-9 |E|, agreement of the fp32 +
  refinement energy with the plain binary64 one, and sum_i <s^z_i> =
  N/2 - N_down on the solved state."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import lib_basis, olat, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reduced():
    spec = qi.disordered_open_square(8)
    lat = olat(spec)
    d = orc.binom(64, 3)
    v0 = qi.gaussian_start(11, d, False).astype(np.complex128)
    E, vec = orc.lanczos_ground(lambda p: orc.hphi_u1(lat, 3, p), v0, max_iter=200)
    r = orc.hphi_u1(lat, 3, vec) - E * vec
    assert np.linalg.norm(r) <= 1e-10 * abs(E)
    _, _, sz = orc.corr_u1(64, 3, vec)
    return spec, E, sz


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_reduced_disordered_ground_state_vs_oracle(reduced, prec):
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec, E, sz_ref = reduced
    b = lib_basis(spec, 3)
    o = qs3.SolveOpts(n_eig=1, n_keep=8, n_max=40, max_iter=5000, eps=1e-12, precision=prec, refine_tol=1e-10,
                      seed=3)
    e, v, info = b.trlanczos(o)
    assert info["status"] == "QS3_OK"
    assert abs(e[0, 0] - E) <= 1e-9 * abs(E)
    assert info["max_residual"] <= 1e-9 * abs(E)
    sz = b.correlations(v, local=True)["sz"]
    assert float(np.max(np.abs(sz - sz_ref))) <= 1e-8
    assert abs(sz.sum() - (32 - 3)) <= 1e-9


def test_full_size_disordered_ground_state():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.disordered_open_square(32)
    b = lib_basis(spec, 3)
    assert b.total_dim == 178_433_024
    res = {}
    for prec in ("f32", "f64"):
        o = qs3.SolveOpts(n_eig=1, n_keep=8, n_max=48, max_iter=20000, eps=1e-12, precision=prec,
                          refine_tol=1e-10, seed=7)
        e, v, info = b.trlanczos(o, vectors=(prec == "f32"))
        assert info["status"] == "QS3_OK"
        E = float(e[0, 0])
        assert info["max_residual"] <= 1e-9 * abs(E)
        res[prec] = (E, v)
    assert abs(res["f32"][0] - res["f64"][0]) <= 1e-9 * abs(res["f64"][0])
    sz = b.correlations(res["f32"][1], local=True)["sz"]
    torch.cuda.synchronize()
    assert abs(float(sz.sum()) - (1024 / 2 - 3)) <= 1e-6
    assert float(sz.max()) <= 0.5 + 1e-12 and float(sz.min()) >= -0.5 - 1e-12
