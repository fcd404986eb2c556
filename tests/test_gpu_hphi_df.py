"""The double-float product (QS3_C128DF): H applied to a vector held as
(re.hi, re.lo, im.hi, im.lo) floats, in error-free fp32 arithmetic.  It must
agree with the IEEE complex128 product to a few 2^-48 per term and with the
oracle's Alg. 9 to the fp64 bound, on the representative table and on the
representative search, with uniform and bond-dependent hop amplitudes, a
uniform field and states of every |Stab|; the split itself is exact IEEE
rounding; the fp64 solvers that use it agree with the IEEE ones."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, tol_hphi, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def j1j2_chain(N, J1, J2, Jz_ratio, h):
    """Periodic chain with nearest (J1) and next-nearest (J2) bonds, XXZ
    anisotropy Jz = Jz_ratio J and a uniform field h: two hop amplitudes."""
    bi = np.array([i for i in range(N)] * 2, np.int32)
    bj = np.array([(i + 1) % N for i in range(N)] + [(i + 2) % N for i in range(N)], np.int32)
    jxy = np.array([J1] * N + [J2] * N, float)
    return qi.LatticeSpec(N, bi, bj, jxy, Jz_ratio * jxy, np.full(N, h), (N, 1, 1), f"j1j2_{N}")


def aniso_square(Lx, Ly, Jx, Jy, Jz):
    """Periodic square lattice with hop amplitude Jx on x bonds, Jy on y bonds."""
    s = qi.hypercubic((Lx, Ly, 1), J=1.0, Jz=Jz)
    dx = (s.bj - s.bi) % Lx != 0
    s.jxy = np.where(dx, Jx, Jy).astype(float)
    return s


CASES = [
    ("square6_nd3", lambda: qi.square(6), 3),
    ("chain12_nd4_stab", lambda: qi.chain(12, Jz=0.7), 4),
    ("cube3_nd3", lambda: qi.cubic(3, Jz=0.8), 3),
    ("j1j2_chain14_nd4_field", lambda: j1j2_chain(14, 1.0, 0.45, 0.8, 0.3), 4),
    ("aniso_square5x4_nd3", lambda: aniso_square(5, 4, 1.0, 0.6, 0.9), 3),
    ("triangular4x4_nd2", lambda: qi.triangular(4, 4, J=1.0, Jz=1.1), 2),
]

# per term a few 2^-48 relative (splits of phi, phase, coupling; dropped lo*lo)
DF_REL = 2.0 ** -44


@pytest.mark.parametrize("table", [True, False], ids=["table", "search"])
@pytest.mark.parametrize("name,make,nd", CASES, ids=[c[0] for c in CASES])
def test_df_product(name, make, nd, table):
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = make()
    Ks = qi.all_k(spec.L)
    b = lib_basis(spec, nd, Ks)
    if not table:
        b.rep_table(0)
    x = gaussian(41, b.total_dim, True)
    phi = to_dev(x, torch.complex128)
    ref = b.hphi(phi)
    got = b.hphi_df(qs3.split_df(phi))
    again = b.hphi_df(qs3.split_df(phi))
    torch.cuda.synchronize()
    assert torch.equal(got, again)                     # deterministic: no atomics
    m = float(np.max(np.abs(x)))
    row_weight = 16.0
    assert float((got - ref).abs().max()) <= DF_REL * m * row_weight
    out = got.cpu().numpy()
    for s, K in enumerate(Ks):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        if hi > lo:
            sec = orc.mk_list(olat(spec), nd, K)
            assert np.max(np.abs(out[lo:hi] - orc.hphi_k(sec, x[lo:hi]))) <= tol_hphi(x[lo:hi], False), K


def test_split_is_ieee_rounding():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(10007) * np.exp(rng.uniform(-30, 30, 10007))
         + 1j * rng.standard_normal(10007) * np.exp(rng.uniform(-30, 30, 10007)))
    x[:4] = [0.0, 1.0, -2.5 + 1e-300j, 1e-40 - 1e-40j]
    got = qs3.split_df(to_dev(x, torch.complex128)).cpu().numpy().reshape(-1, 4)
    want = np.empty((len(x), 4), np.float32)
    for c, part in enumerate((x.real, x.imag)):
        hi = part.astype(np.float32)
        want[:, 2 * c] = hi
        want[:, 2 * c + 1] = (part - hi.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    # hi + lo carries 48 bits of the normal-range values
    nrm = (np.abs(x.real) > 1e-30) & (np.abs(x.real) < 1e30)
    back = got[:, 0].astype(np.float64) + got[:, 1].astype(np.float64)
    assert np.all(np.abs(back - x.real)[nrm] <= 2.0 ** -47 * np.abs(x.real)[nrm])


def test_df_edge_bases():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    # N_down = 0: H = c0 on the single all-up state of the k = 0 sector
    b0 = lib_basis(qi.chain(8, Jz=0.6), 0, qi.all_k((8, 1, 1)))
    x = to_dev(gaussian(3, b0.total_dim, True), torch.complex128)
    got, ref = b0.hphi_df(qs3.split_df(x)), b0.hphi(x)
    assert float((got - ref).abs().max()) <= 1e-14
    # an empty sector list entry and a U(1)-only basis
    u1 = lib_basis(qi.chain(10), 3)
    with pytest.raises(qs3.QS3Error):
        u1.hphi_df(torch.zeros(4 * u1.total_dim, dtype=torch.float32, device="cuda"))
    # sectors with no compatible representative (dimension 0) next to others
    b = lib_basis(qi.chain(8), 4, [(1, 0, 0), (2, 0, 0), (4, 0, 0)])
    x = to_dev(gaussian(5, b.total_dim, True), torch.complex128)
    assert float((b.hphi_df(qs3.split_df(x)) - b.hphi(x)).abs().max()) <= DF_REL * 16


@pytest.mark.parametrize("solver", ["lanczos", "trl"])
def test_solvers_df_vs_ieee(solver):
    """The double-float engine (precision "df", with its double-float or its
    IEEE H Phi) against the binary64 engine (precision "f64")."""
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.square(6)
    Ks = [(0, 0, 0), (1, 2, 0), (3, 3, 0), (2, 0, 0)]
    b = lib_basis(spec, 3, Ks)
    res = {}
    for mode in ("f64", "df", "df_ieee_hphi"):
        prec = "f64" if mode == "f64" else "df"
        ieee = mode == "df_ieee_hphi"
        if solver == "lanczos":
            o = qs3.SolveOpts(n_max=150, eps=1e-14, res_tol=1e-12, precision=prec, hphi_ieee=ieee)
            e, _, info = b.lanczos(o, vectors=False)
        else:
            o = qs3.SolveOpts(n_eig=3, n_keep=8, n_max=32, eps=1e-13, precision=prec, hphi_ieee=ieee)
            e, _, info = b.trlanczos(o, vectors=False)
        assert info["status"] == "QS3_OK"
        assert info["max_residual"] <= 1e-10
        res[mode] = e
    scale = float(np.max(np.abs(res["f64"])))
    for mode in ("df", "df_ieee_hphi"):
        assert float(np.max(np.abs(res[mode] - res["f64"]))) <= 1e-12 * scale
    # the lowest level of each sector against the oracle (higher TRL levels
    # may skip a copy of a point-group degenerate level: one start vector)
    for s, K in enumerate(Ks):
        w = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(spec), 3, K)))
        for mode in res:
            assert abs(res[mode][s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))
