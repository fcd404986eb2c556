"""The binary64 engine's H Phi on the integer units (QS3_C128X): each hop's
phase x phi formed exactly on fixed-point images and summed exactly per row.
Against the oracle's Alg. 9 on every sector (lattices with non-trivial
stabilisers, ragged chunks, vectors over many binades), against the binary64
FMA product, in the solver (strict64 off and on), and its limits."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests.gpu_common import gaussian, lib_basis, olat, tol_hphi, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ("chain12_nd3", (12, 1, 1), 3),
    ("chain8_nd4", (8, 1, 1), 4),
    ("square4_nd4", (4, 4, 1), 4),
    ("square6x4_nd3", (6, 4, 1), 3),
    ("cube3_nd3", (3, 3, 3), 3),
    ("square8_nd3", (8, 8, 1), 3),
]


def _vector(seed, d, kind):
    x = gaussian(seed, d, True)
    if kind == "binades":          # magnitudes over 40 binades
        rng = np.random.default_rng(seed)
        x = x * 2.0 ** rng.uniform(-40, 0, d)
    x /= np.linalg.norm(x)
    return x


@pytest.mark.parametrize("name,dims,nd", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["gauss", "binades"])
def test_integer_hphi_vs_oracle(name, dims, nd, kind):
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=0.7)
    K = qi.all_k(dims)
    b = lib_basis(spec, nd, K)
    phi_h = _vector(11, b.total_dim, kind)
    phi = to_dev(phi_h, torch.complex128)
    xi = b.hphi(phi, integer=True)
    fm = b.hphi(phi)
    torch.cuda.synchronize()
    out = xi.cpu().numpy()
    # the binary64 FMA product: the same terms, within a few roundings
    assert np.max(np.abs(out - fm.cpu().numpy())) <= 1e-13 * np.max(np.abs(phi_h)) * 16
    for i, k in enumerate(K):
        sec = orc.mk_list(olat(spec), nd, k)
        lo, hi = b.offsets[i], b.offsets[i + 1]
        ref = orc.hphi_k(sec, phi_h[lo:hi])
        tol = tol_hphi(phi_h[lo:hi], False)
        assert np.max(np.abs(out[lo:hi] - ref), initial=0.0) <= tol, (name, k)


def test_integer_hphi_full_size_square10_nd4():
    """All 100 momenta of the 10x10, N_down = 4 workload (3,921,225 rows)
    against the binary64 FMA product, and sampled rows against the oracle."""
    torch = torch_cuda()
    spec = qi.square(10)
    K = qi.all_k((10, 10, 1))
    b = lib_basis(spec, 4, K)
    phi_h = _vector(5, b.total_dim, "gauss")
    phi = to_dev(phi_h, torch.complex128)
    xi = b.hphi(phi, integer=True).cpu().numpy()
    fm = b.hphi(phi).cpu().numpy()
    scale = np.max(np.abs(phi_h))
    assert np.max(np.abs(xi - fm)) <= 16e-13 * scale
    for s in (0, 37, 99):
        sec = orc.mk_list(olat(spec), 4, K[s])
        lo, hi = b.offsets[s], b.offsets[s + 1]
        rows = np.random.default_rng(s).choice(hi - lo, 64, replace=False)
        ref = orc.hphi_k_rows(sec, phi_h[lo:hi], rows)
        assert np.max(np.abs(xi[lo:hi][rows] - ref)) <= tol_hphi(phi_h[lo:hi], False)


def test_integer_hphi_in_the_solver():
    """The binary64 engine uses the integer product unless strict64: both
    solves match the oracle's dense spectrum and each other."""
    torch_cuda()
    import paper_2107_00872_gb300 as qs3
    spec = qi.square(6)
    Ks = [(0, 0, 0), (1, 2, 0), (3, 3, 0)]
    b = lib_basis(spec, 3, Ks)
    e = {}
    for strict in (False, True):
        o = qs3.SolveOpts(n_max=200, eps=1e-14, res_tol=1e-12, precision="f64", strict64=strict)
        ev, _, info = b.lanczos(o, vectors=False)
        assert info["status"] == "QS3_OK"
        assert info["max_residual"] <= 1e-11 * max(1.0, float(np.max(np.abs(ev))))
        e[strict] = ev
    assert float(np.max(np.abs(e[False] - e[True]))) <= 1e-13 * float(np.max(np.abs(e[True])))
    for s, K in enumerate(Ks):
        w = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(spec), 3, K)))
        assert abs(e[False][s, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


def test_integer_hphi_limits():
    torch = torch_cuda()
    import dataclasses
    import paper_2107_00872_gb300 as qs3
    # U(1)-only basis: no k-sector table
    u1 = lib_basis(qi.chain(10), 3)
    with pytest.raises(qs3.QS3Error):
        u1.hphi(torch.zeros(u1.total_dim, dtype=torch.complex128, device="cuda"), integer=True)
    # without the representative table
    kb = lib_basis(qi.chain(10), 3, [(0, 0, 0)])
    kb.rep_table(0)
    with pytest.raises(qs3.QS3Error):
        kb.hphi(torch.zeros(kb.total_dim, dtype=torch.complex128, device="cuda"), integer=True)
    with pytest.raises(TypeError):
        kb.hphi(torch.zeros(kb.total_dim, dtype=torch.complex64, device="cuda"), integer=True)
    # bond-dependent J^xy (translation invariant: J along x, 0.5 J along y)
    sq = qi.square(4)
    along_y = (sq.bj - sq.bi) % 4 == 0
    aniso = dataclasses.replace(sq, jxy=np.where(along_y, 0.5, 1.0))
    ab = lib_basis(aniso, 2, [(1, 0, 0)])
    with pytest.raises(qs3.QS3Error):
        ab.hphi(torch.zeros(ab.total_dim, dtype=torch.complex128, device="cuda"), integer=True)
    # the solver falls back to the binary64 product there and still matches the oracle
    e, _, info = ab.lanczos(qs3.SolveOpts(n_max=120, eps=1e-14, res_tol=1e-12, precision="f64"), vectors=False)
    assert info["status"] == "QS3_OK"
    w = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(olat(aniso), 2, (1, 0, 0))))
    assert abs(e[0, 0] - w[0]) <= 1e-12 * max(1.0, abs(w[0]))


@pytest.mark.parametrize("name,dims,nd", [("square6_nd3", (6, 6, 1), 3), ("chain12_nd4", (12, 1, 1), 4),
                                          ("cube3_nd3", (3, 3, 3), 3)])
def test_orbit_batched_equals_per_sector(name, dims, nd):
    """A basis of several momenta runs the orbit-batched kernel (each orbit's
    hops listed once for a group of sectors); one-sector bases run the
    per-row kernel.  The integer row sums are exact and the binary64 terms
    come in the same order, so the outputs agree bit for bit."""
    torch = torch_cuda()
    spec = qi.hypercubic(dims, J=1.0, Jz=0.6)
    K = qi.all_k(dims)
    b = lib_basis(spec, nd, K)
    phi_h = _vector(3, b.total_dim, "binades")
    multi = b.hphi(to_dev(phi_h, torch.complex128), integer=True).cpu().numpy()
    for s, k in enumerate(K):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        one = lib_basis(spec, nd, [k])
        got = one.hphi(to_dev(phi_h[lo:hi], torch.complex128), integer=True).cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint64), multi[lo:hi].view(np.uint64))
