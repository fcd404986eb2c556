"""Pins of the CPU oracle against values and constructions that do not come
from the oracle itself: the paper's worked example and quoted dimensions,
brute-force enumerations, Eq. (1) built from Kronecker products, closed forms
and exact identities of the symmetry-adapted basis."""
from __future__ import annotations

import os
from math import comb

import numpy as np
import pytest

import oracle as orc
import qs3_inputs as qi
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def olat(spec: qi.LatticeSpec) -> orc.Lattice:
    return orc.Lattice(**spec.as_dict())


def read_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [int(x) for x in v]
    return out


# ------------------------------------------------------------ Eq. a_of_n, Alg 1


def test_worked_example_fbar():
    g = read_kv("fbar_worked_example.txt")
    N, nd = g["N"][0], g["Nd"][0]
    assert orc.F(N, g["n"]) == g["a"][0]
    n, trace = orc.f_bar(N, nd, g["a"][0])
    assert n == g["n"]
    assert trace == g["trace"]


@pytest.mark.parametrize("N,nd", [(1, 1), (5, 0), (6, 1), (7, 3), (9, 4), (10, 5), (12, 6), (12, 12), (13, 2)])
def test_rank_is_colex_position(N, nd):
    subs = pins.colex_subsets(N, nd)
    assert orc.binom(N, nd) == len(subs) == comb(N, nd)
    for k, c in enumerate(subs):
        n1 = [s + 1 for s in c]
        assert orc.F(N, n1) == k + 1
        assert orc.f_bar(N, nd, k + 1)[0] == n1
    if nd:
        lists = orc.unrank_all(N, nd)
        assert [tuple(r) for r in lists] == subs


def test_rank_large_values():
    # C(1000,4) and C(1024,3): ranks beyond 2^32 survive the round trip
    for N, nd in ((1000, 4), (1024, 3), (100, 8)):
        D = orc.binom(N, nd)
        assert D == comb(N, nd)
        rng = np.random.default_rng(N)
        for _ in range(200):
            c = sorted(rng.choice(N, nd, replace=False) + 1)
            a = orc.F(N, c)
            expect = 1 + sum(comb(int(c[m]) - 1, m + 1) for m in range(nd))
            assert a == expect
            assert orc.f_bar(N, nd, a)[0] == [int(x) for x in c]
    assert orc.binom(200, 100) == 0          # beyond 2^63: reported as overflow


def test_spin_exchange_matches_set_moves():
    rng = np.random.default_rng(7)
    N, nd = 15, 4
    for _ in range(300):
        c = sorted(int(x) for x in rng.choice(N, nd, replace=False) + 1)
        r, rp = sorted(int(x) for x in rng.choice(N, 2, replace=False) + 1)
        got = orc.spin_exchange_index(N, c, r, rp)
        inr, inrp = r in c, rp in c
        if inr == inrp:
            assert got == 0
            continue
        new = set(c) ^ {r, rp}
        assert got == orc.F(N, sorted(new))
        assert got == pins.colex_subsets(N, nd).index(tuple(s - 1 for s in sorted(new))) + 1


# --------------------------------------------------------------- Eq. (1), Alg 4


@pytest.mark.parametrize("seed", [1, 2])
def test_dense_u1_equals_kronecker_hamiltonian(seed):
    spec = qi.random_graph(7, 11, seed)
    Hfull = pins.kron_hamiltonian(spec)
    for nd in range(0, 8):
        P = pins.sector_projector(7, nd)
        Hk = (P.T @ Hfull @ P)
        assert np.abs(Hk.imag).max() < 1e-14
        Ho = orc.dense_u1(olat(spec), nd)
        np.testing.assert_allclose(Ho, Hk.real, atol=1e-13, rtol=0)
        # the full space is block diagonal in N_down (U(1) symmetry of Eq. (1))
    mask = np.zeros_like(Hfull, dtype=bool)
    for nd in range(8):
        P = pins.sector_projector(7, nd).astype(bool)
        idx = np.where(P.any(1))[0]
        mask[np.ix_(idx, idx)] = True
    assert np.abs(Hfull[~mask]).max() == 0


def test_dense_u1_bit_construction_chain16():
    spec = qi.chain(16)
    for nd in (1, 2, 3):
        np.testing.assert_allclose(orc.dense_u1(olat(spec), nd), pins.bit_hamiltonian_sector(spec, nd),
                                   atol=1e-13, rtol=0)


def test_hphi_u1_matches_dense():
    spec = qi.disordered_open_square(5, seed=3)
    lat = olat(spec)
    for nd in (1, 3):
        H = orc.dense_u1(lat, nd)
        x = qi.gaussian_start(11, H.shape[0], True)
        np.testing.assert_allclose(orc.hphi_u1(lat, nd, x), H @ x, atol=1e-12, rtol=0)
        rows = np.array([0, 3, H.shape[0] - 1])
        np.testing.assert_allclose(orc.hphi_u1_rows(lat, nd, x, rows), (H @ x)[rows], atol=1e-12, rtol=0)


def test_one_and_two_magnon_chain_against_closed_forms():
    N = 16
    spec = qi.chain(N)
    H1 = orc.dense_u1(olat(spec), 1)
    e1 = np.sort(np.linalg.eigvalsh(H1))
    expect = np.sort([pins.one_magnon_energy(spec, (k, 0, 0)) for k in range(N)])
    np.testing.assert_allclose(e1, expect, atol=1e-12)
    # two magnons: block of Eq. (1) built on bit strings (independent construction)
    H2 = orc.dense_u1(olat(spec), 2)
    np.testing.assert_allclose(np.linalg.eigvalsh(H2), np.linalg.eigvalsh(pins.bit_hamiltonian_sector(spec, 2)),
                               atol=1e-12)


@pytest.mark.parametrize("N,Jz", [(15, 1.0), (13, 0.6), (11, -0.5), (9, 2.0)])
def test_two_magnon_chain_against_two_body_problem(N, Jz):
    """The oracle's N_down = 2 block of the periodic XXZ chain against the
    two-body problem in the relative coordinate (total momentum conserved,
    hard-core nearest-neighbour pair): every one of the C(N, 2) levels."""
    spec = qi.chain(N, J=1.0, Jz=Jz)
    e = np.sort(np.linalg.eigvalsh(orc.dense_u1(olat(spec), 2)))
    np.testing.assert_allclose(e, pins.two_magnon_chain_spectrum(N, 1.0, Jz), atol=1e-12, rtol=0)


# ------------------------------------------------------- Alg 5-7, dimensions


@pytest.mark.parametrize("dims,nd", [((12, 1, 1), 3), ((12, 1, 1), 4), ((8, 1, 1), 4), ((4, 3, 1), 3),
                                     ((4, 4, 1), 4), ((3, 3, 2), 3), ((6, 1, 1), 0), ((6, 1, 1), 6)])
def test_sector_dims_closed_form_and_sum(dims, nd):
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    N = spec.n_sites
    total = 0
    for K in qi.all_k(dims):
        sec = orc.mk_list(lat, nd, K)
        assert sec.dim == pins.sector_dim_closed_form(dims, nd, K)
        total += sec.dim
    assert total == comb(N, nd)


def test_paper_dimensions_by_closed_form():
    for line in open(os.path.join(GOLDEN, "paper_dims.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, Lx, Ly, Lz, nd, val = line.split()
        L = (int(Lx), int(Ly), int(Lz))
        N = L[0] * L[1] * L[2]
        if kind == "U1":
            assert orc.binom(N, int(nd)) == int(val)
        else:
            assert pins.sector_dim_closed_form(L, int(nd), (0, 0, 0)) == int(val)


def test_representatives_are_orbit_minima():
    dims = (4, 3, 1)
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    nd = 3
    subs = pins.colex_subsets(12, nd)
    index = {c: k + 1 for k, c in enumerate(subs)}
    for K in qi.all_k(dims):
        sec = orc.mk_list(lat, nd, K)
        reps = set(int(a) for a in sec.sigma1)
        for c in subs:
            orb = {pins.translate_set(c, t, dims) for t in pins.group(dims)}
            rep = min(index[o] for o in orb)
            stab = sum(1 for t in pins.group(dims) if pins.translate_set(c, t, dims) == c)
            compat = all(abs(np.exp(2j * np.pi * sum(K[a] * t[a] / dims[a] for a in range(3))) - 1) < 1e-9
                         for t in pins.group(dims) if pins.translate_set(c, t, dims) == c)
            a = index[c]
            r, l = orc.representative(lat, nd, a)
            assert r == rep
            assert index[pins.translate_set(c, l, dims)] == rep
            assert (a in reps) == (a == rep and compat)
            if a in reps:
                i = list(sec.sigma1).index(a)
                assert sec.stab[i] == stab
                assert abs(sec.Nak[i] - 12 * stab) < 1e-9
        assert list(sec.sigma1) == sorted(sec.sigma1)


@pytest.mark.parametrize("name,nd", [("honeycomb3x2", 3), ("kagome2x2", 3), ("kagome2x2", 4), ("honeycomb2x2", 2)])
def test_multi_spin_cells_dims_and_representatives(name, nd):
    """Lattices with several spins per unit cell: translations move cells,
    each spin keeps its place in the cell.  Sector dimensions against the
    character sum over the cell group (and their total, C(N, nd)); every
    representative is the minimum of its orbit under the cell translations,
    with its stabiliser, compatibility and N_{a,k} = (number of cells) |Stab|."""
    spec = {"honeycomb3x2": qi.honeycomb(3, 2), "kagome2x2": qi.kagome(2, 2),
            "honeycomb2x2": qi.honeycomb(2, 2)}[name]
    L, ns, N = spec.L, spec.n_sub, spec.n_sites
    G = L[0] * L[1] * L[2]
    lat = olat(spec)
    subs = pins.colex_subsets(N, nd)
    index = {c: k + 1 for k, c in enumerate(subs)}
    total = 0
    for K in qi.all_k(L):
        sec = orc.mk_list(lat, nd, K)
        assert sec.dim == pins.sector_dim_closed_form(L, nd, K, ns)
        total += sec.dim
        reps = set(int(a) for a in sec.sigma1)
        for c in subs:
            orb = {pins.translate_set(c, t, L, ns) for t in pins.group(L)}
            rep = min(index[o] for o in orb)
            fix = [t for t in pins.group(L) if pins.translate_set(c, t, L, ns) == c]
            compat = all(abs(np.exp(2j * np.pi * sum(K[a] * t[a] / L[a] for a in range(3))) - 1) < 1e-9 for t in fix)
            a = index[c]
            r, l = orc.representative(lat, nd, a)
            assert r == rep and index[pins.translate_set(c, l, L, ns)] == rep
            assert (a in reps) == (a == rep and compat)
            if a in reps:
                i = list(sec.sigma1).index(a)
                assert sec.stab[i] == len(fix)
                assert abs(sec.Nak[i] - G * len(fix)) < 1e-9
    assert total == comb(N, nd)


@pytest.mark.parametrize("name,nd,anis", [("honeycomb3x2", 3, 1.0), ("kagome2x2", 3, 0.6), ("kagome2x2", 4, 1.0)])
def test_multi_spin_cells_dense_k_unfolds_and_spectra_union(name, nd, anis):
    """The k-blocks of a multi-spin-cell lattice: Hermitian, H_U U_k = U_k H_k
    with U_k^H U_k = I, and the union of their spectra equals the spectrum of
    the N_down block built on bit strings (no translations involved)."""
    spec = {"honeycomb3x2": qi.honeycomb(3, 2, Jz=anis), "kagome2x2": qi.kagome(2, 2, Jz=anis)}[name]
    lat = olat(spec)
    HU = orc.dense_u1(lat, nd)
    np.testing.assert_allclose(np.linalg.eigvalsh(HU), np.linalg.eigvalsh(pins.bit_hamiltonian_sector(spec, nd)),
                               atol=1e-12)
    eig_all = []
    for K in qi.all_k(spec.L):
        sec = orc.mk_list(lat, nd, K)
        if sec.dim == 0:
            continue
        Hk = orc.dense_k(sec)
        np.testing.assert_allclose(Hk, Hk.conj().T, atol=1e-13)
        U = _unfold_matrix(sec)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(sec.dim), atol=1e-12)
        np.testing.assert_allclose(HU @ U, U @ Hk, atol=1e-12)
        eig_all.append(np.linalg.eigvalsh(Hk))
    np.testing.assert_allclose(np.sort(np.concatenate(eig_all)), np.linalg.eigvalsh(HU), atol=1e-11)


# ----------------------------------------------------------- Alg 8 / 9, Eq.


def _unfold_matrix(sec):
    d = sec.dim
    return np.stack([orc.unfold(sec, np.eye(d)[i]) for i in range(d)], 1)


@pytest.mark.parametrize("dims,nd", [((12, 1, 1), 3), ((4, 3, 1), 3), ((3, 3, 2), 2)])
def test_unfolded_states_are_translation_eigenstates(dims, nd):
    """|a,k> of Eq. (akstate): unit norm, orthogonal, T|a,k> = e^{ik}|a,k>."""
    spec = qi.hypercubic(dims)
    subs = pins.colex_subsets(spec.n_sites, nd)
    index = {c: k for k, c in enumerate(subs)}
    for K in qi.all_k(dims)[:5]:
        sec = orc.mk_list(olat(spec), nd, K)
        U = _unfold_matrix(sec)
        np.testing.assert_allclose(U.conj().T @ U, np.eye(sec.dim), atol=1e-12)
        for a in range(3):
            if dims[a] == 1:
                continue
            t = [0, 0, 0]
            t[a] = 1
            perm = [index[pins.translate_set(c, t, dims)] for c in subs]
            TU = np.zeros_like(U)
            TU[perm, :] = U
            ph = np.exp(2j * np.pi * K[a] / dims[a])
            np.testing.assert_allclose(TU, ph * U, atol=1e-12)


@pytest.mark.parametrize("dims,nd,anis", [((12, 1, 1), 3, 1.0), ((4, 3, 1), 3, 0.7), ((3, 3, 2), 3, 1.3),
                                          ((5, 3, 1), 2, 0.5)])
def test_dense_k_hermitian_unfolds_and_spectra_union(dims, nd, anis):
    spec = qi.hypercubic(dims, J=1.0, Jz=anis)
    lat = olat(spec)
    HU = orc.dense_u1(lat, nd)
    eig_all = []
    for K in qi.all_k(dims):
        sec = orc.mk_list(lat, nd, K)
        if sec.dim == 0:
            continue
        Hk = orc.dense_k(sec)
        np.testing.assert_allclose(Hk, Hk.conj().T, atol=1e-13)
        U = _unfold_matrix(sec)
        np.testing.assert_allclose(HU @ U, U @ Hk, atol=1e-12)
        x = qi.gaussian_start(5, sec.dim, True)
        np.testing.assert_allclose(orc.hphi_k(sec, x), Hk @ x, atol=1e-12)
        rows = np.arange(0, sec.dim, 3)
        np.testing.assert_allclose(orc.hphi_k_rows(sec, x, rows), (Hk @ x)[rows], atol=1e-12)
        eig_all.append(np.linalg.eigvalsh(Hk))
    np.testing.assert_allclose(np.sort(np.concatenate(eig_all)), np.linalg.eigvalsh(HU), atol=1e-11)


@pytest.mark.parametrize("dims", [(10, 1, 1), (5, 4, 1), (4, 3, 3)])
def test_one_magnon_dispersion_k_sectors(dims):
    spec = qi.hypercubic(dims, J=1.0, Jz=0.8)
    for K in qi.all_k(dims):
        sec = orc.mk_list(olat(spec), 1, K)
        assert sec.dim == 1
        E = orc.dense_k(sec)[0, 0].real
        assert abs(E - pins.one_magnon_energy(spec, K)) < 1e-12


def test_su2_descent_isotropic():
    """Isotropic Eq. (1): spec(N_down-1, k) is contained in spec(N_down, k)."""
    dims = (4, 3, 1)
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    for K in qi.all_k(dims)[:6]:
        e3 = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(lat, 3, K)))
        e2 = np.linalg.eigvalsh(orc.dense_k(orc.mk_list(lat, 2, K)))
        for e in e2:
            assert np.min(np.abs(e3 - e)) < 1e-10


# --------------------------------------------------- Alg 10, correlations, CF


def test_lanczos_and_trl_lowest_eigenvalues_chain16():
    spec = qi.chain(16)
    lat = olat(spec)
    H = orc.dense_u1(lat, 3)
    ev = np.linalg.eigvalsh(H)
    v0 = qi.gaussian_start(1, H.shape[0], False).astype(np.complex128)
    E0, vec = orc.lanczos_ground(lambda x: orc.hphi_u1(lat, 3, x), v0, max_iter=200)
    assert abs(E0 - ev[0]) < 1e-12 * abs(ev[0])
    r = orc.hphi_u1(lat, 3, vec) - E0 * vec
    assert np.linalg.norm(r) < 1e-10
    e, vecs, it = orc.thick_restart_lanczos(lambda x: orc.hphi_u1(lat, 3, x), v0, 8, 32, 500, 1e-14)
    np.testing.assert_allclose(e[:4], ev[:4], atol=1e-11)


def test_trl_k_sector_square():
    spec = qi.square(4, 3)
    lat = olat(spec)
    sec = orc.mk_list(lat, 4, (1, 0, 0))
    ev = np.linalg.eigvalsh(orc.dense_k(sec))
    v0 = qi.gaussian_start(2, sec.dim, True)
    e, vecs, it = orc.thick_restart_lanczos(lambda x: orc.hphi_k(sec, x), v0, 6, 20, 500, 1e-14)
    np.testing.assert_allclose(e[:4], ev[:4], atol=1e-10)


def test_correlations_against_kronecker_operators():
    spec = qi.random_graph(7, 10, 4)
    Hfull = pins.kron_hamiltonian(spec)
    nd = 3
    P = pins.sector_projector(7, nd)
    rng = np.random.default_rng(0)
    phi = rng.normal(size=P.shape[1]) + 1j * rng.normal(size=P.shape[1])
    phi /= np.linalg.norm(phi)
    full = P @ phi
    szsz, spsm, sz = orc.corr_u1(7, nd, phi)
    s_p = np.array([[0, 1], [0, 0]])        # s^+ raises: |down> -> |up>
    s_m = s_p.T
    szm = np.diag([0.5, -0.5])
    eye = np.eye(2)

    def op(m):
        out = np.array([[1.0 + 0j]])
        for i in reversed(range(7)):
            out = np.kron(out, m.get(i, eye))
        return out
    for i in range(7):
        assert abs(sz[i] - np.vdot(full, op({i: szm}) @ full).real) < 1e-12
        for j in range(7):
            zz = np.vdot(full, op({i: szm}) @ op({j: szm}) @ full) if i != j else np.vdot(full, op({i: szm @ szm}) @ full)
            assert abs(szsz[i, j] - zz.real) < 1e-12
            pm = np.vdot(full, op({i: s_p}) @ op({j: s_m}) @ full) if i != j else np.vdot(full, op({i: s_p @ s_m}) @ full)
            assert abs(spsm[i, j] - pm) < 1e-12
    del Hfull


def _smq_dense_u1(N, nd, phi_u, Q, L):
    """S^-_q = N^{-1/2} sum_r e^{-iq.r} s^-_r applied on colex-ordered sets."""
    src = pins.colex_subsets(N, nd)
    dst = {c: k for k, c in enumerate(pins.colex_subsets(N, nd + 1))}
    out = np.zeros(len(dst), np.complex128)
    for k, c in enumerate(src):
        for r in range(N):
            if r in c:
                continue
            x, y, z = pins.coords(r, L)
            qr = 2 * np.pi * (Q[0] * x / L[0] + Q[1] * y / L[1] + Q[2] * z / L[2])
            out[dst[tuple(sorted(c + (r,)))]] += np.exp(-1j * qr) * phi_u[k] / np.sqrt(N)
    return out


@pytest.mark.parametrize("dims,nd", [((12, 1, 1), 2), ((4, 3, 1), 2), ((3, 3, 2), 1)])
def test_smq_push_form_against_definition(dims, nd):
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    N = spec.n_sites
    for K in qi.all_k(dims)[:3]:
        src = orc.mk_list(lat, nd, K)
        phi = qi.gaussian_start(3, src.dim, True)
        for Q in qi.all_k(dims)[:4]:
            K2 = tuple((K[a] + Q[a]) % dims[a] for a in range(3))
            dst = orc.mk_list(lat, nd + 1, K2)
            got = orc.smq(src, phi, Q, dst)
            want = orc.fold(dst, _smq_dense_u1(N, nd, orc.unfold(src, phi), Q, dims))
            np.testing.assert_allclose(got, want, atol=1e-12)


def test_smq_on_vacuum_has_unit_norm():
    dims = (4, 3, 1)
    lat = olat(qi.hypercubic(dims))
    vac = orc.mk_list(lat, 0, (0, 0, 0))
    assert vac.dim == 1
    for Q in qi.all_k(dims):
        dst = orc.mk_list(lat, 1, Q)
        v = orc.smq(vac, np.ones(1, np.complex128), Q, dst)
        assert abs(np.vdot(v, v).real - 1.0) < 1e-13


def test_continued_fraction_equals_lorentzian_sum():
    """Eq. (cfe) with a full Lanczos run equals the spectral sum of the
    resolvent built from a dense eigendecomposition; the weights sum to the
    static factor |S_q phi|^2 (sum rule)."""
    dims = (8, 1, 1)
    spec = qi.hypercubic(dims)
    lat = olat(spec)
    gs_sec = None
    best = None
    for K in qi.all_k(dims):
        sec = orc.mk_list(lat, 2, K)
        e, v = np.linalg.eigh(orc.dense_k(sec))
        if best is None or e[0] < best[0] - 1e-12:
            best, gs_sec = (e[0], v[:, 0]), sec
    E0, phi = best
    Q = (3, 0, 0)
    K2 = tuple((gs_sec.K[a] + Q[a]) % dims[a] for a in range(3))
    dst = orc.mk_list(lat, 3, K2)
    v = orc.smq(gs_sec, phi, Q, dst)
    norm2 = np.vdot(v, v).real
    Hd = orc.dense_k(dst)
    alpha, beta, Psi, b0 = orc.lanczos(lambda x: Hd @ x, v, 200)
    assert abs(b0 ** 2 - norm2) < 1e-13
    omega = np.linspace(-2, 6, 801)
    h, eta = 1.5, 0.05
    s_cf = orc.continued_fraction(alpha, beta, norm2, omega, E0, eta, shift=h)
    en, U = np.linalg.eigh(Hd)
    w = np.abs(U.conj().T @ v) ** 2
    s_ex = sum(w[n] * (eta / np.pi) / ((omega + E0 - h - en[n]) ** 2 + eta ** 2) for n in range(len(en)))
    np.testing.assert_allclose(s_cf, s_ex, atol=1e-10 * s_ex.max())
    T = orc.tridiag(alpha, beta[:-1])
    eT, C = np.linalg.eigh(T)
    assert abs(norm2 * (C[0] ** 2).sum() - norm2) < 1e-12
    # weights at the poles equal the spectral weights
    assert abs((norm2 * C[0] ** 2).max() - w.max()) < 1e-10


def test_row_terms_without_sigma_equal_dense_rows():
    """The list-free row of Alg. 9 (Alg. 7 and Alg. 5 per hop target) equals
    the corresponding row of the dense Alg. 8 matrix."""
    for dims, nd, K in (((4, 3, 1), 3, (1, 2, 0)), ((3, 3, 2), 3, (0, 1, 1)), ((8, 1, 1), 3, (3, 0, 0))):
        spec = qi.hypercubic(dims, Jz=0.7)
        lat = olat(spec)
        sec = orc.mk_list(lat, nd, K)
        H = orc.dense_k(sec)
        index = {int(a): i for i, a in enumerate(sec.sigma1)}
        for i, a in enumerate(sec.sigma1):
            dg, tgt, cf = orc.row_terms_k(lat, nd, K, int(a))
            row = np.zeros(sec.dim, complex)
            row[i] += dg
            for t, c in zip(tgt, cf):
                row[index[int(t)]] += c
            np.testing.assert_allclose(row, H[i], atol=1e-13)
            assert abs(orc.check_state(lat, nd, K, int(a)) - sec.Nak[i]) < 1e-12
        # a non-representative is rejected
        a_non = next(a for a in range(1, orc.binom(spec.n_sites, nd) + 1) if a not in index)
        assert orc.row_terms_k(lat, nd, K, a_non) is None


# ------------------------------------------------ S^+_q and S^z_q (spsmsz 1, 3)

@pytest.mark.parametrize("dims,nd", [((8, 1, 1), 2), ((4, 3, 1), 2), ((3, 2, 2), 2)])
def test_sq_apply_sminus_equals_alg11(dims, nd):
    """The definition-based operator code reproduces Alg. 11 (the C push form)."""
    lat = olat(qi.hypercubic(dims))
    for K in qi.all_k(dims)[:2]:
        src = orc.mk_list(lat, nd, K)
        phi = qi.gaussian_start(9, src.dim, True)
        for Q in qi.all_k(dims)[:3]:
            dst = orc.mk_list(lat, nd + 1, tuple((K[a] + Q[a]) % dims[a] for a in range(3)))
            np.testing.assert_allclose(orc.sq_apply_k(src, phi, orc.OP_SMINUS, Q, dst), orc.smq(src, phi, Q, dst),
                                       atol=1e-12)


@pytest.mark.parametrize("dims,nd", [((8, 1, 1), 2), ((4, 3, 1), 2), ((3, 2, 2), 1)])
def test_splus_is_the_adjoint_of_sminus(dims, nd):
    """<chi, S^-_q phi> = <S^+_{-q} chi, phi>, with S^-_q from Alg. 11."""
    lat = olat(qi.hypercubic(dims))
    for K in qi.all_k(dims)[:2]:
        src = orc.mk_list(lat, nd, K)
        phi = qi.gaussian_start(4, src.dim, True)
        for Q in qi.all_k(dims)[:3]:
            K2 = tuple((K[a] + Q[a]) % dims[a] for a in range(3))
            dst = orc.mk_list(lat, nd + 1, K2)
            chi = qi.gaussian_start(5, dst.dim, True)
            mq = tuple((-Q[a]) % dims[a] for a in range(3))
            lhs = np.vdot(chi, orc.smq(src, phi, Q, dst))
            rhs = np.vdot(orc.sq_apply_k(dst, chi, orc.OP_SPLUS, mq, src), phi)
            assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs)), (K, Q)


@pytest.mark.parametrize("dims,nd", [((8, 1, 1), 3), ((4, 3, 1), 2)])
def test_sz_adjoint_and_zero_momentum(dims, nd):
    """(S^z_q)^dag = S^z_{-q}, and S^z_{q=0} phi = (N/2 - N_down) N^{-1/2} phi."""
    lat = olat(qi.hypercubic(dims))
    N = lat.n_sites
    for K in qi.all_k(dims)[:2]:
        src = orc.mk_list(lat, nd, K)
        phi = qi.gaussian_start(6, src.dim, True)
        np.testing.assert_allclose(orc.sq_apply_k(src, phi, orc.OP_SZ, (0, 0, 0), src),
                                   (N / 2 - nd) / np.sqrt(N) * phi, atol=1e-12)
        for Q in qi.all_k(dims)[1:3]:
            K2 = tuple((K[a] + Q[a]) % dims[a] for a in range(3))
            dst = orc.mk_list(lat, nd, K2)
            chi = qi.gaussian_start(7, dst.dim, True)
            mq = tuple((-Q[a]) % dims[a] for a in range(3))
            lhs = np.vdot(chi, orc.sq_apply_k(src, phi, orc.OP_SZ, Q, dst))
            rhs = np.vdot(orc.sq_apply_k(dst, chi, orc.OP_SZ, mq, src), phi)
            assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs)), (K, Q)


def test_sq_sum_rules_u1():
    """Parseval over all q: sum_q |S^z_q phi|^2 = N/4, sum_q |S^+_q phi|^2 =
    N_down, sum_q |S^-_q phi|^2 = N - N_down (unit phi)."""
    N, nd = 10, 3
    rng = np.random.default_rng(1)
    phi = rng.normal(size=comb(N, nd)) + 1j * rng.normal(size=comb(N, nd))
    phi /= np.linalg.norm(phi)
    tot = {orc.OP_SZ: 0.0, orc.OP_SPLUS: 0.0, orc.OP_SMINUS: 0.0}
    for q in range(N):
        for op in tot:
            v = orc.sq_apply_u1(N, nd, op, phi, (q, 0, 0), (N, 1, 1))
            tot[op] += np.vdot(v, v).real
    assert abs(tot[orc.OP_SZ] - N / 4) < 1e-12
    assert abs(tot[orc.OP_SPLUS] - nd) < 1e-12
    assert abs(tot[orc.OP_SMINUS] - (N - nd)) < 1e-12


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (6, 3), (5, 5)])
def test_triangular_one_magnon_dispersion(Lx, Ly):
    """One down spin on the periodic triangular lattice (three bond directions
    a1, a2, a1 - a2, six neighbours): E(k) = sum_b Jz/4 - 6 Jz/2 +
    J sum_{delta in a1, a2, a1-a2} cos(k.delta)."""
    J, Jz = 1.0, 0.7
    spec = qi.triangular(Lx, Ly, J=J, Jz=Jz)
    lat = olat(spec)
    nb = len(spec.bi)
    assert nb == 3 * Lx * Ly
    for K in qi.all_k((Lx, Ly, 1)):
        k1, k2 = 2 * np.pi * K[0] / Lx, 2 * np.pi * K[1] / Ly
        want = nb * Jz / 4 - 6 * Jz / 2 + J * (np.cos(k1) + np.cos(k2) + np.cos(k1 - k2))
        sec = orc.mk_list(lat, 1, K)
        assert sec.dim == 1
        assert abs(orc.dense_k(sec)[0, 0].real - want) < 1e-12


def test_thermal_average_over_sectors_equals_full_trace():
    """Eq. (ens): the levels of every (N_down, k) sector together give the
    partition function and energy of the whole 2^N space (Kronecker-built
    Hamiltonian, independent of the sector machinery)."""
    spec = qi.chain(8, J=1.0, Jz=0.6)
    lat = olat(spec)
    levels = []
    for nd in range(9):
        for K in qi.all_k((8, 1, 1)):
            sec = orc.mk_list(lat, nd, K)
            if sec.dim:
                levels.append(np.linalg.eigvalsh(orc.dense_k(sec)))
    E = np.concatenate(levels)
    assert len(E) == 256
    Hf = pins.kron_hamiltonian(spec)
    Ef = np.linalg.eigvalsh(Hf)
    np.testing.assert_allclose(np.sort(E), Ef, atol=1e-11)
    beta = np.array([0.1, 1.0, 5.0, 40.0])
    logZ, eavg = orc.thermal(E, None, beta)
    for i, b in enumerate(beta):
        w = np.exp(-b * Ef)
        assert abs(logZ[i] - np.log(w.sum())) < 1e-12 * max(1.0, abs(logZ[i]))
        assert abs(eavg[i] - (w * Ef).sum() / w.sum()) < 1e-11
