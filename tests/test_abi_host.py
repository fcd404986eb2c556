"""The C ABI without a GPU: the library loads, exports every function that
include/qs3.h declares (and the binding knows each signature), and the host
side of qs3_basis_create rejects bad input with the documented status before
any device work -- invalid bonds (INVALID_ARG), sizes beyond the kernels'
limits (OVERFLOW), symmetry violations (SYMMETRY) -- and turns an injected
allocation failure into QS3_ERR_OOM.  The host-only thermal average of Eq.
(ens) is checked against its definition."""
from __future__ import annotations

import math
import os
import re

import numpy as np
import pytest

import qs3_inputs as qi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs3():
    import paper_2107_00872_gb300 as q
    from paper_2107_00872_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    q.load()
    return q


def declared_functions() -> list:
    text = open(os.path.join(ROOT, "include", "qs3.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qs3_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function(qs3):
    from paper_2107_00872_gb300 import _abi
    lib = qs3.load()
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), f"{n} is declared but not exported"
        assert n in _abi.SIGNATURES, f"{n} has no binding signature"
    assert set(_abi.SIGNATURES) <= set(names)


def test_status_texts(qs3):
    lib = qs3.load()
    assert lib.qs3_strerror(0) == b"ok"
    for code in range(-8, 0):
        assert lib.qs3_strerror(code) and lib.qs3_strerror(code) != b"ok"
    assert b"sm_103a" in lib.qs3_version()


def _status(qs3, fn):
    with pytest.raises(qs3.QS3Error) as e:
        fn()
    return e.value.status


def _spec(N, bonds, jxy=None, jz=None, h=None, L=(0, 0, 0)):
    bi = np.array([b[0] for b in bonds], np.int32)
    bj = np.array([b[1] for b in bonds], np.int32)
    jxy = np.ones(len(bonds)) if jxy is None else np.asarray(jxy, float)
    jz = np.ones(len(bonds)) if jz is None else np.asarray(jz, float)
    return qi.LatticeSpec(N, bi, bj, jxy, jz, h, L, "t")


INVALID, OVERFLOW, SYMMETRY, OOM = -1, -2, -3, -4


def test_invalid_bonds(qs3):
    ring = [(i, (i + 1) % 6) for i in range(6)]
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring[:5] + [(3, 3)]), 2)) == INVALID      # i == j
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring[:5] + [(3, 6)]), 2)) == INVALID      # out of range
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring[:5] + [(-1, 2)]), 2)) == INVALID     # negative
    bad = np.ones(6)
    bad[2] = np.nan
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring, jxy=bad), 2)) == INVALID           # non-finite J
    bad = np.ones(6)
    bad[4] = np.inf
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring, jz=bad), 2)) == INVALID            # non-finite Jz
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring, L=(4, 1, 1)), 2)) == INVALID       # Lx Ly Lz != N
    assert _status(qs3, lambda: qs3.Basis(_spec(6, ring), 7)) == INVALID                    # N_down > N


def test_overflow_limits(qs3):
    # N_down above QS3_MAX_NDOWN = 8
    assert _status(qs3, lambda: qs3.Basis(qi.chain(20), 9)) == OVERFLOW
    # more than QS3_MAX_SITES = 4096 sites
    assert _status(qs3, lambda: qs3.Basis(_spec(4097, [(0, 1)]), 1)) == OVERFLOW
    # C(N, N_down) >= 2^63: C(4096, 8) ~ 2e24; C(1000, 8) ~ 2.4e19 > 2^63 ~ 9.2e18
    assert math.comb(1000, 8) >= 2 ** 63 > math.comb(1000, 7)
    ring = lambda n: _spec(n, [(i, (i + 1) % n) for i in range(n)])  # noqa: E731  (no translation group)
    assert _status(qs3, lambda: qs3.Basis(ring(4096), 8)) == OVERFLOW
    assert _status(qs3, lambda: qs3.Basis(ring(1000), 8)) == OVERFLOW


def test_symmetry_violations(qs3):
    sq = qi.square(4)
    # a bond that breaks the translations, with momenta
    broken = qi.LatticeSpec(sq.n_sites, sq.bi, sq.bj, sq.jxy.copy(), sq.jz, None, sq.L, "b")
    broken.jxy[3] = 0.5
    assert _status(qs3, lambda: qs3.Basis(broken, 2, [(0, 0, 0)])) == SYMMETRY
    # a non-uniform site field with momenta
    h = np.zeros(sq.n_sites)
    h[5] = 0.1
    fld = qi.LatticeSpec(sq.n_sites, sq.bi, sq.bj, sq.jxy, sq.jz, h, sq.L, "h")
    assert _status(qs3, lambda: qs3.Basis(fld, 2, [(1, 0, 0)])) == SYMMETRY
    # K out of range, and momenta without a translation group
    assert _status(qs3, lambda: qs3.Basis(sq, 2, [(4, 0, 0)])) == SYMMETRY
    assert _status(qs3, lambda: qs3.Basis(sq, 2, [(0, -1, 0)])) == SYMMETRY
    noL = qi.LatticeSpec(sq.n_sites, sq.bi, sq.bj, sq.jxy, sq.jz, None, (0, 0, 0), "n")
    assert _status(qs3, lambda: qs3.Basis(noL, 2, [(0, 0, 0)])) == SYMMETRY


def test_unit_cell_validation(qs3):
    """Several spins per unit cell: n_sub Lx Ly Lz must equal N, n_sub needs a
    translation group, and a field must repeat from cell to cell."""
    kg = qi.kagome(2, 2)
    bad = qi.LatticeSpec(kg.n_sites, kg.bi, kg.bj, kg.jxy, kg.jz, None, (2, 2, 1), "k", None, 2)
    assert _status(qs3, lambda: qs3.Basis(bad, 2, [(0, 0, 0)])) == INVALID
    noL = qi.LatticeSpec(kg.n_sites, kg.bi, kg.bj, kg.jxy, kg.jz, None, (0, 0, 0), "k", None, 3)
    assert _status(qs3, lambda: qs3.Basis(noL, 2)) == INVALID
    h = np.tile([0.1, 0.2, 0.3], 4)
    h[7] = 0.5
    fld = qi.LatticeSpec(kg.n_sites, kg.bi, kg.bj, kg.jxy, kg.jz, h, (2, 2, 1), "k", None, 3)
    assert _status(qs3, lambda: qs3.Basis(fld, 2, [(0, 0, 0)])) == SYMMETRY


def test_injected_allocation_failure_is_oom(qs3):
    prev = qs3.inject_alloc_failure(0)
    try:
        assert _status(qs3, lambda: qs3.Basis(qi.chain(12), 3)) == OOM
        assert b"injected" in qs3.load().qs3_last_error()
    finally:
        assert qs3.inject_alloc_failure(prev) == 0


def test_wait_timeout_injection_counter(qs3):
    """The host side of the wait-timeout injection: a count of ring launches
    to starve, set, read back and cleared (n <= 0 switches it off)."""
    assert qs3.inject_wait_timeout(3) == 0
    assert qs3.inject_wait_timeout(-5) == 3
    assert qs3.inject_wait_timeout(0) == 0


def test_null_handles(qs3):
    lib = qs3.load()
    assert lib.qs3_basis_create(None, 2, 1, None, None) == INVALID
    assert lib.qs3_hphi(None, 3, None, None, None) == INVALID
    assert lib.qs3_lanczos(None, None, None, None, None, None) == INVALID
    assert lib.qs3_basis_tuning(None, 0, None, None, None) == INVALID
    assert lib.qs3_probe_peaks(None, None) == INVALID
    assert lib.qs3_gs_dots(None, 3, 1, None, 0, None, None, 0, None) == INVALID


def test_thermal_average_definition(qs3):
    """qs3_thermal (Eq. (ens)) against the weighted Boltzmann sums written out."""
    import ctypes
    lib = qs3.load()
    rng = np.random.default_rng(3)
    E = rng.uniform(-30.0, 5.0, 40)
    A = rng.normal(size=40)
    m = rng.integers(1, 4, 40).astype(float)
    beta = np.array([0.0, 0.3, 2.0, 50.0])
    lz = np.zeros(4)
    av = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.qs3_thermal(40, p(E), p(A), p(m), 4, p(beta), p(lz), p(av)) == 0
    for k, b in enumerate(beta):
        w = m * np.exp(-b * (E - E.min()))
        assert abs(lz[k] - (math.log(w.sum()) - b * E.min())) <= 1e-12 * max(1.0, abs(lz[k]))
        assert abs(av[k] - (w * A).sum() / w.sum()) <= 1e-12
    bad = E.copy()
    bad[0] = np.nan
    assert lib.qs3_thermal(40, p(bad), None, None, 4, p(beta), p(lz), p(av)) == INVALID
    assert lib.qs3_thermal(0, p(E), None, None, 4, p(beta), p(lz), p(av)) == INVALID
