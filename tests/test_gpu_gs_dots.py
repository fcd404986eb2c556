"""The Gram-Schmidt dot products of the fp64 solves (qs3_gs_dots) against
exact rational dot products.

The default dots round every operand once onto a fixed-point grid set by the
largest exponent of its warp's 128 rows (error at most 2^-53 of that largest
magnitude) and sum the products of those images exactly; the strict64 dots
are binary64 FMA chains.  Both are checked against the exact value of
sum_i conj(v_i) w_i, computed here in integer arithmetic on the binary64
inputs, within the bound that the rounding onto the grid gives:
|error| <= 2^-52 (max|v| sum|w_i| + max|w| sum|v_i|) + 2^-49 sum|v_i||w_i|
per sector.  Inputs span many binades, contain zeros, subnormals and exact
cancellations, and the sectors cover several 2048-row chunks with ragged
tails."""
from __future__ import annotations

import ctypes
from fractions import Fraction

import numpy as np
import pytest

import qs3_inputs as qi
from tests.gpu_common import lib_basis, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SCALE = 1074          # every binary64 is an integer multiple of 2^-1074


def _ints(x: np.ndarray) -> list:
    out = []
    for v in x.tolist():
        n, d = float(v).as_integer_ratio()
        out.append(n * ((1 << SCALE) // d))
    return out


def _exact_dot(a: np.ndarray, w: np.ndarray) -> complex:
    """sum conj(a_i) w_i exactly, rounded once to binary64 per component."""
    if np.iscomplexobj(a):
        ar, ai, wr, wi = _ints(a.real), _ints(a.imag), _ints(w.real), _ints(w.imag)
        re = sum(x * y for x, y in zip(ar, wr)) + sum(x * y for x, y in zip(ai, wi))
        im = sum(x * y for x, y in zip(ar, wi)) - sum(x * y for x, y in zip(ai, wr))
        return complex(float(Fraction(re, 1 << (2 * SCALE))), float(Fraction(im, 1 << (2 * SCALE))))
    ar, wr = _ints(a), _ints(w)
    return float(Fraction(sum(x * y for x, y in zip(ar, wr)), 1 << (2 * SCALE)))


def _bound(a: np.ndarray, w: np.ndarray) -> float:
    aa, ww = np.abs(a), np.abs(w)
    if aa.size == 0:
        return 0.0
    return 2.0 ** -52 * (aa.max() * ww.sum() + ww.max() * aa.sum()) + 2.0 ** -49 * float(aa @ ww) + 1e-300


def _vectors(n: int, cx: bool, seed: int) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)

    def one(kind: str) -> np.ndarray:
        def real():
            if kind == "gauss":
                return rng.standard_normal(n)
            if kind == "binades":       # magnitudes over 60 binades, random signs
                return rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-60, 0, n)
            if kind == "sparse":        # mostly zero, a few values incl. subnormals
                x = np.zeros(n)
                idx = rng.choice(n, min(n, 40), replace=False)
                x[idx] = rng.standard_normal(idx.size) * 2.0 ** rng.integers(-1074, 3, idx.size).astype(float)
                return x
            if kind == "zero":
                return np.zeros(n)
            if kind == "wide":          # one huge element per 4096 rows next to tiny ones
                x = rng.standard_normal(n) * 1e-12
                x[::4096] = 1e3
                return x
            raise ValueError(kind)
        x = real()
        if cx:
            x = x + 1j * real()
        return x

    kinds = ["gauss", "binades", "sparse", "zero", "wide"]
    V = np.stack([one(k) for k in kinds])
    w = one("gauss")
    # row 5: w / |w| (its dot with w is |w|)
    V = np.concatenate([V, (w / np.linalg.norm(w))[None, :]], axis=0)
    V[0] /= np.linalg.norm(V[0])
    return V, w


@pytest.mark.parametrize("name,spec,nd,Ks", [
    ("square8_k", qi.square(8), 4, [(0, 0, 0), (1, 2, 0), (4, 4, 0)]),
    ("chain22_u1", qi.chain(22, Jz=0.5), 5, None),
])
def test_gs_dots_exact_and_strict(name, spec, nd, Ks):
    torch = torch_cuda()
    b = lib_basis(spec, nd, Ks)
    cx = Ks is not None
    assert max(b.dims) > 2 * 2048                 # several chunks and a ragged tail
    V, w = _vectors(b.total_dim, cx, seed=7)
    dt = torch.complex128 if cx else torch.float64
    Vd, wd = to_dev(V, dt), to_dev(w, dt)
    got = {mode: b.gs_dots(Vd, wd, exact=mode) for mode in (True, False)}
    for s in range(b.n_sectors):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        for j in range(V.shape[0]):
            a, ws = V[j, lo:hi], w[lo:hi]
            ex = _exact_dot(a, ws)
            bd = _bound(a, ws)
            for mode in (True, False):
                g = got[mode][s, j]
                assert abs(g.real - np.real(ex)) <= bd, (name, s, j, mode, g, ex, bd)
                assert abs(np.imag(g) - np.imag(ex)) <= bd, (name, s, j, mode, g, ex, bd)
            if j == 3:                              # the zero vector
                assert got[True][s, j] == 0
    # w against itself: |w|^2 per sector to a few ulps
    self_dot = b.gs_dots(wd[None, :].contiguous(), wd, exact=True)
    for s in range(b.n_sectors):
        ws = w[b.offsets[s]:b.offsets[s + 1]]
        ref = float(np.vdot(ws, ws).real)
        assert abs(self_dot[s, 0].real - ref) <= 8 * 2.0 ** -53 * ref


def test_gs_dots_empty_and_invalid():
    torch = torch_cuda()
    import paper_2107_00872_gb300 as qs3
    b = lib_basis(qi.square(6), 3, [(0, 0, 0), (1, 0, 0)])
    wd = torch.zeros(b.total_dim, dtype=torch.complex128, device="cuda")
    out = b.gs_dots(torch.zeros((0, b.total_dim), dtype=torch.complex128, device="cuda"), wd)
    assert out.shape == (2, 0)
    with pytest.raises(TypeError):
        b.gs_dots(torch.zeros((1, b.total_dim), dtype=torch.complex64, device="cuda"), wd.to(torch.complex64))
    lib = qs3.load()
    # NULL vectors, negative m, ldv below the dimension, real-only dtype
    assert lib.qs3_gs_dots(b.handle, qs3.QS3_C128, 1, None, b.total_dim, None, None, 0, None) == -1
    assert lib.qs3_gs_dots(b.handle, qs3.QS3_C128, -1, None, b.total_dim, None, None, 0, None) == -1
    buf = np.zeros(8)
    p = ctypes.c_void_p(wd.data_ptr())
    assert lib.qs3_gs_dots(b.handle, qs3.QS3_C128, 2, p, b.total_dim - 1, p, buf.ctypes.data_as(ctypes.c_void_p),
                           0, None) == -1
    assert lib.qs3_gs_dots(b.handle, qs3.QS3_C64, 1, p, b.total_dim, p, buf.ctypes.data_as(ctypes.c_void_p),
                           0, None) == -1
    assert lib.qs3_gs_dots(b.handle, qs3.QS3_C128, 1, p, b.total_dim, p, buf.ctypes.data_as(ctypes.c_void_p),
                           2, None) == -1


def test_gs_dots_many_slices():
    """A sector of 1,184,040 rows (578 chunks, 9,248 warp partials): the
    partials are reduced in slices of 4,096, then the slices; the result is
    still the exact dot within the grid bound."""
    torch = torch_cuda()
    b = lib_basis(qi.chain(28, Jz=0.5), 7)
    assert b.total_dim == 1184040
    rng = np.random.default_rng(3)
    w = rng.standard_normal(b.total_dim)
    V = np.stack([rng.standard_normal(b.total_dim) * 2.0 ** rng.uniform(-30, 0, b.total_dim), w / np.linalg.norm(w)])
    got = b.gs_dots(to_dev(V, torch.float64), to_dev(w, torch.float64), exact=True)
    for j in range(2):
        ex = _exact_dot(V[j], w)
        assert abs(got[0, j] - ex) <= _bound(V[j], w), (j, got[0, j], ex)


@pytest.mark.parametrize("name,spec,nd,Ks", [
    ("square8_k", qi.square(8), 4, [(0, 0, 0), (1, 2, 0), (4, 4, 0)]),
    ("square6_k_odd", qi.square(6), 3, [(0, 0, 0), (1, 0, 0), (2, 1, 0)]),
    ("chain21_u1_odd", qi.chain(21, Jz=0.5), 5, None),
])
def test_gs_dots_copy_ring_identical(name, spec, nd, Ks):
    """The dot pass with the stored vectors' digits brought in by bulk copies
    into a ring in shared memory (k_dotb: dot_vectors64 = 8) sums the
    same integer products as the register-staged pass (k_dotx): the results
    agree bit for bit, and stay within the grid bound of the exact dots.
    Odd dimensions put the digit planes and sector starts off the 16-byte
    boundary, so the copies start below the chunk."""
    torch = torch_cuda()
    b = lib_basis(spec, nd, Ks)
    cx = Ks is not None
    esz = 8 if cx else 4                      # bytes of one element of a digit plane
    if name.endswith("_odd"):
        assert (b.total_dim * esz) % 16 != 0
        assert Ks is None or any((o * esz) % 16 for o in b.offsets)
    V, w = _vectors(b.total_dim, cx, seed=11)
    dt = torch.complex128 if cx else torch.float64
    Vd, wd = to_dev(V, dt), to_dev(w, dt)
    got = {}
    for nv in (2, 8):
        b.tuning(dot_vectors64=nv)
        got[nv] = b.gs_dots(Vd, wd, exact=True)
        assert b.tuning()["dot_vectors64"] == nv
    np.testing.assert_array_equal(got[8], got[2])
    for s in range(b.n_sectors):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        for j in range(V.shape[0]):
            ex = _exact_dot(V[j, lo:hi], w[lo:hi])
            bd = _bound(V[j, lo:hi], w[lo:hi])
            assert abs(np.real(got[8][s, j]) - np.real(ex)) <= bd, (name, s, j)
            assert abs(np.imag(got[8][s, j]) - np.imag(ex)) <= bd, (name, s, j)
