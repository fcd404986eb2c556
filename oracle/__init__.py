"""CPU oracle of the QS^3 hot path (Ueda, Yunoki, Shimokawa, arXiv 2107.00872).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import it.  The
GPU library never imports, links or calls anything here, and nothing here
imports the GPU package.

The integer/graph parts (Alg. 1-9, 11 of the paper and the two-point
functions) are a literal C restatement in ``qs3_oracle.c`` (fp64, 1-based
as in the paper); the Lanczos, thick-restart Lanczos (Alg. 10) and the
continued fraction (Eq. cfe) are plain numpy below, with numpy's dense
symmetric eigensolver as the library step for the small projected matrices.

Every public function converts to the GPU library's 0-based conventions only
at its boundary: ``rank0 = a - 1``, sites ``c = n - 1``, ``|Stab| = N_{a,k}/N``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs3_oracle.c")
_LIB = os.path.join(_HERE, "libqs3_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc, OpenMP over rows as in the paper)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            U = ctypes.c_uint64
            L = ctypes.c_int64
            lat = [I, I, I, P, P, P, P, P, P]
            sig = {
                "orc_set_threads": ([I], I),
                "orc_binom": ([I, I], U),
                "orc_F": ([I, I, P], U),
                "orc_f_bar": ([I, I, U, P, P], I),
                "orc_unrank_all": ([I, I, P], I),
                "orc_spin_exchange": ([I, I, P, I, I], U),
                "orc_dense_u1": (lat + [P], I),
                "orc_hphi_u1": (lat + [P, P], I),
                "orc_hphi_u1_rows": (lat + [P, L, P, P, P], I),
                "orc_mk_list": (lat + [P, P, P], L),
                "orc_representative": (lat + [U, P], U),
                "orc_orbit": (lat + [U, P], I),
                "orc_hphi_k": (lat + [P, P, P, L, P, P], I),
                "orc_hphi_k_rows": (lat + [P, P, P, L, P, L, P, P, P], I),
                "orc_dense_k": (lat + [P, P, P, L, P], I),
                "orc_smq": (lat + [P, P, P, L, P, P, P, P, P, L, P], I),
                "orc_corr_u1": ([I, I, P, P, P, P], I),
                "orc_row_terms_k": (lat + [P, U, L, P, P, P], L),
                "orc_check_state": (lat + [P, U], ctypes.c_double),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of the C oracle; returns the count in use."""
    return _load().orc_set_threads(int(n))


# --------------------------------------------------------------------- model


@dataclass
class Lattice:
    """Bonds of Eq. (1) with 0-based sites (converted to 1-based inside).

    ``L`` is the translation group (Lx, Ly, Lz) of the unit cells; ``(N,1,1)``
    for a chain.  ``n_sub`` spins per cell: site r (0-based) is spin
    r % n_sub of cell r // n_sub, cells numbered x + Lx (y + Ly z).  The group
    is only used by the k-sector functions and needs n_sub*Lx*Ly*Lz == N.
    """
    n_sites: int
    bi: np.ndarray
    bj: np.ndarray
    jxy: np.ndarray
    jz: np.ndarray
    h: np.ndarray | None = None
    L: tuple = (0, 0, 0)
    n_sub: int = 1

    def _args(self, nd: int):
        lo = np.minimum(self.bi, self.bj).astype(np.int32) + 1
        hi = np.maximum(self.bi, self.bj).astype(np.int32) + 1
        self._keep = [np.ascontiguousarray(lo), np.ascontiguousarray(hi),
                      np.ascontiguousarray(self.jxy, dtype=np.float64),
                      np.ascontiguousarray(self.jz, dtype=np.float64),
                      None if self.h is None else np.ascontiguousarray(self.h, dtype=np.float64),
                      np.ascontiguousarray(np.array(tuple(self.L if tuple(self.L) != (0, 0, 0)
                                                          else (self.n_sites, 1, 1)) + (int(self.n_sub),),
                                                    dtype=np.int32))]
        k = self._keep
        return (int(self.n_sites), int(nd), int(len(lo)), _p(k[0]), _p(k[1]), _p(k[2]), _p(k[3]),
                _p(k[4]), _p(k[5]))


def binom(N: int, nd: int) -> int:
    return int(_load().orc_binom(N, nd))


def F(N: int, n1: list[int]) -> int:
    """Eq. (a_of_n): 1-based index of the 1-based sorted site list n1."""
    a = np.ascontiguousarray(n1, dtype=np.int32)
    return int(_load().orc_F(N, len(n1), _p(a)))


def f_bar(N: int, nd: int, a: int):
    """Alg. 1: (1-based site list, trace of s after each column step)."""
    n = np.zeros(max(nd, 1), np.int32)
    tr = np.zeros(max(nd, 1), np.uint64)
    if _load().orc_f_bar(N, nd, a, _p(n), _p(tr)) != 0:
        raise ValueError("index out of range")
    return [int(v) for v in n[:nd]], [int(v) for v in tr[: max(nd - 1, 0)]]


def unrank_all(N: int, nd: int) -> np.ndarray:
    """0-based down-spin lists of every U(1) state, in index order (D x nd)."""
    D = binom(N, nd)
    out = np.zeros((D, max(nd, 1)), np.int32)
    _load().orc_unrank_all(N, nd, _p(out))
    return out[:, :nd] - 1


def spin_exchange_index(N: int, n1: list[int], r: int, rp: int) -> int:
    a = np.ascontiguousarray(n1, dtype=np.int32)
    return int(_load().orc_spin_exchange(N, len(n1), _p(a), r, rp))


def dense_u1(lat: Lattice, nd: int) -> np.ndarray:
    """Alg. 4: dense U(1) block, rows/cols in 0-based rank order."""
    D = binom(lat.n_sites, nd)
    H = np.zeros((D, D), np.float64)
    if _load().orc_dense_u1(*lat._args(nd), _p(H)) != 0:
        raise ValueError("bad lattice")
    return H


def hphi_u1(lat: Lattice, nd: int, phi: np.ndarray) -> np.ndarray:
    """U(1) H phi (fp64, complex result)."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    y = np.zeros_like(x)
    _load().orc_hphi_u1(*lat._args(nd), _p(x), _p(y))
    return y


def hphi_u1_rows(lat: Lattice, nd: int, phi: np.ndarray, rows: np.ndarray, count: bool = False):
    """U(1) H phi on the given 0-based rows; with count=True also the number
    of matrix terms applied."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros(len(r), np.complex128)
    n = np.zeros(1, np.int64)
    _load().orc_hphi_u1_rows(*lat._args(nd), _p(x), len(r), _p(r), _p(y), _p(n))
    return (y, int(n[0])) if count else y


@dataclass
class Sector:
    """Output of Alg. 6 for one (N_down, K): sigma (1-based), N_{a,k}."""
    lat: Lattice
    nd: int
    K: tuple
    sigma1: np.ndarray
    Nak: np.ndarray

    @property
    def dim(self) -> int:
        return len(self.sigma1)

    @property
    def rank0(self) -> np.ndarray:
        return self.sigma1.astype(np.uint64) - np.uint64(1)

    @property
    def stab(self) -> np.ndarray:
        """|Stab| = N_{a,k} / (number of cell translations)"""
        L = tuple(self.lat.L) if tuple(self.lat.L) != (0, 0, 0) else (self.lat.n_sites, 1, 1)
        return np.rint(self.Nak / (L[0] * L[1] * L[2])).astype(np.int64)


def mk_list(lat: Lattice, nd: int, K) -> Sector:
    """Alg. 5 + 6 with every translation of the group."""
    Kc = np.ascontiguousarray(K, dtype=np.int32)
    lib = _load()
    d = lib.orc_mk_list(*lat._args(nd), _p(Kc), None, None)
    if d < 0:
        raise ValueError("bad lattice")
    sig = np.zeros(max(d, 1), np.uint64)
    nak = np.zeros(max(d, 1), np.float64)
    lib.orc_mk_list(*lat._args(nd), _p(Kc), _p(sig), _p(nak))
    return Sector(lat, nd, tuple(int(v) for v in K), sig[:d], nak[:d])


def representative(lat: Lattice, nd: int, a1: int):
    """Alg. 7: (1-based rep index, translation l with T^l a = rep)."""
    l = np.zeros(3, np.int32)
    rep = _load().orc_representative(*lat._args(nd), a1, _p(l))
    return int(rep), tuple(int(v) for v in l)


def orbit(lat: Lattice, nd: int, a1: int) -> np.ndarray:
    """1-based indices of T^t |a>, t over the Lx Ly Lz cell translations in
    the order tx fastest."""
    L = tuple(lat.L) if tuple(lat.L) != (0, 0, 0) else (lat.n_sites, 1, 1)
    out = np.zeros(L[0] * L[1] * L[2], np.uint64)
    _load().orc_orbit(*lat._args(nd), a1, _p(out))
    return out


def hphi_k(sec: Sector, phi: np.ndarray) -> np.ndarray:
    """Alg. 9 over every row of the sector."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    y = np.zeros_like(x)
    Kc = np.ascontiguousarray(sec.K, dtype=np.int32)
    _load().orc_hphi_k(*sec.lat._args(sec.nd), _p(Kc), _p(sec.sigma1), _p(sec.Nak), sec.dim, _p(x), _p(y))
    return y


def hphi_k_rows(sec: Sector, phi: np.ndarray, rows: np.ndarray, count: bool = False):
    """Alg. 9 on the given 0-based rows; with count=True also the number of
    matrix terms applied."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros(len(r), np.complex128)
    n = np.zeros(1, np.int64)
    Kc = np.ascontiguousarray(sec.K, dtype=np.int32)
    _load().orc_hphi_k_rows(*sec.lat._args(sec.nd), _p(Kc), _p(sec.sigma1), _p(sec.Nak), sec.dim, _p(x),
                            len(r), _p(r), _p(y), _p(n))
    return (y, int(n[0])) if count else y


def row_terms_k(lat: Lattice, nd: int, K, a1: int, max_terms: int = 4096):
    """One row of Alg. 9 for the representative a1 (1-based) without a
    representative list: (diagonal, 1-based target representatives,
    coefficients), or None when a1 is not a compatible representative."""
    Kc = np.ascontiguousarray(K, dtype=np.int32)
    t = np.zeros(max_terms, np.uint64)
    c = np.zeros(max_terms, np.complex128)
    dg = np.zeros(1, np.float64)
    n = _load().orc_row_terms_k(*lat._args(nd), _p(Kc), int(a1), max_terms, _p(t), _p(c), _p(dg))
    if n < 0:
        return None
    return float(dg[0]), t[:n], c[:n]


def check_state(lat: Lattice, nd: int, K, a1: int) -> float:
    """Alg. 5: N_{a,k} of the 1-based index a1 (0 if not a compatible representative)."""
    Kc = np.ascontiguousarray(K, dtype=np.int32)
    return float(_load().orc_check_state(*lat._args(nd), _p(Kc), int(a1)))


def dense_k(sec: Sector) -> np.ndarray:
    """Alg. 8: dense symmetry-adapted block."""
    d = sec.dim
    H = np.zeros((d, d), np.complex128)
    Kc = np.ascontiguousarray(sec.K, dtype=np.int32)
    _load().orc_dense_k(*sec.lat._args(sec.nd), _p(Kc), _p(sec.sigma1), _p(sec.Nak), d, _p(H))
    return H


def smq(src: Sector, phi: np.ndarray, Q, dst: Sector, pos: np.ndarray | None = None) -> np.ndarray:
    """Alg. 11 (push form): S^-_q phi from (nd, K) into (nd+1, K+Q)."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    y = np.zeros(dst.dim, np.complex128)
    Kc = np.ascontiguousarray(src.K, dtype=np.int32)
    Qc = np.ascontiguousarray(Q, dtype=np.int32)
    pc = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64)
    _load().orc_smq(*src.lat._args(src.nd), _p(Kc), _p(src.sigma1), _p(src.Nak), src.dim, _p(x), _p(Qc),
                    _p(pc), _p(dst.sigma1), _p(dst.Nak), dst.dim, _p(y))
    return y


def corr_u1(N: int, nd: int, phi: np.ndarray):
    """<s^z_i s^z_j>, <s^+_i s^-_j>, <s^z_i> of a U(1) vector (0-based sites)."""
    x = np.ascontiguousarray(phi, dtype=np.complex128)
    szsz = np.zeros((N, N), np.float64)
    spsm = np.zeros((N, N), np.complex128)
    sz = np.zeros(N, np.float64)
    _load().orc_corr_u1(N, nd, _p(x), _p(szsz), _p(spsm), _p(sz))
    return szsz, spsm, sz


# ------------------------------------------------- symmetry-adapted <-> U(1)


def unfold(sec: Sector, phi_k: np.ndarray) -> np.ndarray:
    """Eq. (akstate) written out: sum_a phi_a N_a^{-1/2} sum_t e^{-ik.t} T^t|a>."""
    lat = sec.lat
    L = np.array(lat.L, dtype=np.int64)
    N = lat.n_sites
    t = np.stack(np.meshgrid(np.arange(L[0]), np.arange(L[1]), np.arange(L[2]), indexing="ij"), -1)
    t = t.transpose(2, 1, 0, 3).reshape(-1, 3)          # tx fastest, like orc_orbit
    kt = 2 * np.pi * (t * (np.array(sec.K) / L)).sum(1)
    out = np.zeros(binom(N, sec.nd), np.complex128)
    for i, a in enumerate(sec.sigma1):
        orb = orbit(lat, sec.nd, int(a)).astype(np.int64) - 1
        np.add.at(out, orb, phi_k[i] * np.exp(-1j * kt) / np.sqrt(sec.Nak[i]))
    return out


def fold(sec: Sector, phi_u: np.ndarray) -> np.ndarray:
    """Projection <a,k|phi> of a U(1) vector onto the sector basis."""
    lat = sec.lat
    L = np.array(lat.L, dtype=np.int64)
    t = np.stack(np.meshgrid(np.arange(L[0]), np.arange(L[1]), np.arange(L[2]), indexing="ij"), -1)
    t = t.transpose(2, 1, 0, 3).reshape(-1, 3)
    kt = 2 * np.pi * (t * (np.array(sec.K) / L)).sum(1)
    out = np.zeros(sec.dim, np.complex128)
    for i, a in enumerate(sec.sigma1):
        orb = orbit(lat, sec.nd, int(a)).astype(np.int64) - 1
        out[i] = (np.exp(1j * kt) * phi_u[orb]).sum() / np.sqrt(sec.Nak[i])
    return out


# ------------------------------------------- S^alpha_q from its definition
# "In the same manner" as Alg. 11 the paper also applies S^+_q and S^z_q
# (input_dynamic: spsmsz = 1 for S^+, 2 for S^-, 3 for S^z).  Written here
# from S^alpha_q = N^{-1/2} sum_j e^{-i q.R_j} S^alpha_j and each S^alpha_j's
# action on one U(1) state, then carried to a momentum sector by unfold/fold.

OP_SPLUS, OP_SMINUS, OP_SZ = 1, 2, 3


def site_phases_q(N: int, L, Q, pos: np.ndarray | None = None) -> np.ndarray:
    """e^{-i q.R_j} for every site j with q.a_alpha = 2 pi Q_alpha / L_alpha;
    R_j = (x, y, z) of the site index j = x + Lx (y + Ly z), or pos[j]."""
    L = np.array(L if tuple(L) != (0, 0, 0) else (N, 1, 1), dtype=np.int64)
    if pos is None:
        j = np.arange(N)
        R = np.stack([j % L[0], (j // L[0]) % L[1], j // (L[0] * L[1])], -1).astype(np.float64)
    else:
        R = np.asarray(pos, np.float64).reshape(N, 3)
    return np.exp(-2j * np.pi * (R * (np.asarray(Q, np.float64) / L)).sum(1))


def sq_apply_u1(N: int, nd: int, op: int, phi_u: np.ndarray, Q, L, pos: np.ndarray | None = None) -> np.ndarray:
    """S^alpha_q phi on a U(1) vector of nd down spins (0-based rank order):
    S^+_j removes the down spin at j (zero if j is up), S^-_j puts one at an
    up site j, S^z_j multiplies by 1/2 - n_j.  The result has nd - 1 (S^+),
    nd + 1 (S^-) or nd (S^z) down spins."""
    states = unrank_all(N, nd)
    ph = site_phases_q(N, L, Q, pos)
    nd2 = nd - 1 if op == OP_SPLUS else (nd + 1 if op == OP_SMINUS else nd)
    if nd2 < 0 or nd2 > N:
        raise ValueError("operator leaves the state space")
    out = np.zeros(binom(N, nd2), np.complex128)

    def idx(sites):
        return F(N, [v + 1 for v in sites]) - 1 if sites else 0

    for a in range(len(phi_u)):
        x = phi_u[a]
        if x == 0:
            continue
        down = set(int(v) for v in states[a]) if nd > 0 else set()
        if op == OP_SZ:
            out[a] += x * sum(ph[j] * (0.5 - (1.0 if j in down else 0.0)) for j in range(N))
        elif op == OP_SPLUS:
            for j in down:
                out[idx(sorted(down - {j}))] += ph[j] * x
        else:
            for j in range(N):
                if j not in down:
                    out[idx(sorted(down | {j}))] += ph[j] * x
    return out / np.sqrt(N)


def sq_apply_k(src: Sector, phi_k: np.ndarray, op: int, Q, dst: Sector, pos: np.ndarray | None = None) -> np.ndarray:
    """S^alpha_q on a vector of sector (nd, K) into sector dst (nd2, K + Q):
    unfold to the U(1) basis, apply sq_apply_u1, project onto dst."""
    lat = src.lat
    u = unfold(src, np.asarray(phi_k, np.complex128))
    v = sq_apply_u1(lat.n_sites, src.nd, op, u, Q, lat.L, pos)
    return fold(dst, v)


# ------------------------------------------- thermal averages, Eq. (ens)


def thermal(E: np.ndarray, A: np.ndarray | None, beta: np.ndarray, mult: np.ndarray | None = None):
    """Eq. (ens) over a list of levels E_nu (all sectors): returns (log Z(beta),
    <A>(beta)) with Z = sum_nu m_nu e^{-beta E_nu} and <A> = sum_nu m_nu
    e^{-beta E_nu} A_nu / Z (A = E when None).  Written directly, with the
    exponents shifted by min E so large beta does not underflow."""
    E = np.asarray(E, np.float64)
    A = E if A is None else np.asarray(A, np.float64)
    m = np.ones_like(E) if mult is None else np.asarray(mult, np.float64)
    e0 = E.min()
    logZ, avg = [], []
    for b in np.atleast_1d(beta):
        w = m * np.exp(-b * (E - e0))
        z = w.sum()
        logZ.append(np.log(z) - b * e0)
        avg.append((w * A).sum() / z)
    return np.array(logZ), np.array(avg)


# ------------------------------------------------------ Lanczos, Alg. 10, CF


def _mgs(Psi: list[np.ndarray], v: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt against the stored vectors (Alg. 10 comment)."""
    for p in Psi:
        v = v - np.vdot(p, v) * p
    return v


def lanczos(apply_h, v0: np.ndarray, n_iter: int, reorth: bool = True):
    """Alg. 10 lines 2-11 (conventional Lanczos part): returns alpha, beta,
    the Lanczos vectors and beta_0 = |v0|.  beta[x] couples psi_{x+1} and
    psi_{x+2} (0-based x); iteration stops early on an invariant subspace."""
    beta0 = float(np.sqrt(np.vdot(v0, v0).real))
    psi = v0 / beta0
    Psi = [psi]
    alpha, beta = [], []
    prev = None
    for x in range(n_iter):
        v = apply_h(Psi[-1])
        a = np.vdot(Psi[-1], v).real
        w = v - a * Psi[-1]
        if prev is not None:
            w = w - beta[-1] * prev
        if reorth:
            w = _mgs(Psi, w)
        b = float(np.sqrt(np.vdot(w, w).real))
        alpha.append(a)
        beta.append(b)
        if b <= 1e-13 * max(1.0, abs(a)) or x == n_iter - 1:
            break
        prev = Psi[-1]
        Psi.append(w / b)
    return np.array(alpha), np.array(beta), Psi, beta0


def tridiag(alpha, beta):
    n = len(alpha)
    T = np.diag(alpha).astype(np.float64)
    for i in range(n - 1):
        T[i, i + 1] = T[i + 1, i] = beta[i]
    return T


def lanczos_ground(apply_h, v0: np.ndarray, max_iter: int = 400, tol: float = 1e-13):
    """Conventional Lanczos to the lowest eigenpair (paper defaults: checks
    every 5 iterations after at least 20); returns (E0, normalised vector)."""
    alpha, beta, Psi, _ = lanczos(apply_h, v0, max_iter)
    T = tridiag(alpha, beta)
    e, C = np.linalg.eigh(T)
    vec = sum(C[i, 0] * Psi[i] for i in range(len(alpha)))
    vec = vec / np.linalg.norm(vec)
    return float(e[0]), vec


def thick_restart_lanczos(apply_h, v0: np.ndarray, n_keep: int, n_max: int, max_restart: int,
                          eps: float):
    """Alg. 10 (thick-restart Lanczos), written in the paper's order.

    Returns the lowest n_keep Ritz values, the Ritz vectors and the number of
    restarts performed.  Reorthogonalisation is modified Gram-Schmidt against
    every stored vector."""
    d = len(v0)
    n_max = min(n_max, d)
    n_keep = min(n_keep, n_max - 1) if n_max > 1 else 1
    beta0 = np.sqrt(np.vdot(v0, v0).real)
    Psi = [v0 / beta0]
    alpha = np.zeros(n_max)
    beta = np.zeros(n_max)
    # first part: N_M Lanczos steps (lines 4-12)
    x = 0
    while x < n_max:
        v = apply_h(Psi[x])
        alpha[x] = np.vdot(Psi[x], v).real
        w = v - alpha[x] * Psi[x] - (beta[x - 1] * Psi[x - 1] if x > 0 else 0)
        w = _mgs(Psi, w)
        beta[x] = np.sqrt(np.vdot(w, w).real)
        Psi.append(w / beta[x] if beta[x] > 0 else w)
        x += 1
        if beta[x - 1] <= 1e-13 * max(1.0, abs(alpha[x - 1])):
            T = tridiag(alpha[:x], beta[:x])
            e, C = np.linalg.eigh(T)
            vecs = [sum(C[i, y] * Psi[i] for i in range(x)) for y in range(min(n_keep, x))]
            return e[:n_keep], vecs, 0
    T = tridiag(alpha, beta)
    e, C = np.linalg.eigh(T)
    e_prev = None
    for it in range(1, max_restart + 1):
        # line 14: Ritz vectors
        keep = [sum(C[i, y] * Psi[i] for i in range(n_max)) for y in range(n_keep)]
        if e_prev is not None and np.max(np.abs(e_prev / e[:n_keep] - 1.0)) < eps:
            return e[:n_keep], keep, it
        e_prev = e[:n_keep].copy()
        bK = beta[n_max - 1] * C[n_max - 1, :n_keep]      # beta_y = beta_{N_M} c_{N_M, y}
        resid = Psi[n_max]                                  # psi_{N_M+1}
        Psi = keep + [resid]
        alpha = np.zeros(n_max)
        beta = np.zeros(n_max)
        alpha[:n_keep] = e[:n_keep]
        # lines 21-25: one step from psi_{N_K+1} with the arrowhead couplings
        xk = n_keep
        v = apply_h(Psi[xk])
        alpha[xk] = np.vdot(Psi[xk], v).real
        v = v - sum(bK[y] * Psi[y] for y in range(n_keep))
        w = v - alpha[xk] * Psi[xk]
        w = _mgs(Psi, w)
        beta[xk] = np.sqrt(np.vdot(w, w).real)
        Psi.append(w / beta[xk])
        # line 26: remaining steps
        for x in range(xk + 1, n_max):
            v = apply_h(Psi[x])
            alpha[x] = np.vdot(Psi[x], v).real
            w = v - alpha[x] * Psi[x] - beta[x - 1] * Psi[x - 1]
            w = _mgs(Psi, w)
            beta[x] = np.sqrt(np.vdot(w, w).real)
            Psi.append(w / beta[x])
        # lines 27-30: arrowhead + tridiagonal T
        T = np.zeros((n_max, n_max))
        np.fill_diagonal(T, alpha)
        T[:n_keep, xk] = bK
        T[xk, :n_keep] = bK
        for z in range(xk, n_max - 1):
            T[z, z + 1] = T[z + 1, z] = beta[z]
        e, C = np.linalg.eigh(T)
    keep = [sum(C[i, y] * Psi[i] for i in range(n_max)) for y in range(n_keep)]
    return e[:n_keep], keep, max_restart


def continued_fraction(alpha, beta, norm2: float, omega: np.ndarray, e0: float, eta: float,
                       shift: float = 0.0) -> np.ndarray:
    """Eq. (cfe): S(omega) = -(1/pi) Im[ norm2 / (z - a_1 - b_1^2/(z - a_2 - ...)) ],
    z = omega + e0 - shift + i eta (reading of the resolvent; shift = h for S^-),
    evaluated from the deepest level up.  beta[x] couples levels x and x+1."""
    z = omega + e0 - shift + 1j * eta
    n = len(alpha)
    g = z - alpha[n - 1]
    for x in range(n - 2, -1, -1):
        g = z - alpha[x] - beta[x] ** 2 / g
    return -(norm2 / g).imag / np.pi
