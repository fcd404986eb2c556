"""Independent constructions that pin the oracle (and, through it, the GPU
path): nothing here calls the oracle or the GPU library.

- colex enumeration of subsets by brute force (itertools), which fixes the
  ordering that Eq. (a_of_n) must reproduce;
- the spin-1/2 Hamiltonian of Eq. (1) built from Kronecker products of the
  spin matrices, and an equivalent bit-string construction;
- translations of site sets by coordinate arithmetic;
- closed forms: sector dimensions by a character sum over the translation
  group, the one-magnon dispersion, the two-magnon chain spectrum from the
  two-body problem in the relative coordinate.
"""
from __future__ import annotations

import itertools
from math import comb, gcd

import numpy as np


def colex_subsets(N: int, nd: int) -> list:
    """All nd-subsets of range(N), sorted in colexicographic order (compare
    the largest element first)."""
    subs = list(itertools.combinations(range(N), nd))
    subs.sort(key=lambda c: tuple(reversed(c)))
    return subs


def kron_hamiltonian(spec) -> np.ndarray:
    """Eq. (1) (plus the site field -sum h_i s^z_i) on the full 2^N space from
    Kronecker products; basis bit i (little endian) = 1 means spin down."""
    N = spec.n_sites
    sx = np.array([[0, 0.5], [0.5, 0]])
    sy = np.array([[0, -0.5j], [0.5j, 0]])
    sz = np.array([[0.5, 0], [0, -0.5]])
    eye = np.eye(2)

    def op(mats: dict) -> np.ndarray:
        out = np.array([[1.0 + 0j]])
        for i in reversed(range(N)):          # site N-1 is the most significant factor
            out = np.kron(out, mats.get(i, eye))
        return out

    H = np.zeros((2 ** N, 2 ** N), np.complex128)
    for b in range(len(spec.bi)):
        i, j = int(spec.bi[b]), int(spec.bj[b])
        H += spec.jxy[b] * (op({i: sx, j: sx}) + op({i: sy, j: sy})) + spec.jz[b] * op({i: sz, j: sz})
    if spec.h is not None:
        for i in range(N):
            H -= spec.h[i] * op({i: sz})
    return H


def bit_hamiltonian_sector(spec, nd: int) -> np.ndarray:
    """The N_down = nd block of Eq. (1) built on bit strings, rows in colex
    order of the down-spin sets."""
    N = spec.n_sites
    subs = colex_subsets(N, nd)
    index = {sum(1 << s for s in c): k for k, c in enumerate(subs)}
    D = len(subs)
    H = np.zeros((D, D))
    for k, c in enumerate(subs):
        bits = sum(1 << s for s in c)
        for b in range(len(spec.bi)):
            i, j = int(spec.bi[b]), int(spec.bj[b])
            di, dj = (bits >> i) & 1, (bits >> j) & 1
            H[k, k] += spec.jz[b] * (0.25 if di == dj else -0.25)
            if di != dj:
                H[index[bits ^ (1 << i) ^ (1 << j)], k] += spec.jxy[b] / 2
        if spec.h is not None:
            for i in range(N):
                H[k, k] -= spec.h[i] * (-0.5 if (bits >> i) & 1 else 0.5)
    return H


def sector_projector(N: int, nd: int) -> np.ndarray:
    """Columns: full-space basis vectors of the nd-down states, colex order."""
    subs = colex_subsets(N, nd)
    P = np.zeros((2 ** N, len(subs)))
    for k, c in enumerate(subs):
        P[sum(1 << s for s in c), k] = 1.0
    return P


def coords(r: int, L, nsub: int = 1) -> tuple:
    """cell coordinates of site r (spin r % nsub of cell r // nsub)"""
    q = r // nsub
    return q % L[0], (q // L[0]) % L[1], q // (L[0] * L[1])


def translate_set(c, t, L, nsub: int = 1) -> tuple:
    """the site set c with every cell moved by t (each spin keeps its place in the cell)"""
    out = []
    for r in c:
        x, y, z = coords(r, L, nsub)
        x, y, z = (x + t[0]) % L[0], (y + t[1]) % L[1], (z + t[2]) % L[2]
        out.append(r % nsub + nsub * (x + L[0] * (y + L[1] * z)))
    return tuple(sorted(out))


def group(L) -> list:
    return [(tx, ty, tz) for tz in range(L[2]) for ty in range(L[1]) for tx in range(L[0])]


def order(t, L) -> int:
    o = 1
    for a in range(3):
        o = o * (L[a] // gcd(L[a], t[a])) // gcd(o, L[a] // gcd(L[a], t[a]))
    return o


def sector_dim_closed_form(L, nd: int, K, nsub: int = 1) -> int:
    """dim_k = (1/G) sum_t e^{-ik.t} [o(t) | nd] C(N/o(t), nd/o(t)) over the G =
    Lx Ly Lz cell translations t of an N = nsub G site lattice: the number of
    nd-subsets fixed by t is C(N/o, nd/o) when o divides nd (t moves every
    site in cycles of length o, N/o of them), and 0 otherwise."""
    G = L[0] * L[1] * L[2]
    N = nsub * G
    s = 0j
    for t in group(L):
        o = order(t, L)
        if nd % o == 0:
            ph = np.exp(-2j * np.pi * sum(K[a] * t[a] / L[a] for a in range(3)))
            s += ph * comb(N // o, nd // o)
    v = s / G
    assert abs(v.imag) < 1e-6 and abs(v.real - round(v.real)) < 1e-6
    return int(round(v.real))


def one_magnon_energy(spec, K) -> float:
    """E(k) of one down spin on a uniform periodic hypercubic lattice:
    sum_b Jz/4 - z Jz/2 + (J/2) sum_{delta} e^{ik.delta}."""
    L = spec.L
    nb = len(spec.bi)
    J, Jz = spec.jxy[0], spec.jz[0]
    D = sum(1 for a in range(3) if L[a] > 1)
    z = 2 * D
    hop = sum(2 * np.cos(2 * np.pi * K[a] / L[a]) for a in range(3) if L[a] > 1)
    return nb * Jz / 4 - z * Jz / 2 + J / 2 * hop


def two_magnon_chain_spectrum(N: int, J: float, Jz: float) -> np.ndarray:
    """All C(N, 2) levels of two down spins on the uniform periodic chain of
    odd length N, from the two-body problem in the relative coordinate.

    For total momentum K = 2 pi n / N the states |K, r> = N^{-1/2} sum_x
    e^{iKx} |{x, x+r}> (r = 1..R, R = (N-1)/2) are orthonormal, and
    |K, N-r> = e^{iKr} |K, r>.  Each down spin hops with amplitude J/2: the
    spin at x moves to x -/+ 1 (separation r +/- 1, phase e^{+/-iK}), the one
    at x + r to x + r +/- 1, so H|K,r> = d(r)|K,r> + (J/2)[(1 + e^{iK})|K,r+1>
    + (1 + e^{-iK})|K,r-1>], with no |K,0> (hard core) and |K,R+1> =
    e^{iKR}|K,R>.  The diagonal is the ferromagnetic energy N Jz/4 minus Jz
    per flipped spin's two broken bonds, -2 Jz, plus Jz when the two spins are
    neighbours (r = 1: their common bond stays satisfied)."""
    assert N % 2 == 1 and N >= 5
    R = (N - 1) // 2
    out = []
    for n in range(N):
        K = 2 * np.pi * n / N
        M = np.zeros((R, R), np.complex128)
        for r in range(1, R + 1):
            M[r - 1, r - 1] = N * Jz / 4 - 2 * Jz + (Jz if r == 1 else 0.0)
            if r < R:
                M[r, r - 1] += J / 2 * (1 + np.exp(1j * K))          # <K, r+1| H |K, r>
                M[r - 1, r] += J / 2 * (1 + np.exp(-1j * K))         # <K, r| H |K, r+1>
        M[R - 1, R - 1] += J / 2 * (1 + np.exp(1j * K)) * np.exp(1j * K * R)
        out.extend(np.linalg.eigvalsh(M))
    return np.sort(np.array(out))
