"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  It holds lattice geometry, coupling draws, sampled instance lists
and the start-vector random numbers only -- none of the method's arithmetic.

Workloads follow the paper's benchmark systems: periodic chains, the 10x10
square lattice (static / dynamical structure factor study), the 10x10x10
cubic lattice (dispersion study), a bond-disordered open 32x32 square lattice
and a mix of small uneven instances.

Site numbering: r = x + Lx*(y + Ly*z), 0-based.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


@dataclass
class LatticeSpec:
    n_sites: int
    bi: np.ndarray
    bj: np.ndarray
    jxy: np.ndarray
    jz: np.ndarray
    h: np.ndarray | None = None
    L: tuple = (0, 0, 0)                 # translation group of the cells, (0,0,0) = none
    name: str = ""
    pos: np.ndarray | None = field(default=None, repr=False)
    n_sub: int = 1                       # spins per unit cell (site r: spin r % n_sub of cell r // n_sub)

    def as_dict(self) -> dict:
        return dict(n_sites=self.n_sites, bi=self.bi, bj=self.bj, jxy=self.jxy, jz=self.jz,
                    h=self.h, L=tuple(self.L), n_sub=int(self.n_sub))

    @property
    def n_bonds(self) -> int:
        return int(len(self.bi))


def hypercubic(dims: tuple, periodic: bool = True, J: float = 1.0, Jz: float | None = None,
               name: str = "") -> LatticeSpec:
    """Nearest-neighbour bonds r -> r + e_alpha of an Lx x Ly x Lz lattice."""
    dims = tuple(dims) + (1,) * (3 - len(dims))
    Lx, Ly, Lz = dims
    N = Lx * Ly * Lz
    Jz = J if Jz is None else Jz
    bi, bj = [], []
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                r = x + Lx * (y + Ly * z)
                for a, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    if dims[a] == 1:
                        continue
                    nx, ny, nz = x + dx, y + dy, z + dz
                    if (nx, ny, nz)[a] >= dims[a]:
                        if not periodic:
                            continue
                        nx, ny, nz = nx % Lx, ny % Ly, nz % Lz
                    s = nx + Lx * (ny + Ly * nz)
                    if s == r:
                        continue
                    bi.append(r)
                    bj.append(s)
    nb = len(bi)
    L = dims if periodic else (0, 0, 0)
    return LatticeSpec(N, np.array(bi, np.int32), np.array(bj, np.int32), np.full(nb, float(J)),
                       np.full(nb, float(Jz)), None, L, name or f"{'x'.join(map(str, dims))}")


def triangular(Lx: int, Ly: int | None = None, J: float = 1.0, Jz: float | None = None) -> LatticeSpec:
    """Periodic Lx x Ly triangular lattice: sites r = x + Lx y on the lattice
    vectors a1, a2 (60 degrees apart), bonds r -> r + a1, r + a2, r + a1 - a2
    (six neighbours).  The translation group is that of the Lx x Ly square,
    and momenta are taken in the a1, a2 coordinates."""
    Ly = Ly or Lx
    Jz = J if Jz is None else Jz
    bi, bj = [], []
    for y in range(Ly):
        for x in range(Lx):
            r = x + Lx * y
            for dx, dy in ((1, 0), (0, 1), (1, -1)):
                s = (x + dx) % Lx + Lx * ((y + dy) % Ly)
                if s != r:
                    bi.append(r)
                    bj.append(s)
    nb = len(bi)
    return LatticeSpec(Lx * Ly, np.array(bi, np.int32), np.array(bj, np.int32), np.full(nb, float(J)),
                       np.full(nb, float(Jz)), None, (Lx, Ly, 1), f"triangular{Lx}x{Ly}")


def chain(N: int, J: float = 1.0, Jz: float | None = None, periodic: bool = True) -> LatticeSpec:
    return hypercubic((N,), periodic, J, Jz, name=f"chain{N}")


def square(Lx: int, Ly: int | None = None, J: float = 1.0, Jz: float | None = None,
           periodic: bool = True) -> LatticeSpec:
    return hypercubic((Lx, Ly or Lx), periodic, J, Jz, name=f"square{Lx}x{Ly or Lx}")


def cubic(L: int, J: float = 1.0, Jz: float | None = None, periodic: bool = True) -> LatticeSpec:
    return hypercubic((L, L, L), periodic, J, Jz, name=f"cubic{L}")


def disordered_open_square(L: int = 32, seed: int = 20210702) -> LatticeSpec:
    """Open LxL square lattice with J ~ U[0.5,1.5], Jz = 0.8 J, h_i ~ U[-0.1,0.1]."""
    base = hypercubic((L, L), periodic=False)
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, base.n_bonds)
    h = rng.uniform(-0.1, 0.1, base.n_sites)
    return LatticeSpec(base.n_sites, base.bi, base.bj, J, 0.8 * J, h, (0, 0, 0),
                       f"disordered_open_square{L}")


def _cell_lattice(Lx: int, Ly: int, nsub: int, bonds, J: float, Jz: float | None, name: str) -> LatticeSpec:
    """Periodic Lx x Ly lattice of nsub-spin unit cells; bonds = [(s, s2, dx,
    dy)]: spin s of cell (x, y) to spin s2 of cell (x + dx, y + dy)."""
    Jz = J if Jz is None else Jz
    bi, bj = [], []
    for y in range(Ly):
        for x in range(Lx):
            for s, s2, dx, dy in bonds:
                a = s + nsub * (x + Lx * y)
                b = s2 + nsub * ((x + dx) % Lx + Lx * ((y + dy) % Ly))
                bi.append(min(a, b))
                bj.append(max(a, b))
    nb = len(bi)
    N = nsub * Lx * Ly
    return LatticeSpec(N, np.array(bi, np.int32), np.array(bj, np.int32), np.full(nb, float(J)),
                       np.full(nb, float(Jz)), None, (Lx, Ly, 1), name, None, nsub)


def honeycomb(Lx: int, Ly: int | None = None, J: float = 1.0, Jz: float | None = None) -> LatticeSpec:
    """Periodic honeycomb lattice of Lx x Ly two-spin cells (A = spin 0, B =
    spin 1): A(x, y) joins B(x, y), B(x - 1, y) and B(x, y - 1)."""
    Ly = Ly or Lx
    return _cell_lattice(Lx, Ly, 2, [(0, 1, 0, 0), (0, 1, -1, 0), (0, 1, 0, -1)], J, Jz, f"honeycomb{Lx}x{Ly}")


def kagome(Lx: int, Ly: int | None = None, J: float = 1.0, Jz: float | None = None) -> LatticeSpec:
    """Periodic kagome lattice of Lx x Ly three-spin cells (A, B, C = spins 0,
    1, 2 at 0, a1/2, a2/2): the up triangle A-B-C of each cell and the down
    triangle B(x, y), A(x + 1, y), C(x + 1, y - 1)."""
    Ly = Ly or Lx
    return _cell_lattice(Lx, Ly, 3, [(0, 1, 0, 0), (0, 2, 0, 0), (1, 2, 0, 0), (1, 0, 1, 0), (0, 2, 0, -1),
                                     (1, 2, 1, -1)], J, Jz, f"kagome{Lx}x{Ly}")


def random_graph(N: int, n_bonds: int, seed: int, field: bool = True) -> LatticeSpec:
    """Random XXZ couplings on a random graph (oracle pin tests)."""
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < n_bonds:
        i, j = rng.integers(0, N, 2)
        if i != j:
            pairs.add((min(i, j), max(i, j)))
    pairs = sorted(pairs)
    bi = np.array([p[0] for p in pairs], np.int32)
    bj = np.array([p[1] for p in pairs], np.int32)
    jxy = rng.uniform(-1.5, 1.5, n_bonds)
    jz = rng.uniform(-1.5, 1.5, n_bonds)
    h = rng.uniform(-0.5, 0.5, N) if field else None
    return LatticeSpec(N, bi, bj, jxy, jz, h, (0, 0, 0), f"random{N}_{seed}")


def all_k(L: tuple) -> list:
    L = tuple(L) + (1,) * (3 - len(L))
    return [(kx, ky, kz) for kz in range(L[2]) for ky in range(L[1]) for kx in range(L[0])]


def cubic_kpath(L: int = 10) -> list:
    """Gamma-X-M-Gamma-R-X | M-R on an LxLxL lattice with X=(0,0,pi),
    M=(0,pi,pi), R=(pi,pi,pi): 31 path points for L=10 (Gamma, X and R are visited twice, so
    28 distinct sectors)."""
    h = L // 2
    G, X, M, R = (0, 0, 0), (0, 0, h), (0, h, h), (h, h, h)

    def seg(a, b):
        n = max(abs(b[i] - a[i]) for i in range(3))
        return [tuple(a[i] + (b[i] - a[i]) * s // n for i in range(3)) for s in range(n + 1)]

    pts = [G]
    for a, b in ((G, X), (X, M), (M, G), (G, R), (R, X)):
        pts += seg(a, b)[1:]
    pts += seg(M, R)[1:]                        # the separate M-R branch
    return [(p[2], p[1], p[0]) for p in pts]       # (Kx, Ky, Kz) with X along z


# --------------------------------------------------------------- start vector


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), vectorised."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def gaussian_start(seed: int, d: int, complex_: bool) -> np.ndarray:
    """Seeded Gaussian start vector: Box-Muller on two SplitMix64 draws per
    real number, uniforms on (0,1] from the top 53 bits.  Element i uses
    counters 2i, 2i+1 (real part) and 2(d+i), 2(d+i)+1 (imaginary part)."""
    def normals(base: int, n: int) -> np.ndarray:
        i = np.arange(n, dtype=np.uint64) + np.uint64(base)
        s = np.uint64(seed & MASK64)
        u1 = ((splitmix64(s ^ (np.uint64(2) * i)) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = ((splitmix64(s ^ (np.uint64(2) * i + np.uint64(1))) >> np.uint64(11)).astype(np.float64) + 1.0) \
            * 2.0 ** -53
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    re = normals(0, d)
    if not complex_:
        return re
    return re + 1j * normals(d, d)


# ------------------------------------------------------- uneven instance mix


def instance_mix(n: int = 64, seed0: int = 5000, dim_range=(1e3, 1e7)):
    """Seeded uneven XXZ instances: chains of 24-64 sites, LxL squares with
    L=6-12, LxLxL cubes with L=4-6, periodic, Delta ~ U[0.5,1.5] (Jz = Delta J,
    J = 1), N_down ~ U{2..5}, half with a random momentum sector.  Each seed
    is redrawn (seed + 1000 k) until the U(1) or sector dimension, estimated
    as C(N, Nd) / N for k-sectors, lies in dim_range."""
    from math import comb
    out = []
    for i in range(n):
        s = seed0 + i
        while True:
            rng = np.random.default_rng(s)
            fam = int(rng.integers(0, 3))
            if fam == 0:
                N = int(rng.integers(24, 65))
                dims = (N, 1, 1)
            elif fam == 1:
                Ls = int(rng.integers(6, 13))
                dims = (Ls, Ls, 1)
            else:
                Ls = int(rng.integers(4, 7))
                dims = (Ls, Ls, Ls)
            delta = float(rng.uniform(0.5, 1.5))
            nd = int(rng.integers(2, 6))
            use_k = bool(rng.integers(0, 2))
            Nsite = dims[0] * dims[1] * dims[2]
            K = tuple(int(rng.integers(0, dims[a])) for a in range(3)) if use_k else None
            est = comb(Nsite, nd) / (Nsite if use_k else 1)
            if dim_range[0] <= est <= dim_range[1]:
                lat = hypercubic(dims, True, 1.0, delta)
                lat.name = f"inst{i}_{lat.name}"
                out.append(dict(lattice=lat, n_down=nd, K=K, seed=s))
                break
            s += 1000
    return out
