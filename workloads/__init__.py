"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and bench.py.

This module only draws data.  It holds none of the method's arithmetic (no kinetic
operator, no shift, no pole rule, no solver): potentials sampled on a periodic grid,
Gaussian starting blocks, and the table of workloads with their sizes.

Grid convention (Sec. 4, Test 1): the box is [0, L)^d sampled at x_j = L*j/m in each
dimension; a grid function is stored as one contiguous column of n = prod(m) values with
the x index fastest, i.e. flat index = x + m_x*(y + m_y*z).

The potentials mimic the paper's test potentials (Sec. 4): Gaussian wells on a periodic
box (Test 1-3 use a Gaussian well per cell), and a smooth random field.  The paper does
not print the well depth/width, so the sizes below are the workload definitions of this
project, not values from the paper.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np


def grid_coords(m: Sequence[int], L: float) -> list[np.ndarray]:
    """Per-axis sample coordinates x_j = L*j/m_axis (axis order x, y, z)."""
    return [L * np.arange(mi) / mi for mi in m]


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def gaussian_wells(m: Sequence[int], L: float, centers: np.ndarray, depths: np.ndarray,
                   width: float) -> np.ndarray:
    """V(x) = -sum_i depth_i * exp(-|x - c_i|^2 / (2 width^2)), periodic (minimum image).

    Returns a float64 array of n values in flat order (x fastest).
    """
    d = len(m)
    coords = grid_coords(m, L)
    # mesh in (z, y, x) order so that a C-order ravel gives x fastest
    mesh = np.meshgrid(*coords[::-1], indexing="ij")[::-1]  # mesh[0]=x, mesh[1]=y, ...
    V = np.zeros(mesh[0].shape)
    for c, dep in zip(centers, depths):
        r2 = np.zeros_like(V)
        for a in range(d):
            r2 += _min_image(mesh[a] - c[a], L) ** 2
        V -= dep * np.exp(-r2 / (2.0 * width * width))
    return V.ravel().astype(np.float64)


def wells_2d(m: int, L: float = 10.0, n_wells: int = 4, seed: int = 0,
             depth_range=(5.0, 10.0), width_frac: float = 0.1) -> np.ndarray:
    """2D: n_wells Gaussian wells, depth ~ U[5,10], width (std) = 0.1 L, centres ~ U[0,L)^2."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, L, size=(n_wells, 2))
    depths = rng.uniform(depth_range[0], depth_range[1], size=n_wells)
    return gaussian_wells((m, m), L, centers, depths, width_frac * L)


def smooth_field_2d(m: int, L: float = 10.0, amplitude: float = 10.0, seed: int = 0,
                    decay: float = 8.0) -> np.ndarray:
    """2D smooth random field: Fourier coefficients (a+ib)*exp(-|k|^2/decay), a,b ~ N(0,1),
    integer wave vectors k; V = Re(inverse DFT), rescaled so that max|V| = amplitude."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(m, 1.0 / m)
    k2 = k[:, None] ** 2 + k[None, :] ** 2          # (y, x)
    c = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) * np.exp(-k2 / decay)
    V = np.real(np.fft.ifft2(c))
    V *= amplitude / np.max(np.abs(V))
    return V.ravel().astype(np.float64)


def lattice_wells_3d(m: int, L: float = 40.0, cells: int = 4, depth: float = 8.0,
                     width_frac: float = 0.08) -> np.ndarray:
    """3D: one Gaussian well (depth 8, std 0.08 lattice constants) per cell of a
    cells^3 simple-cubic lattice with lattice constant a = L/cells, wells at the cell
    centres."""
    a = L / cells
    idx = (np.arange(cells) + 0.5) * a
    centers = np.array([[x, y, z] for z in idx for y in idx for x in idx])
    return gaussian_wells((m, m, m), L, centers, np.full(len(centers), depth), width_frac * a)


def gaussian_block(n: int, N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex Gaussian n x N block, real and imaginary parts ~ N(0, 1/(2n)), so that each
    column has unit expected norm.  Returned column-major as an (N, n) C-order array whose
    row j is column j (the device layout: column j at offset j*n)."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(0.5 / n)
    Z = s * (rng.standard_normal((N, n)) + 1j * rng.standard_normal((N, n)))
    return Z.astype(dtype)


def gaussian_block_real(n: int, N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Real Gaussian n x N block, entries ~ N(0, 1/n) (unit expected column norm), in the
    same (N, n) row-per-column layout as gaussian_block, imaginary parts zero."""
    rng = np.random.default_rng(seed)
    Z = np.sqrt(1.0 / n) * rng.standard_normal((N, n))
    return Z.astype(dtype)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    m: int            # points per dimension
    L: float          # box length
    N: int            # number of states
    P: int            # number of poles
    potential: str    # 'wells2d' | 'smooth2d' | 'lattice3d'
    seed: int = 0
    precision: str = "fp64"   # 'fp64' | 'mixed'

    @property
    def n(self) -> int:
        return self.m ** self.dim

    @property
    def shape(self) -> tuple:
        return (self.m,) * self.dim

    def potential_values(self) -> np.ndarray:
        if self.potential == "wells2d":
            return wells_2d(self.m, self.L, seed=self.seed)
        if self.potential == "smooth2d":
            return smooth_field_2d(self.m, self.L, seed=self.seed)
        if self.potential == "lattice3d":
            return lattice_wells_3d(self.m, self.L)
        raise ValueError(self.potential)

    def initial_block(self, dtype=np.complex128, real: bool = False) -> np.ndarray:
        """The seeded starting block; real=True gives the real block of the same seed
        (real orbitals, stored in the complex dtype with zero imaginary parts)."""
        if real:
            return gaussian_block_real(self.n, self.N, seed=1000 + self.seed, dtype=dtype)
        return gaussian_block(self.n, self.N, seed=1000 + self.seed, dtype=dtype)


# The workloads.  'wells2d-32' is the small case whose whole solve the oracle finishes in
# seconds; 'smooth2d-128' is the 2D 128^2, N=128, 16-pole mixed-precision solve;
# 'lattice3d-48' the 3D 48^3, N=256 lattice.
WORKLOADS = {
    "wells2d-32": Workload("wells2d-32", 2, 32, 10.0, 16, 16, "wells2d", 0, "fp64"),
    "smooth2d-128": Workload("smooth2d-128", 2, 128, 10.0, 128, 16, "smooth2d", 0, "mixed"),
    "lattice3d-48": Workload("lattice3d-48", 3, 48, 40.0, 256, 16, "lattice3d", 0, "mixed"),
}


def small_case(m: int = 16, N: int = 8, dim: int = 2, L: float = 10.0, seed: int = 0,
               potential: str = "wells2d") -> Workload:
    """A tiny workload for parity tests (dense oracle on n <= 4096)."""
    pot = potential if dim == 2 else "lattice3d"
    return Workload(f"small-{dim}d-{m}-{N}", dim, m, L, N, 16, pot, seed, "fp64")


# ---- many-Hamiltonian workloads (batched and served solves)
@dataclasses.dataclass(frozen=True)
class HamSpec:
    key: str
    m: int
    N: int
    L: float
    potential: str     # 'smooth2d' | 'wells2d' | 'lattice3d'
    seed: int
    dim: int = 2

    @property
    def n(self) -> int:
        return self.m ** self.dim

    @property
    def shape(self) -> tuple:
        return (self.m,) * self.dim

    def potential_values(self) -> np.ndarray:
        if self.potential == "smooth2d":
            return smooth_field_2d(self.m, self.L, seed=self.seed)
        if self.potential == "lattice3d":
            return lattice_wells_3d(self.m, self.L)
        return wells_2d(self.m, self.L, seed=self.seed)


def batch_mix(count: int = 64, seed: int = 0) -> list:
    """Independent 2D Hamiltonians: grid uniform from {32, 64, 96, 128}^2, N uniform in
    [16, 128] (at most n/4), smooth random V (seed 100 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice([32, 64, 96, 128]))
        N = int(rng.integers(16, 129))
        N = min(N, m * m // 4)
        out.append(HamSpec(f"batch{i}", m, N, 10.0, "smooth2d", 100 + i))
    return out


def serving_mix(count: int = 12, seed: int = 1) -> list:
    """Distinct Hamiltonians a request stream draws from: 2D grids from {64, 72, 96, 128}^2,
    N uniform in [32, 128], four Gaussian wells per box (seed 200 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice([64, 72, 96, 128]))
        N = int(rng.integers(32, 129))
        out.append(HamSpec(f"serve{i}", m, N, 10.0, "wells2d", 200 + i))
    return out


def serving_mix_wide(count: int = 4, seed: int = 3) -> list:
    """More served 2D Hamiltonians, with N uniform in [129, 256] (at most n/4): grids from
    {64, 96, 128}^2, four Gaussian wells per box (seed 220 + i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.choice([64, 96, 128]))
        N = min(int(rng.integers(129, 257)), m * m // 4)
        out.append(HamSpec(f"serve-wide{i}", m, N, 10.0, "wells2d", 220 + i))
    return out


def serving_mix_3d() -> list:
    """Served 3D Hamiltonians: the 4^3 lattice of Gaussian wells of the 48^3 workload (box
    L = 40) on a 32^3 grid with N = 64 (the s band; its p band is not separated from the
    next states at 8 points per cell) and on 48^3 with N = 64 and N = 256 (s and p bands)."""
    return [HamSpec("serve3d-32", 32, 64, 40.0, "lattice3d", 300, 3),
            HamSpec("serve3d-48s", 48, 64, 40.0, "lattice3d", 301, 3),
            HamSpec("serve3d-48", 48, 256, 40.0, "lattice3d", 302, 3)]


def poisson_arrivals(count: int, rate: float, nkeys: int, seed: int = 2):
    """Arrival times (s) of `count` requests at `rate` per second and the Hamiltonian index
    each one asks for (uniform over nkeys)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    keys = rng.integers(0, nkeys, size=count)
    return t, keys
