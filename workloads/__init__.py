"""Seeded synthetic inputs for the IFMM workloads.

This module is shared by the CPU oracle, the tests, ``bench.py`` and the
CUDA path.  It draws random points and right-hand sides and states each
workload's parameters; it contains none of the method's arithmetic.

Seeds: points of system ``s`` of a workload with base seed ``B`` use
``B + s`` (bases 1000, 2000, 3000, 4000, 5000 for the five workloads below);
the right-hand sides of that system use the point seed + 1.  All draws use
numpy's PCG64 generator.

Workloads (the paper's own examples, Sec. 3.1-3.2, use random points in a
cube or on a sphere; these follow the same shapes):

* ``cube_2k``   N=2048 uniform in the unit cube, A_ij = 1/r, A_ii = 2 N^(1/3),
                leaves <= 64, Chebyshev 3x3x3, eps = 1e-6, 1 RHS.
* ``cube_64k``  N=65536 uniform in the unit cube, same kernel rule, leaves <= 64,
                Chebyshev 4x4x4, eps = 1e-8, 1 RHS (the bench workload).
* ``square_gauss_1m``  N=2^20 uniform in the unit square, Gaussian RBF
                sigma = 0.05 with 1e-2 added on the diagonal, leaves <= 128,
                Chebyshev 6x6, eps = 1e-6, 4 RHS.
* ``sphere_system(s)``  system s of 256, N log-uniform in [1024, 65536] on the
                unit sphere surface, A_ii = 2 sqrt(N), Chebyshev 4x4x4, eps = 1e-4.
* ``serving_cube_system(s)``  system s of 64, N log-uniform in [4096, 262144]
                in the unit cube, 1/r kernel, A_ii = 2 N^(1/3), Chebyshev 3x3x3,
                eps = 1e-6.
* ``paper_cube``  the replication workload of Sec. 3.2: N points uniform in
                [-1, 1]^3 with the kernel of Eq. (K_ij) (parameter d).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# kernel kinds, numbered as in include/ifmm.h
K_INV_R = 0
K_GAUSSIAN = 1
K_PAPER_D = 2


@dataclass
class Kernel:
    kind: int
    param: float = 0.0      # Gaussian sigma, or the paper kernel's d
    diag: float = float("nan")  # A_ii; NaN means "the kernel's own value at r = 0"


@dataclass
class Workload:
    name: str
    points: np.ndarray          # (N, dim) float64, user order
    kernel: Kernel
    dim: int
    cheb_n: int
    leaf_max: int
    eps: float
    nrhs: int
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.points.shape[0])

    def rhs(self, nrhs: int | None = None) -> np.ndarray:
        """Standard-normal right-hand sides, (N, nrhs) column-major-friendly."""
        k = self.nrhs if nrhs is None else nrhs
        g = np.random.Generator(np.random.PCG64(self.seed + 1))
        return np.asfortranarray(g.standard_normal((self.N, k)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(N: int, seed: int, dim: int = 3, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    g = _rng(seed)
    return np.ascontiguousarray(lo + (hi - lo) * g.random((N, dim)))


def unit_sphere(N: int, seed: int) -> np.ndarray:
    g = _rng(seed)
    v = g.standard_normal((N, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.ascontiguousarray(v)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> list[int]:
    g = _rng(seed)
    u = g.random(count)
    return [int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))))) for x in u]


def inv_r_cube(N: int, seed: int, name: str, cheb_n: int, leaf_max: int, eps: float,
               nrhs: int = 1) -> Workload:
    pts = uniform_cube(N, seed, 3)
    return Workload(name, pts, Kernel(K_INV_R, 0.0, 2.0 * N ** (1.0 / 3.0)), 3, cheb_n,
                    leaf_max, eps, nrhs, seed)


def cube_2k() -> Workload:
    """2,048 points uniform in the unit cube, 1/r, Chebyshev 3^3, eps = 1e-6."""
    return inv_r_cube(2048, 1000, "cube-2k", 3, 64, 1e-6)


def cube_64k() -> Workload:
    """65,536 points uniform in the unit cube, 1/r, Chebyshev 4^3, eps = 1e-8."""
    return inv_r_cube(65536, 2000, "cube-64k", 4, 64, 1e-8)


def square_gauss_1m(N: int = 1 << 20) -> Workload:
    """2^20 points uniform in the unit square, Gaussian RBF sigma = 0.05 with
    A_ii = 1.01, leaves <= 128, Chebyshev 6^2, eps = 1e-6, 4 right-hand sides."""
    seed = 3000
    pts = uniform_cube(N, seed, 2)
    return Workload("square-gauss-1m", pts, Kernel(K_GAUSSIAN, 0.05, 1.0 + 1e-2), 2, 6, 128, 1e-6, 4, seed)


def sphere_system(s: int) -> Workload:
    """System s of 256 on the unit sphere: N log-uniform in [1024, 65536],
    1/r with A_ii = 2 sqrt(N), Chebyshev 4^3, eps = 1e-4."""
    sizes = log_uniform_sizes(256, 1024, 65536, 4000 + 999)
    N = sizes[s]
    seed = 4000 + s
    pts = unit_sphere(N, seed)
    return Workload(f"sphere[{s}]", pts, Kernel(K_INV_R, 0.0, 2.0 * math.sqrt(N)), 3, 4, 64, 1e-4,
                    1, seed)


def serving_cube_system(s: int) -> Workload:
    """System s of 64 in the unit cube: N log-uniform in [4096, 262144], 1/r,
    Chebyshev 3^3, eps = 1e-6."""
    sizes = log_uniform_sizes(64, 4096, 262144, 5000 + 999)
    N = sizes[s]
    return inv_r_cube(N, 5000 + s, f"serving-cube[{s}]", 3, 64, 1e-6)


def paper_cube(N: int, d: float, cheb_n: int, seed: int = 6000, leaf_max: int = 100,
               eps: float = 1e-3) -> Workload:
    """Sec. 3.2: N random points in [-1,1]^3, kernel Eq. (K_ij) with parameter d."""
    pts = uniform_cube(N, seed, 3, -1.0, 1.0)
    return Workload(f"paper[N={N},d={d},n={cheb_n}]", pts, Kernel(K_PAPER_D, d, 1.0), 3, cheb_n,
                    leaf_max, eps, 1, seed)


def small_cube(N: int, seed: int, cheb_n: int = 3, leaf_max: int = 16, eps: float = 1e-6,
               dim: int = 3, kernel: Kernel | None = None) -> Workload:
    """Small seeded cases for parity tests (the cube recipes at reduced N)."""
    pts = uniform_cube(N, seed, dim)
    if kernel is None:
        kernel = Kernel(K_INV_R, 0.0, 2.0 * N ** (1.0 / dim))
    return Workload(f"small[N={N},d={dim},n={cheb_n}]", pts, kernel, dim, cheb_n, leaf_max, eps,
                    1, seed)


def by_name(name: str) -> Workload:
    table = {"cube-2k": cube_2k, "cube-64k": cube_64k, "square-gauss-1m": square_gauss_1m}
    return table[name]()
