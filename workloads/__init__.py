"""Seeded synthetic workloads for the parametric RTE solver.

This module only describes problems: mesh sizes, quadrature orders, region
grids, source boxes and the random draws of the material parameters.  It
holds none of the method's arithmetic (no quadrature nodes, no basis, no
operators), so both the CUDA path and the CPU oracle may consume it.

Parameter draws use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014):
    x += 0x9E3779B97F4A7C15
    z = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)
and u = (out >> 11) * 2^-53 in [0, 1).  Per instance, sigma_s[0..R) is drawn
first, then sigma_a[0..R), regions in row-major order (iy * Rx + ix).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (published constants, see module docstring)."""

    def __init__(self, seed: int):
        self.x = seed & _MASK

    def next_u64(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & _MASK
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class ProblemSpec:
    """Geometry, discretisation orders and parameter distribution of one workload.

    dim        1 (slab) or 2 (X-Y geometry).
    nx, ny     cells per instance (lists of length n_instances; ny = 1 in 1D).
    box        domain (x0, x1, y0, y1); y ignored in 1D.
    n_polar    1D: Gauss-Legendre points in mu on [-1, 1];
               2D: Gauss-Legendre points for Omega_z (Chebyshev-Legendre product rule).
    n_azim     2D: Chebyshev azimuthal points (ignored in 1D).
    rx, ry     region grid (equal blocks); R = rx * ry regions.
    src_q      isotropic source value inside src_box, zero outside.
    src_box    (xa, xb, ya, yb); y ignored in 1D.
    inflow_g   isotropic inflow value on the inflow boundary faces (0 = vacuum).
    sigma_s_range  log-uniform range of sigma_s per region.
    sigma_a_range  uniform range of sigma_a per region.
    src_gauss  None, or (A, a, xc, yc): the source A exp(-a ((x-xc)^2 + (y-yc)^2)) replaces the box source.
    inflow_faces  domain faces that carry the inflow g: a subset of ("x-", "x+", "y-", "y+") (2D).
    sigma_modes   None: sigma_s and sigma_a are constant on each of the R regions.  "variable_scattering":
               the R = 2 entries are the coefficients of two cross-section profiles over the whole domain,
               sigma(x, y) = c_0 f(x, y) + c_1 with f = r^4 (2 - r^2)^2 inside the unit disc and 1 outside
               (r^2 = x^2 + y^2), so that Sigma is a full 4x4 block per cell (2D).
    """

    name: str
    dim: int
    nx: List[int]
    ny: List[int]
    box: Sequence[float]
    n_polar: int
    n_azim: int
    rx: int
    ry: int
    src_q: float
    src_box: Sequence[float]
    inflow_g: float
    sigma_s_range: Sequence[float]
    sigma_a_range: Sequence[float]
    restart: int = 30
    rtol: float = 1e-10
    rom_rank: int = 32
    window: int = 2
    n_train: int = 20
    src_gauss: Optional[Sequence[float]] = None
    inflow_faces: Sequence[str] = ("x-", "x+", "y-", "y+")
    sigma_modes: Optional[str] = None

    @property
    def n_instances(self) -> int:
        return len(self.nx)

    @property
    def n_regions(self) -> int:
        return self.rx * self.ry

    @property
    def n_directions(self) -> int:
        return self.n_polar if self.dim == 1 else self.n_polar * self.n_azim

    @property
    def dofs_per_cell(self) -> int:
        return 2 if self.dim == 1 else 4

    def ndof(self, b: int) -> int:
        return self.nx[b] * self.ny[b] * self.dofs_per_cell

    def with_instances(self, nx: Sequence[int], ny: Sequence[int]) -> "ProblemSpec":
        return dataclasses.replace(self, nx=list(nx), ny=list(ny))

    def with_mesh(self, nx: int, ny: int, n_instances: int = 1) -> "ProblemSpec":
        return dataclasses.replace(self, nx=[nx] * n_instances, ny=[ny] * n_instances)


def draw_params(spec: ProblemSpec, n: int, seed: int):
    """Draw n parameter instances: (sigma_s[n][R], sigma_a[n][R]) as float64 arrays."""
    rng = SplitMix64(seed)
    R = spec.n_regions
    lo, hi = spec.sigma_s_range
    alo, ahi = spec.sigma_a_range
    ss = np.empty((n, R))
    sa = np.empty((n, R))
    for i in range(n):
        for r in range(R):
            u = rng.uniform()
            ss[i, r] = math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
        for r in range(R):
            u = rng.uniform()
            sa[i, r] = alo + u * (ahi - alo)
    return ss, sa


def seed_for(config: int, split: int) -> int:
    """Seed of a configuration's draw: 1000 * config + split (0 train, 1 test)."""
    return 1000 * config + split


def config(n: int) -> ProblemSpec:
    """The five workloads of the hot path, sized as stated in their descriptions.

    1: 1D slab [0,1], 128 cells, 16-point GL, 4 regions, source q=1 on [0.25,0.5].
    2: 2D [0,1]^2, 64x64, 8 polar GL x 16 azimuthal, 2x2 regions, source in the
       central 0.2x0.2 box.
    3: config 2's problem, 256 instances on 96 x 32^2, 96 x 64^2, 64 x 128^2.
    4: config 2's problem with rank-32 ROM and an MLP (2048 train / 512 test).
    5: 256x256, 8 polar x 24 azimuthal, 8x8 regions, sigma_s in [1,1e4],
       sigma_a in [0,1], 64 instances, restart 40.
    """
    if n == 1:
        return ProblemSpec("slab1d_128", 1, [128], [1], (0.0, 1.0, 0.0, 1.0), 16, 1, 4, 1,
                           1.0, (0.25, 0.5, 0.0, 1.0), 0.0, (1.0, 100.0), (0.0, 1.0),
                           restart=30, rtol=1e-10, rom_rank=10, window=2, n_train=20)
    base2 = ProblemSpec("square2d_64", 2, [64], [64], (0.0, 1.0, 0.0, 1.0), 8, 16, 2, 2,
                        1.0, (0.4, 0.6, 0.4, 0.6), 0.0, (1.0, 1e3), (0.0, 0.5),
                        restart=30, rtol=1e-10, rom_rank=32, window=2, n_train=64)
    if n == 2:
        return base2
    if n == 3:
        nx = [32] * 96 + [64] * 96 + [128] * 64
        return dataclasses.replace(base2, name="batch256_uneven", nx=nx, ny=list(nx), rtol=1e-8)
    if n == 4:
        return dataclasses.replace(base2, name="learned_64", rtol=1e-8, n_train=2048)
    if n == 5:
        return ProblemSpec("large256_192", 2, [256] * 64, [256] * 64, (0.0, 1.0, 0.0, 1.0), 8, 24,
                           8, 8, 1.0, (0.4, 0.6, 0.4, 0.6), 0.0, (1.0, 1e4), (0.0, 1.0),
                           restart=40, rtol=1e-8, rom_rank=32, window=2, n_train=256)
    raise ValueError(f"no workload {n}")


# ---------------------------------------------------------------- the paper's other 2D problems (N2)
# Region grid 4 x 4 on [-1, 1]^2: the central 2 x 2 blocks are the inner square |x|, |y| <= 0.5.
_INNER = (5, 6, 9, 10)


def pincell() -> ProblemSpec:
    """Pin-cell problem (Sec. 5): [-1,1]^2, 80 x 80 cells, CL(30, 6), zero inflow, source exp(-100 (x^2+y^2)),
    sigma_s = 100 and sigma_a = 0 outside the inner square, (sigma_a, sigma_s) = (mu_a, mu_s) in
    [0.05, 0.5]^2 inside; relative residual 1e-11."""
    return ProblemSpec("pincell_80", 2, [80], [80], (-1.0, 1.0, -1.0, 1.0), 6, 30, 4, 4,
                       0.0, (0.0, 0.0, 0.0, 0.0), 0.0, (0.05, 0.5), (0.05, 0.5),
                       restart=30, rtol=1e-11, rom_rank=64, window=2, n_train=25, src_gauss=(1.0, 100.0, 0.0, 0.0))


def pincell_params(mu_a: float, mu_s: float):
    """Per-region (sigma_s [16], sigma_a [16]) of the pin-cell problem for one parameter point."""
    ss = np.full(16, 100.0)
    sa = np.zeros(16)
    for r in _INNER:
        ss[r], sa[r] = mu_s, mu_a
    return ss, sa


def param_inflow() -> ProblemSpec:
    """Two-material problem with a parametric inflow (Sec. 5): [-1,1]^2, 64 x 64 cells, CL(60, 6), no source,
    sigma_s = mu_s and sigma_a = 0 in the inner square, sigma_s = 0 and sigma_a = 1 outside; inflow
    mu_bc on the left face only (Omega_x > 0); mu = (mu_s, mu_bc) in [1, 5] x [0.5, 1.5]; residual 1e-11.
    The inflow value is the spec's inflow_g (set per parameter point with dataclasses.replace)."""
    return ProblemSpec("param_inflow_64", 2, [64], [64], (-1.0, 1.0, -1.0, 1.0), 6, 60, 4, 4,
                       0.0, (0.0, 0.0, 0.0, 0.0), 1.0, (1.0, 5.0), (0.0, 0.0),
                       restart=30, rtol=1e-11, rom_rank=32, window=2, n_train=99, inflow_faces=("x-",))


def param_inflow_params(mu_s: float):
    """Per-region (sigma_s [16], sigma_a [16]) of the two-material problem."""
    ss = np.zeros(16)
    sa = np.ones(16)
    for r in _INNER:
        ss[r], sa[r] = mu_s, 0.0
    return ss, sa


def variable_scattering() -> ProblemSpec:
    """Variable-scattering problem (Sec. 5): [-1,1]^2, 80 x 80 cells, CL(30, 6), zero inflow, source
    (10/pi) exp(-100 (x^2+y^2)), sigma_a = 0 and sigma_s = mu_s f + 0.1 with the profile f of sigma_modes,
    mu_s in [49.9, 99.9]; 51 training points, window 2, eps_ROM 1e-9, relative residual 1e-11."""
    return ProblemSpec("varscat_80", 2, [80], [80], (-1.0, 1.0, -1.0, 1.0), 6, 30, 2, 1,
                       0.0, (0.0, 0.0, 0.0, 0.0), 0.0, (49.9, 99.9), (0.0, 0.0),
                       restart=30, rtol=1e-11, rom_rank=32, window=2, n_train=51,
                       src_gauss=(10.0 / np.pi, 100.0, 0.0, 0.0), sigma_modes="variable_scattering")


def variable_scattering_params(mu_s: float):
    """Mode coefficients (sigma_s [2], sigma_a [2]) of the variable-scattering problem: sigma_s = mu_s f + 0.1."""
    return np.array([mu_s, 0.1]), np.zeros(2)


def draw_box(n: int, lo: Sequence[float], hi: Sequence[float], seed: int) -> np.ndarray:
    """n points uniform in the box [lo, hi] (SplitMix64, coordinates in order): [n][len(lo)]."""
    rng = SplitMix64(seed)
    out = np.empty((n, len(lo)))
    for i in range(n):
        for k in range(len(lo)):
            out[i, k] = lo[k] + rng.uniform() * (hi[k] - lo[k])
    return out
