"""Seeded synthetic inputs for the ROM hot path.

This module builds problem data only -- grids, cross sections, sources, inflow
values and plain random numbers -- and holds none of the method's arithmetic
(no quadrature, no sweep, no source iteration).  Both the CUDA path and the
FP64 oracle take their inputs from here; neither is imported by this module.

Workloads (all synthetic; the paper uses no datasets):
  * ``example_2_1``   -- Example 2.1 of the paper (Sec. 2): [0,1]^2, sigma_T = 1,
    sigma_S = 0.5, q = 2 on [0.4,0.6]^2, vacuum inflow.
  * ``dom_small``     -- 32 x 32 on [0,1]^2, sigma_T = 1, sigma_S = 0.5, q = 1 on the
    central 8 x 8 cells (12..19), vacuum; 4 polar x 8 azimuthal product set.
  * ``point_source``  -- 256 x 256 on [-1,1]^2, sigma_T = 1, sigma_S = 0.9, Gaussian
    source exp(-r^2 / (2 * 0.02^2)) at the centre, vacuum; ROM 64 samples x 16
    ordinates against plain DOM with 256 ordinates.
  * ``checkerboard``  -- 448 x 448 on [0,7]^2, 7 x 7 blocks of 64 x 64 cells; absorber
    blocks (bi + bj even, except the centre) sigma_T = 10, sigma_S = 0; background
    sigma_T = 1, sigma_S = 0.9; q = 1 on the centre block; 256 samples with M drawn
    uniformly from {8, 16, 32, 64}.
  * ``hg_disc``       -- 512 x 512 on [0,1]^2, sigma_T = 1, sigma_S = 0.95, Henyey-
    Greenstein g = 0.8, q = 1 where |z - (0.5,0.5)| <= 0.05; 32 samples x 128.
  * ``lognormal_cube`` -- 3D, 128^3 on [0,1]^3, sigma_T = exp(-0.125 + 0.5 G) with G a
    unit-variance Gaussian random field (white noise from a seeded PCG64 stream,
    convolved by FFT with a Gaussian of standard deviation 8/sqrt(2) cells, i.e.
    covariance exp(-r^2 / (2 * 8^2)), periodic), so E[sigma_T] = 1; sigma_S =
    0.8 sigma_T; q = 1 on the central 8^3 cells (60..67); vacuum; 64 samples x 48
    ordinates (8 octants x 2 x 3 cells).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem2D:
    name: str
    I: int
    J: int
    bounds: tuple  # (x_L, x_R, y_B, y_T)
    sigma_t: np.ndarray  # [J, I]
    sigma_s: np.ndarray  # [J, I]
    q: np.ndarray  # [J, I]
    kernel: str = "iso"
    g: float = 0.0
    # ordinate description: ("rom", n_samples, m_per_quadrant list) or ("uniform", N) ...
    ordinates: dict = field(default_factory=dict)
    inflow: np.ndarray | None = None  # isotropic face values [2J + 2I] or None (vacuum)

    @property
    def n_cells(self) -> int:
        return self.I * self.J

    def centres(self):
        xl, xr, yb, yt = self.bounds
        dx, dy = (xr - xl) / self.I, (yt - yb) / self.J
        x = xl + (np.arange(self.I) + 0.5) * dx
        y = yb + (np.arange(self.J) + 0.5) * dy
        return np.meshgrid(x, y, indexing="xy")  # X[j, i], Y[j, i]


def _centres(I, J, bounds):
    xl, xr, yb, yt = bounds
    x = xl + (np.arange(I) + 0.5) * (xr - xl) / I
    y = yb + (np.arange(J) + 0.5) * (yt - yb) / J
    return np.meshgrid(x, y, indexing="xy")


def example_2_1(I: int = 100, J: int = 100, g: float = 0.0) -> Problem2D:
    bounds = (0.0, 1.0, 0.0, 1.0)
    X, Y = _centres(I, J, bounds)
    q = np.where((X >= 0.4) & (X <= 0.6) & (Y >= 0.4) & (Y <= 0.6), 2.0, 0.0)
    return Problem2D("example_2_1", I, J, bounds, np.ones((J, I)), np.full((J, I), 0.5), q,
                     kernel="iso" if g == 0.0 else "linear", g=g)


def dom_small() -> Problem2D:
    I = J = 32
    q = np.zeros((J, I))
    q[12:20, 12:20] = 1.0
    return Problem2D("dom_small_32x32", I, J, (0.0, 1.0, 0.0, 1.0), np.ones((J, I)),
                     np.full((J, I), 0.5), q, ordinates={"kind": "product_gl", "n_polar": 4,
                                                         "n_azim": 8})


def point_source(n: int = 256, n_samples: int = 64, m_quadrant: int = 4) -> Problem2D:
    bounds = (-1.0, 1.0, -1.0, 1.0)
    X, Y = _centres(n, n, bounds)
    q = np.exp(-(X * X + Y * Y) / (2.0 * 0.02 ** 2))
    return Problem2D("point_source_256", n, n, bounds, np.ones((n, n)), np.full((n, n), 0.9), q,
                     ordinates={"kind": "rom", "n_samples": n_samples,
                                "m_quadrant": [m_quadrant] * n_samples, "dom_uniform_N": 8})


def checkerboard(block: int = 64, n_blocks: int = 7, n_samples: int = 256,
                 seed: int = 3000) -> Problem2D:
    n = block * n_blocks
    bi = np.arange(n) // block
    BJ, BI = np.meshgrid(bi, bi, indexing="ij")  # BJ[j, i] = block row, BI[j, i] = block col
    c = n_blocks // 2
    absorber = ((BI + BJ) % 2 == 0) & ~((BI == c) & (BJ == c))
    sigma_t = np.where(absorber, 10.0, 1.0)
    sigma_s = np.where(absorber, 0.0, 0.9)
    q = np.where((BI == c) & (BJ == c), 1.0, 0.0)
    rng = np.random.default_rng(seed)
    M = rng.choice(np.array([8, 16, 32, 64]), size=n_samples)
    return Problem2D("checkerboard_448", n, n, (0.0, float(n_blocks), 0.0, float(n_blocks)),
                     sigma_t, sigma_s, q,
                     ordinates={"kind": "rom", "n_samples": n_samples,
                                "m_quadrant": [int(m) // 4 for m in M]})


def hg_disc(n: int = 512, n_samples: int = 32, m_quadrant: int = 32) -> Problem2D:
    bounds = (0.0, 1.0, 0.0, 1.0)
    X, Y = _centres(n, n, bounds)
    q = np.where((X - 0.5) ** 2 + (Y - 0.5) ** 2 <= 0.05 ** 2, 1.0, 0.0)
    return Problem2D("hg_disc_512", n, n, bounds, np.ones((n, n)), np.full((n, n), 0.95), q,
                     kernel="hg", g=0.8,
                     ordinates={"kind": "rom", "n_samples": n_samples,
                                "m_quadrant": [m_quadrant] * n_samples})


@dataclass
class Problem3D:
    name: str
    I: int
    J: int
    K: int
    bounds: tuple  # (x_L, x_R, y_B, y_T, z_B, z_T)
    sigma_t: np.ndarray  # [K, J, I]
    sigma_s: np.ndarray
    q: np.ndarray
    ordinates: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.I * self.J * self.K


def gaussian_random_field(n: int, corr_cells: float, seed: int) -> np.ndarray:
    """Periodic unit-variance Gaussian field on n^3 cells with covariance
    exp(-r^2 / (2 corr^2)): white noise convolved (FFT) with a Gaussian of standard
    deviation corr / sqrt(2) cells, then centred and scaled to unit variance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((n, n, n))
    d = np.minimum(np.arange(n), n - np.arange(n)).astype(np.float64)
    s2 = (corr_cells / np.sqrt(2.0)) ** 2
    g1 = np.exp(-d * d / (2.0 * s2))
    kern = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    field_ = np.fft.irfftn(np.fft.rfftn(noise) * np.fft.rfftn(kern), s=noise.shape)
    field_ -= field_.mean()
    return field_ / field_.std()


def lognormal_cube(n: int = 128, n_samples: int = 64, n_zeta: int = 2, n_theta: int = 3,
                   seed: int = 5000) -> Problem3D:
    G = gaussian_random_field(n, 8.0, seed)
    sigma_t = np.exp(-0.125 + 0.5 * G)
    q = np.zeros((n, n, n))
    c0 = n // 2 - 4
    q[c0:c0 + 8, c0:c0 + 8, c0:c0 + 8] = 1.0
    return Problem3D(f"lognormal_cube_{n}", n, n, n, (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), sigma_t,
                     0.8 * sigma_t, q,
                     ordinates={"kind": "rom3", "n_samples": n_samples,
                                "n_zeta": [n_zeta] * n_samples, "n_theta": [n_theta] * n_samples})


# ------------------------------------------------------- random test inputs

def random_medium(I: int, J: int, seed: int, ratio_max: float = 0.9,
                  sigma_t_range=(0.5, 4.0), q_max: float = 2.0):
    """Heterogeneous sigma_T, sigma_S <= ratio_max * sigma_T, q >= 0 (all [J, I])."""
    rng = np.random.default_rng(seed)
    st = rng.uniform(*sigma_t_range, size=(J, I))
    ss = st * rng.uniform(0.0, ratio_max, size=(J, I))
    q = rng.uniform(0.0, q_max, size=(J, I))
    return st, ss, q


def random_directions(M: int, seed: int, weights: str = "equal"):
    """M directions on the upper unit hemisphere, returned as (c, s, zeta, w), FP64.

    Uniform on the hemisphere (zeta ~ U(0,1), azimuth ~ U(0, 2 pi)); weights equal
    (1/M) or random positive summing to 1.  These are plain inputs for parity
    tests that feed identical ordinate arrays to both implementations."""
    rng = np.random.default_rng(seed)
    zeta = rng.uniform(0.0, 1.0, size=M)
    th = rng.uniform(0.0, 2.0 * np.pi, size=M)
    rho = np.sqrt(1.0 - zeta * zeta)
    if weights == "equal":
        w = np.full(M, 1.0 / M)
    else:
        w = rng.uniform(0.5, 1.5, size=M)
        w /= w.sum()
    return rho * np.cos(th), rho * np.sin(th), zeta, w


def random_directions_sphere(M: int, seed: int, weights: str = "equal"):
    """M directions uniform on the whole unit sphere (mu_z ~ U(-1,1), azimuth ~
    U(0, 2 pi)) as (c, s, mu_z, w), FP64; weights equal or random positive, sum 1."""
    rng = np.random.default_rng(seed)
    mz = rng.uniform(-1.0, 1.0, size=M)
    th = rng.uniform(0.0, 2.0 * np.pi, size=M)
    rho = np.sqrt(1.0 - mz * mz)
    if weights == "equal":
        w = np.full(M, 1.0 / M)
    else:
        w = rng.uniform(0.5, 1.5, size=M)
        w /= w.sum()
    return rho * np.cos(th), rho * np.sin(th), mz, w


def random_medium3(I: int, J: int, K: int, seed: int, ratio_max: float = 0.9,
                   sigma_t_range=(0.5, 4.0), q_max: float = 2.0):
    """3D heterogeneous sigma_T, sigma_S <= ratio_max * sigma_T, q >= 0 ([K, J, I])."""
    rng = np.random.default_rng(seed)
    st = rng.uniform(*sigma_t_range, size=(K, J, I))
    ss = st * rng.uniform(0.0, ratio_max, size=(K, J, I))
    q = rng.uniform(0.0, q_max, size=(K, J, I))
    return st, ss, q


def face_sizes3(I: int, J: int, K: int):
    """Cells of the six faces in the order x_L, x_R, y_B, y_T, z_B, z_T."""
    return [K * J, K * J, K * I, K * I, J * I, J * I]


def random_inflow(I: int, J: int, seed: int, per_ordinate_M: int = 0, scale: float = 1.0):
    """Non-negative face values, layout [x_L: J][x_R: J][y_B: I][y_T: I] (isotropic) or
    [M, 2J + 2I] when per_ordinate_M > 0."""
    rng = np.random.default_rng(seed)
    n = 2 * J + 2 * I
    if per_ordinate_M > 0:
        return rng.uniform(0.0, scale, size=(per_ordinate_M, n))
    return rng.uniform(0.0, scale, size=n)


def partition(m: int):
    """(n_zeta, n_theta) for m cells per quadrant: n_zeta the largest divisor of m that
    is <= sqrt(m) (N x N when m = N^2).  A workload parameter, used by both paths."""
    nz = max(d for d in range(1, int(np.sqrt(m)) + 1) if m % d == 0)
    return nz, m // nz


def ordinate_seed(config_index: int, rep: int = 0) -> int:
    """Seed convention for the ROM draws of a workload: 1000 * config + rep."""
    return 1000 * config_index + rep
