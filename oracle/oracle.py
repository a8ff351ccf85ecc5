"""FP64 CPU oracle for the Random Ordinate Method (arXiv 2407.12527), X-Y and 3D geometry.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``, never by the CUDA library or its binding.
It shares no code with them.

This module holds
  * a ctypes wrapper around ``rom_oracle.c`` (sweeps, source iteration, ROM
    ordinates, kernel matrix; X-Y and 3D octant sets and sweeps; the linear
    kernel's three-moment form), built with gcc by :func:`build`;
  * the deterministic X-Y quadratures of Appendix A (2D uniform, eq. uniform2D;
    2D Gaussian of Lewis & Miller) and a product Gauss-Legendre set, written
    with NumPy (``numpy.polynomial.legendre`` supplies the Legendre roots);
  * the error measures of the paper: the l2 norm of eq. (l2norm2D), e_inf of
    Sec. 4.2.3, the expected single-run error of eq. (norm-error), the bias of
    eq. (norm-bias) and the Monte Carlo error of eq. (1dMCerror), and the
    sample average of Sec. 4.1.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np
from numpy.polynomial import legendre as npleg

HERE = Path(__file__).resolve().parent
SRC = HERE / "rom_oracle.c"
LIB = HERE / "librom_oracle.so"

KERNELS = {"iso": 0, "linear": 1, "hg": 2}
SCHEMES = {"dd": 0, "step": 1}

_lib = None


def build(force: bool = False) -> Path:
    """Compile rom_oracle.c into a shared library next to it (gcc, OpenMP)."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-o", str(tmp), str(SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_splitmix64.restype = ctypes.c_uint64
        L.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_uniform01.restype = ctypes.c_double
        L.oracle_uniform01.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_rom_ordinates_xy.restype = ctypes.c_int
        L.oracle_rom_ordinates_xy.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, dp, dp, dp, dp]
        L.oracle_rom_ordinates_from_u.restype = ctypes.c_int
        L.oracle_rom_ordinates_from_u.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp]
        L.oracle_rom_draws.restype = ctypes.c_int
        L.oracle_rom_draws.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_kernel_matrix.restype = ctypes.c_int
        L.oracle_kernel_matrix.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        L.oracle_solve_xy.restype = ctypes.c_int
        L.oracle_solve_xy.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, dp, dp, dp, ctypes.c_int, ip, dp, dp, dp, dp, dp, ctypes.c_long,
            ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp]
        L.oracle_rom_ordinates_xyz.restype = ctypes.c_int
        L.oracle_rom_ordinates_xyz.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, dp, dp, dp, dp]
        L.oracle_solve_xyz.restype = ctypes.c_int
        L.oracle_solve_xyz.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ip, dp, dp,
            dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            dp, ip, dp, dp]
        L.oracle_solve_xy_linear_moments.restype = ctypes.c_int
        L.oracle_solve_xy_linear_moments.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, dp, dp, dp, ctypes.c_int, ip, dp, dp, dp, ctypes.c_double,
            ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip, dp]
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------- RNG

def splitmix64(seed: int, n: int) -> int:
    """n-th output of SplitMix64 seeded with ``seed`` (C implementation)."""
    return int(lib().oracle_splitmix64(seed, n))


def uniform01(seed: int, n: int) -> float:
    return float(lib().oracle_uniform01(seed, n))


# ------------------------------------------------------------- ordinates

class Ordinates:
    """An ordinate set in X-Y geometry: directions (c, s), polar cosine zeta, weights w."""

    def __init__(self, c, s, zeta, w):
        self.c, self.s, self.zeta, self.w = (_f64(v) for v in (c, s, zeta, w))

    @property
    def M(self) -> int:
        return int(self.c.size)


def _reflect(zeta, theta, w):
    """Quadrants 2-4 from quadrant 1 by the reflections of eq. (2Dordinates_symmetry):
    theta -> pi - theta, theta - pi, 2 pi - theta, same zeta and weight."""
    th = np.concatenate([theta, np.pi - theta, theta - np.pi, 2.0 * np.pi - theta])
    zz = np.tile(zeta, 4)
    ww = np.tile(w, 4)
    rho = np.sqrt(1.0 - zz * zz)
    return Ordinates(rho * np.cos(th), rho * np.sin(th), zz, ww)


def quad_uniform_xy(N: int) -> Ordinates:
    """2D uniform quadrature, Appendix A eq. (uniform2D): per quadrant N^2 nodes
    zeta_i = (2N-2i+1)/(2N), theta_j = (2j-1) pi/(4N), weight 1/(4N^2), l = (i-1)N + j."""
    i = np.repeat(np.arange(1, N + 1), N)
    j = np.tile(np.arange(1, N + 1), N)
    zeta = (2 * N - 2 * i + 1) / (2.0 * N)
    theta = (2 * j - 1) * np.pi / (4.0 * N)
    return _reflect(zeta, theta, np.full(N * N, 1.0 / (4 * N * N)))


def legendre_positive_roots(n2: int):
    """Positive roots (descending) of the Legendre polynomial L_{n2} and L'_{n2} there."""
    x, _ = npleg.leggauss(n2)
    pos = np.sort(x[x > 0])[::-1]
    coef = np.zeros(n2 + 1)
    coef[n2] = 1.0
    dL = npleg.legval(pos, npleg.legder(coef))
    return pos, dL


def quad_gauss_xy(N: int) -> Ordinates:
    """2D Gaussian quadrature of Appendix A: zeta_i the N positive roots of L_{2N}
    (1 > zeta_1 > ... > zeta_N > 0), theta_{i,j} = (2j-1) pi / (4i), j = 1..i, weight
    1 / (2 i (1 - zeta_i^2) L'_{2N}(zeta_i)^2), l = i(i-1)/2 + j; M = N(N+1)/2 per quadrant."""
    zr, dL = legendre_positive_roots(2 * N)
    zeta, theta, w = [], [], []
    for i in range(1, N + 1):
        wi = 1.0 / (2.0 * i * (1.0 - zr[i - 1] ** 2) * dL[i - 1] ** 2)
        for j in range(1, i + 1):
            zeta.append(zr[i - 1])
            theta.append((2 * j - 1) * np.pi / (4.0 * i))
            w.append(wi)
    return _reflect(np.array(zeta), np.array(theta), np.array(w))


def quad_product_gl_xy(n_polar: int, n_azim: int) -> Ordinates:
    """Product set: zeta = the n_polar positive roots of L_{2 n_polar} with their
    Gauss-Legendre weights (which sum to 1 on (0,1)), times n_azim azimuths
    theta_j = (2j-1) pi / n_azim, j = 1..n_azim, each with weight 1/n_azim."""
    x, wx = npleg.leggauss(2 * n_polar)
    keep = x > 0
    zr, wr = x[keep], wx[keep]
    order = np.argsort(-zr)
    zr, wr = zr[order], wr[order]
    theta = (2 * np.arange(1, n_azim + 1) - 1) * np.pi / n_azim
    zz = np.repeat(zr, n_azim)
    ww = np.repeat(wr, n_azim) / n_azim
    th = np.tile(theta, n_polar)
    rho = np.sqrt(1.0 - zz * zz)
    return Ordinates(rho * np.cos(th), rho * np.sin(th), zz, ww)


def rom_ordinates_xy(seed: int, sample: int, n_zeta: int, n_theta: int) -> Ordinates:
    """One ROM ordinate set (Sec. 4.2 partition, eq. 2Dordinates_symmetry), C implementation."""
    m = n_zeta * n_theta
    arr = [np.zeros(4 * m) for _ in range(4)]
    rc = lib().oracle_rom_ordinates_xy(seed, sample, n_zeta, n_theta, *(_dp(a) for a in arr))
    if rc != 0:
        raise ValueError(f"oracle_rom_ordinates_xy failed ({rc})")
    return Ordinates(*arr)


def rom_ordinates_from_u(n_zeta: int, n_theta: int, u_zeta, u_theta) -> Ordinates:
    """ROM ordinates from given uniform numbers in [0,1) (one per quadrant-1 cell)."""
    m = n_zeta * n_theta
    uz, ut = _f64(u_zeta), _f64(u_theta)
    assert uz.size == m and ut.size == m
    arr = [np.zeros(4 * m) for _ in range(4)]
    rc = lib().oracle_rom_ordinates_from_u(n_zeta, n_theta, _dp(uz), _dp(ut),
                                           *(_dp(a) for a in arr))
    if rc != 0:
        raise ValueError(f"oracle_rom_ordinates_from_u failed ({rc})")
    return Ordinates(*arr)


def rom_draws(seed: int, sample: int, m: int):
    """(u_zeta, u_theta): the SplitMix64 uniform numbers of one ROM sample."""
    uz, ut = np.zeros(m), np.zeros(m)
    rc = lib().oracle_rom_draws(seed, sample, m, _dp(uz), _dp(ut))
    if rc != 0:
        raise ValueError(f"oracle_rom_draws failed ({rc})")
    return uz, ut


def rom_partition(m: int):
    """(n_zeta, n_theta) for m cells per quadrant: n_zeta the largest divisor of m
    that is <= sqrt(m) (N x N when m = N^2, as in Sec. 4.2)."""
    nz = max(d for d in range(1, int(np.sqrt(m)) + 1) if m % d == 0)
    return nz, m // nz


def kernel_matrix(o: Ordinates, kernel: str, g: float = 0.0, raw: bool = False,
                  normalize_rows: bool = False) -> np.ndarray:
    """A[l, l'] = w_l' P(u_l', u_l) (eq. wl), optionally row-normalised."""
    A = np.zeros((o.M, o.M))
    rc = lib().oracle_kernel_matrix(o.M, _dp(o.c), _dp(o.s), _dp(o.zeta), _dp(o.w),
                                    KERNELS[kernel], g, int(raw), int(normalize_rows), _dp(A))
    if rc != 0:
        raise ValueError(f"oracle_kernel_matrix failed ({rc})")
    return A


# ----------------------------------------------------------------- solve

def solve_xy(I, J, bounds, sigma_t, sigma_s, q, ordinate_sets, *, kernel="iso", g=0.0,
             raw=False, normalize_rows=False, scheme="dd", tol=1e-10, max_iter=10000,
             fixed_iters=0, inflow=None, inflow_per_ordinate=False, n_threads=0,
             allow_not_converged=False):
    """Source iteration for each ordinate set in ``ordinate_sets`` (list of Ordinates).

    ``bounds`` = (x_L, x_R, y_B, y_T); sigma_t, sigma_s, q are [J, I] arrays (x fastest).
    ``inflow``: None (vacuum), or face values [2J + 2I] (isotropic), or, with
    ``inflow_per_ordinate``, [sum M, 2J + 2I] (face order x_L, x_R, y_B, y_T).
    Returns dict(phi [n_samples, J, I], iters, resid, leak).
    """
    xl, xr, yb, yt = (float(b) for b in bounds)
    st, ss, qq = (_f64(np.broadcast_to(a, (J, I))) for a in (sigma_t, sigma_s, q))
    ns = len(ordinate_sets)
    mps = np.array([o.M for o in ordinate_sets], dtype=np.int32)
    c = _f64(np.concatenate([o.c for o in ordinate_sets])) if ns else np.zeros(1)
    s = _f64(np.concatenate([o.s for o in ordinate_sets])) if ns else np.zeros(1)
    z = _f64(np.concatenate([o.zeta for o in ordinate_sets])) if ns else np.zeros(1)
    w = _f64(np.concatenate([o.w for o in ordinate_sets])) if ns else np.zeros(1)
    nface = 2 * J + 2 * I
    if inflow is None:
        infl, stride = None, 0
    else:
        infl = _f64(inflow)
        if inflow_per_ordinate:
            assert infl.shape == (int(mps.sum()), nface)
            stride = nface
        else:
            assert infl.size == nface
            stride = 0
    phi = np.zeros((ns, J, I))
    iters = np.zeros(ns, dtype=np.int32)
    resid = np.zeros(ns)
    leak = np.zeros(ns)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().oracle_solve_xy(
        I, J, xl, xr, yb, yt, _dp(st), _dp(ss), _dp(qq), ns, mps.ctypes.data_as(ip),
        _dp(c), _dp(s), _dp(z), _dp(w), _dp(infl) if infl is not None else None, stride,
        KERNELS[kernel], float(g), int(raw), int(normalize_rows), SCHEMES[scheme], float(tol),
        int(max_iter), int(fixed_iters), int(n_threads), _dp(phi), iters.ctypes.data_as(ip),
        _dp(resid), _dp(leak))
    if rc == -4 and not allow_not_converged:
        raise RuntimeError("oracle: source iteration did not converge")
    if rc not in (0, -4):
        raise ValueError(f"oracle_solve_xy failed ({rc})")
    return {"phi": phi, "iters": iters, "resid": resid, "leak": leak}


def rom_ordinates_xyz(seed: int, sample: int, n_zeta: int, n_theta: int) -> Ordinates:
    """3D ROM set: the X-Y set of the same draws and its mirror in zeta (8 m ordinates,
    weights 1/(8m)); ``zeta`` holds the z direction cosine mu_z in (-1, 1)."""
    m = n_zeta * n_theta
    arr = [np.zeros(8 * m) for _ in range(4)]
    rc = lib().oracle_rom_ordinates_xyz(seed, sample, n_zeta, n_theta, *(_dp(a) for a in arr))
    if rc != 0:
        raise ValueError(f"oracle_rom_ordinates_xyz failed ({rc})")
    return Ordinates(*arr)


def solve_xyz(I, J, K, bounds, sigma_t, sigma_s, q, ordinate_sets, *, scheme="dd", tol=1e-10,
              max_iter=10000, fixed_iters=0, inflow=None, n_threads=0,
              allow_not_converged=False):
    """3D source iteration, isotropic scattering.  bounds = (x_L, x_R, y_B, y_T, z_B, z_T);
    sigma_t, sigma_s, q are [K, J, I]; ordinate sets carry mu_z in ``zeta``; inflow is
    None or isotropic face values [x_L: K*J][x_R: K*J][y_B: K*I][y_T: K*I][z_B: J*I][z_T: J*I].
    Returns dict(phi [n_samples, K, J, I], iters, resid, leak)."""
    b = _f64(bounds)
    st, ss, qq = (_f64(np.broadcast_to(a, (K, J, I))) for a in (sigma_t, sigma_s, q))
    ns = len(ordinate_sets)
    mps = np.array([o.M for o in ordinate_sets], dtype=np.int32)
    cat = [_f64(np.concatenate([getattr(o, f) for o in ordinate_sets])) if ns else np.zeros(1)
           for f in ("c", "s", "zeta", "w")]
    infl = None if inflow is None else _f64(inflow)
    if infl is not None:
        assert infl.size == 2 * K * J + 2 * K * I + 2 * J * I
    phi = np.zeros((ns, K, J, I))
    iters = np.zeros(ns, dtype=np.int32)
    resid = np.zeros(ns)
    leak = np.zeros(ns)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().oracle_solve_xyz(
        I, J, K, _dp(b), _dp(st), _dp(ss), _dp(qq), ns, mps.ctypes.data_as(ip),
        *(_dp(a) for a in cat), _dp(infl) if infl is not None else None, SCHEMES[scheme],
        float(tol), int(max_iter), int(fixed_iters), int(n_threads), _dp(phi),
        iters.ctypes.data_as(ip), _dp(resid), _dp(leak))
    if rc == -4 and not allow_not_converged:
        raise RuntimeError("oracle: source iteration did not converge")
    if rc not in (0, -4):
        raise ValueError(f"oracle_solve_xyz failed ({rc})")
    return {"phi": phi, "iters": iters, "resid": resid, "leak": leak}


def solve_xy_linear_moments(I, J, bounds, sigma_t, sigma_s, q, ordinate_sets, g, *,
                            scheme="dd", tol=1e-10, max_iter=10000, fixed_iters=0, n_threads=0,
                            allow_not_converged=False):
    """Linear kernel P = 1 + g cos(xi) (mirror-averaged, unnormalised) by its three
    angular moments phi, Jx, Jy (eq. anisotropic kernel), vacuum inflow; for ordinate
    sets too large for the dense operator of solve_xy.  Returns dict(phi, iters, resid)."""
    st, ss, qq = (_f64(np.broadcast_to(a, (J, I))) for a in (sigma_t, sigma_s, q))
    ns = len(ordinate_sets)
    mps = np.array([o.M for o in ordinate_sets], dtype=np.int32)
    cat = [_f64(np.concatenate([getattr(o, f) for o in ordinate_sets])) if ns else np.zeros(1)
           for f in ("c", "s", "w")]
    phi = np.zeros((ns, J, I))
    iters = np.zeros(ns, dtype=np.int32)
    resid = np.zeros(ns)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().oracle_solve_xy_linear_moments(
        I, J, float(bounds[0]), float(bounds[1]), float(bounds[2]), float(bounds[3]), _dp(st),
        _dp(ss), _dp(qq), ns, mps.ctypes.data_as(ip), *(_dp(a) for a in cat), float(g),
        SCHEMES[scheme], float(tol), int(max_iter), int(fixed_iters), int(n_threads), _dp(phi),
        iters.ctypes.data_as(ip), _dp(resid))
    if rc == -4 and not allow_not_converged:
        raise RuntimeError("oracle: source iteration did not converge")
    if rc not in (0, -4):
        raise ValueError(f"oracle_solve_xy_linear_moments failed ({rc})")
    return {"phi": phi, "iters": iters, "resid": resid}


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# --------------------------------------------------------------- metrics

def l2_xy(phi, phi_ref) -> float:
    """eq. (l2norm2D): sqrt( (1/IJ) sum_ij |phi - phi_ref|^2 )."""
    d = np.asarray(phi, dtype=np.float64) - np.asarray(phi_ref, dtype=np.float64)
    return float(np.sqrt(np.mean(d * d)))


def e_inf(phi, phi_ref) -> float:
    """Ray-effect measure of Sec. 4.2.3: max_ij |phi - phi_ref|."""
    return float(np.max(np.abs(np.asarray(phi, np.float64) - np.asarray(phi_ref, np.float64))))


def rom_average(phi_samples) -> np.ndarray:
    """Sample mean (1/t) sum_s phi^{xi_s} (Sec. 4.1), in FP64."""
    p = np.asarray(phi_samples, dtype=np.float64)
    return p.sum(axis=0) / p.shape[0]


def rom_error(phi_samples, phi_ref) -> float:
    """Expected single-run error E ||phi^xi - phi_ref|| (eq. norm-error), sample estimate."""
    return float(np.mean([l2_xy(p, phi_ref) for p in phi_samples]))


def rom_bias(phi_samples, phi_ref) -> float:
    """Bias || E phi^xi - phi_ref || (eq. norm-bias), sample estimate."""
    return l2_xy(rom_average(phi_samples), phi_ref)


def mc_error(phi_samples, expectation, t: int) -> float:
    """Monte Carlo error of the first t samples, eq. (1dMCerror)."""
    return l2_xy(rom_average(np.asarray(phi_samples)[:t]), expectation)
