"""Python binding of the C ABI in include/rom.h (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library ``librom_gb300.so`` built by
``paper_2407_12527_gb300.build``.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls fail with an error.

Low level: :func:`lib` returns the ``ctypes.CDLL`` with typed signatures for
every ``rom_*`` entry point of include/rom.h (same names).  High level:
:class:`RomContext` wraps one ``rom_ctx`` with NumPy / torch marshalling.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "librom_gb300.so"

ROM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NOT_CONVERGED", -5: "DIVERGED",
          -6: "STATE", -7: "UNSUPPORTED", -8: "TIMEOUT"}
SCHEME = {"dd": 0, "step": 1}
KERNEL = {"iso": 0, "linear": 1, "hg": 2}
KERNEL_FLAG_NORMALIZE = 1
KERNEL_FLAG_RAW = 2
QUAD = {"uniform": 0, "gauss": 1, "product_gl": 2}
FACES = {"xl": 0, "xr": 1, "yb": 2, "yt": 3, "zb": 4, "zt": 5}


class rom_options(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("fixed_iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("tile_g", ctypes.c_int), ("time_kernels", ctypes.c_int),
                ("dense_source", ctypes.c_int), ("dense_precision", ctypes.c_int),
                ("rows_per_step", ctypes.c_int),
                ("diverge_window", ctypes.c_int), ("wait_timeout_ms", ctypes.c_double),
                ("test_stall_waits", ctypes.c_int)]


class rom_stats(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_int), ("iterations_max", ctypes.c_int),
                ("iterations_min", ctypes.c_int), ("n_not_converged", ctypes.c_int),
                ("updates", ctypes.c_int64), ("residual_max", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_int64),
                ("source_ms", ctypes.c_double), ("source_launches", ctypes.c_int64),
                ("tile_g", ctypes.c_int), ("rows_per_step", ctypes.c_int),
                ("balance_max", ctypes.c_double),
                ("phi_min", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RomError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rom error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i = ctypes.c_int

SIGNATURES = {
    "rom_version": (ctypes.c_char_p, []),
    "rom_default_options": (None, [ctypes.POINTER(rom_options)]),
    "rom_create": (_i, [ctypes.POINTER(_vp), _i]),
    "rom_destroy": (None, [_vp]),
    "rom_last_error": (ctypes.c_char_p, [_vp]),
    "rom_set_stream": (_i, [_vp, _vp]),
    "rom_set_options": (_i, [_vp, ctypes.POINTER(rom_options)]),
    "rom_set_grid": (_i, [_vp, _i, _i64p, _dp, _dp, _dp, _dp, _dp]),
    "rom_set_grid_device": (_i, [_vp, _i, _i64p, _dp, _dp, _vp, _vp, _vp]),
    "rom_set_grids_xy": (_i, [_vp, _i, _i64p, _dp, _dp, _dp, _dp, _dp, _i32p]),
    "rom_set_inflow_isotropic": (_i, [_vp, _i, _dp]),
    "rom_set_inflow_ordinates": (_i, [_vp, _i, _dp]),
    "rom_set_ordinates": (_i, [_vp, _i, _i32p, _dp, _dp]),
    "rom_set_ordinates_seed": (_i, [_vp, ctypes.c_uint64, _i, _i32p, _i32p]),
    "rom_set_ordinates_seed_offset": (_i, [_vp, ctypes.c_uint64, _i, _i, _i32p, _i32p]),
    "rom_set_ordinates_seed_xyz": (_i, [_vp, ctypes.c_uint64, _i, _i, _i32p, _i32p]),
    "rom_set_quadrature": (_i, [_vp, _i, _i, _i]),
    "rom_quadrature_xy": (_i, [_i, _i, _i, _dp, _dp, _i32p]),
    "rom_get_ordinates": (_i, [_vp, _dp, _dp]),
    "rom_set_kernel": (_i, [_vp, _i, ctypes.c_double, _i]),
    "rom_solve": (_i, [_vp, ctypes.POINTER(rom_stats)]),
    "rom_get_scalar_flux": (_i, [_vp, _i, _dp]),
    "rom_get_scalar_flux_device": (_i, [_vp, _i, _vp]),
    "rom_get_iterations": (_i, [_vp, _i32p, _dp]),
    "rom_get_partial_sum": (_i, [_vp, _dp, _i64p]),
    "rom_get_balance": (_i, [_vp, _dp, _dp, _dp]),
    "rom_get_grid_average": (_i, [_vp, _i, _dp]),
    "rom_sweep_xy_noalloc": (_i, [_vp, _i, _i, ctypes.c_double, ctypes.c_double, _i, _vp, _i,
                                  _i32p, _dp, _dp, _vp, _vp, ctypes.c_char_p, ctypes.c_size_t]),
}


def lib() -> ctypes.CDLL:
    """Load librom_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(
                f"{LIB_PATH.name} is not built; run `python -c 'import __graft_entry__ as g; "
                f"g.build()'` (needs nvcc)")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def quadrature_xy(kind: str, n1: int, n2: int = 0):
    """Deterministic X-Y set from the library (host code): returns (dirs [M,3], weights [M])."""
    L = lib()
    m = ctypes.c_int32(0)
    rc = L.rom_quadrature_xy(QUAD[kind], n1, n2, None, None, ctypes.byref(m))
    if rc != ROM_OK:
        raise RomError(rc, "rom_quadrature_xy")
    dirs = np.zeros((m.value, 3))
    w = np.zeros(m.value)
    rc = L.rom_quadrature_xy(QUAD[kind], n1, n2, _ptr(dirs), _ptr(w), None)
    if rc != ROM_OK:
        raise RomError(rc, "rom_quadrature_xy")
    return dirs, w


def default_options() -> rom_options:
    o = rom_options()
    lib().rom_default_options(ctypes.byref(o))
    return o


class RomContext:
    """One rom_ctx on a CUDA device (thin wrapper; every call is one C-ABI call)."""

    def __init__(self, device: int = 0):
        self.L = lib()
        self.h = _vp()
        rc = self.L.rom_create(ctypes.byref(self.h), device)
        if rc != ROM_OK:
            raise RomError(rc, f"rom_create(device={device}) failed (no usable CUDA device?)")
        self.I = self.J = 0
        self.K = 1
        self.dim = 2
        self.n_samples = 0
        self.grid_shapes = None  # [(J_p, I_p)] of a batch of several grids

    def close(self):
        if self.h:
            self.L.rom_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != ROM_OK:
            msg = self.L.rom_last_error(self.h)
            raise RomError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    # ------------------------------------------------------------ setters
    def set_stream(self, stream_handle: int | None):
        self._check(self.L.rom_set_stream(self.h, _vp(stream_handle or 0) if stream_handle else None),
                    "rom_set_stream")

    def set_options(self, **kw):
        o = default_options()
        for k, v in kw.items():
            if k == "scheme" and isinstance(v, str):
                v = SCHEME[v]
            setattr(o, k, v)
        self._check(self.L.rom_set_options(self.h, ctypes.byref(o)), "rom_set_options")
        return o

    def set_grid(self, I, J, bounds, sigma_t, sigma_s, q):
        n = np.array([I, J, 1], dtype=np.int64)
        lo = np.array([bounds[0], bounds[2], 0.0])
        hi = np.array([bounds[1], bounds[3], 1.0])
        st, ss, qq = (_f64(np.broadcast_to(a, (J, I))) for a in (sigma_t, sigma_s, q))
        self._check(self.L.rom_set_grid(self.h, 2, _ptr(n, _i64p), _ptr(lo), _ptr(hi), _ptr(st),
                                        _ptr(ss), _ptr(qq)), "rom_set_grid")
        self.I, self.J, self.K, self.dim = I, J, 1, 2
        self.grid_shapes = None

    def set_grids(self, grids, samples_per_grid):
        """Several X-Y grids in one batch: grids = [(I, J, bounds, sigma_t, sigma_s, q), ...],
        grid p holding samples_per_grid[p] consecutive samples."""
        n = np.array([[g[0], g[1]] for g in grids], dtype=np.int64).reshape(-1)
        lo = _f64(np.array([[g[2][0], g[2][2]] for g in grids]).reshape(-1))
        hi = _f64(np.array([[g[2][1], g[2][3]] for g in grids]).reshape(-1))
        st, ss, qq = (_f64(np.concatenate([np.broadcast_to(g[k], (g[1], g[0])).reshape(-1)
                                           for g in grids])) for k in (3, 4, 5))
        spg = np.ascontiguousarray(np.asarray(samples_per_grid, dtype=np.int32))
        self._check(self.L.rom_set_grids_xy(self.h, len(grids), _ptr(n, _i64p), _ptr(lo), _ptr(hi),
                                            _ptr(st), _ptr(ss), _ptr(qq), _ptr(spg, _i32p)),
                    "rom_set_grids_xy")
        self.grid_shapes = [(int(g[1]), int(g[0])) for g in grids]
        self.sample_grid = np.repeat(np.arange(len(grids)), spg)
        self.I = max(g[0] for g in grids)
        self.J = max(g[1] for g in grids)
        self.K, self.dim = 1, 2

    def grid_average(self, grid) -> np.ndarray:
        """FP64 sample average of the samples on grid `grid`, [J_p, I_p]."""
        if self.grid_shapes:
            ok = 0 <= grid < len(self.grid_shapes)
            shape = self.grid_shapes[grid] if ok else (1,)  # the library rejects a bad index
        else:
            shape = self._shape()
        out = np.zeros(shape)
        self._check(self.L.rom_get_grid_average(self.h, grid, _ptr(out)), "rom_get_grid_average")
        return out

    def set_grid3(self, I, J, K, bounds, sigma_t, sigma_s, q):
        """3D grid: bounds = (x_L, x_R, y_B, y_T, z_B, z_T); arrays [K, J, I]."""
        n = np.array([I, J, K], dtype=np.int64)
        lo = np.array([bounds[0], bounds[2], bounds[4]], dtype=np.float64)
        hi = np.array([bounds[1], bounds[3], bounds[5]], dtype=np.float64)
        st, ss, qq = (_f64(np.broadcast_to(a, (K, J, I))) for a in (sigma_t, sigma_s, q))
        self._check(self.L.rom_set_grid(self.h, 3, _ptr(n, _i64p), _ptr(lo), _ptr(hi), _ptr(st),
                                        _ptr(ss), _ptr(qq)), "rom_set_grid")
        self.I, self.J, self.K, self.dim = I, J, K, 3
        self.grid_shapes = None

    def set_grid3_device(self, I, J, K, bounds, sigma_t, sigma_s, q):
        """sigma_t, sigma_s, q: contiguous float32 CUDA tensors [K, J, I] (torch)."""
        for t in (sigma_t, sigma_s, q):
            assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4
            assert t.is_contiguous() and tuple(t.shape) == (K, J, I)
        n = np.array([I, J, K], dtype=np.int64)
        lo = np.array([bounds[0], bounds[2], bounds[4]], dtype=np.float64)
        hi = np.array([bounds[1], bounds[3], bounds[5]], dtype=np.float64)
        self._check(self.L.rom_set_grid_device(self.h, 3, _ptr(n, _i64p), _ptr(lo), _ptr(hi),
                                               _vp(sigma_t.data_ptr()), _vp(sigma_s.data_ptr()),
                                               _vp(q.data_ptr())), "rom_set_grid_device")
        self.I, self.J, self.K, self.dim = I, J, K, 3
        self.grid_shapes = None

    def set_grid_device(self, I, J, bounds, sigma_t, sigma_s, q):
        """sigma_t, sigma_s, q: contiguous float32 CUDA tensors [J, I] (torch)."""
        for t in (sigma_t, sigma_s, q):
            assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 4
            assert t.is_contiguous() and tuple(t.shape) == (J, I)
        n = np.array([I, J, 1], dtype=np.int64)
        lo = np.array([bounds[0], bounds[2], 0.0])
        hi = np.array([bounds[1], bounds[3], 1.0])
        self._check(self.L.rom_set_grid_device(self.h, 2, _ptr(n, _i64p), _ptr(lo), _ptr(hi),
                                               _vp(sigma_t.data_ptr()), _vp(sigma_s.data_ptr()),
                                               _vp(q.data_ptr())), "rom_set_grid_device")
        self.I, self.J, self.K, self.dim = I, J, 1, 2
        self.grid_shapes = None

    def set_inflow_isotropic(self, face, values):
        f = FACES[face] if isinstance(face, str) else face
        v = None if values is None else _f64(values)
        self._check(self.L.rom_set_inflow_isotropic(self.h, f, _ptr(v) if v is not None else None),
                    "rom_set_inflow_isotropic")

    def set_inflow_ordinates(self, face, values):
        f = FACES[face] if isinstance(face, str) else face
        v = None if values is None else _f64(values)
        self._check(self.L.rom_set_inflow_ordinates(self.h, f, _ptr(v) if v is not None else None),
                    "rom_set_inflow_ordinates")

    def set_ordinates(self, sets):
        """sets: list of (c, s, zeta, w) FP64 arrays, one per sample."""
        m = np.array([len(s[0]) for s in sets], dtype=np.int32)
        dirs = _f64(np.concatenate([np.stack([s[0], s[1], s[2]], axis=1) for s in sets]))
        w = _f64(np.concatenate([s[3] for s in sets]))
        self._check(self.L.rom_set_ordinates(self.h, len(sets), _ptr(m, _i32p), _ptr(dirs),
                                             _ptr(w)), "rom_set_ordinates")
        self.n_samples = len(sets)

    def set_ordinates_seed(self, seed, n_zeta, n_theta, first_sample=0):
        nz = np.ascontiguousarray(np.asarray(n_zeta, dtype=np.int32))
        nt = np.ascontiguousarray(np.asarray(n_theta, dtype=np.int32))
        self._check(self.L.rom_set_ordinates_seed_offset(self.h, seed, first_sample, nz.size,
                                                         _ptr(nz, _i32p), _ptr(nt, _i32p)),
                    "rom_set_ordinates_seed_offset")
        self.n_samples = int(nz.size)

    def set_ordinates_seed_xyz(self, seed, n_zeta, n_theta, first_sample=0):
        """3D sets: 8 n_zeta n_theta ordinates per sample (octants)."""
        nz = np.ascontiguousarray(np.asarray(n_zeta, dtype=np.int32))
        nt = np.ascontiguousarray(np.asarray(n_theta, dtype=np.int32))
        self._check(self.L.rom_set_ordinates_seed_xyz(self.h, seed, first_sample, nz.size,
                                                      _ptr(nz, _i32p), _ptr(nt, _i32p)),
                    "rom_set_ordinates_seed_xyz")
        self.n_samples = int(nz.size)

    def set_quadrature(self, kind, n1, n2=0):
        self._check(self.L.rom_set_quadrature(self.h, QUAD[kind], n1, n2), "rom_set_quadrature")
        self.n_samples = 1

    def get_ordinates(self, m_total):
        dirs = np.zeros((m_total, 3))
        w = np.zeros(m_total)
        self._check(self.L.rom_get_ordinates(self.h, _ptr(dirs), _ptr(w)), "rom_get_ordinates")
        return dirs, w

    def set_kernel(self, kind="iso", g=0.0, flags=0):
        self._check(self.L.rom_set_kernel(self.h, KERNEL[kind], float(g), int(flags)),
                    "rom_set_kernel")

    # -------------------------------------------------------------- solve
    def solve(self, allow_not_converged=False) -> dict:
        st = rom_stats()
        rc = self.L.rom_solve(self.h, ctypes.byref(st))
        if rc != ROM_OK and not (allow_not_converged and rc in (-4, -5)):
            self._check(rc, "rom_solve")
        d = st.as_dict()
        d["status"] = rc
        return d

    def _shape(self):
        return (self.K, self.J, self.I) if self.dim == 3 else (self.J, self.I)

    def scalar_flux(self, sample=-1) -> np.ndarray:
        out = np.zeros(self.grid_shapes[self.sample_grid[sample]]
                       if self.grid_shapes and sample >= 0 else self._shape())
        self._check(self.L.rom_get_scalar_flux(self.h, sample, _ptr(out)), "rom_get_scalar_flux")
        return out

    def scalar_flux_device(self, out_tensor, sample=-1):
        """Write phi into a float64 CUDA tensor [J, I] ([K, J, I]) on the context stream."""
        assert out_tensor.is_cuda and out_tensor.element_size() == 8 and out_tensor.is_contiguous()
        self._check(self.L.rom_get_scalar_flux_device(self.h, sample, _vp(out_tensor.data_ptr())),
                    "rom_get_scalar_flux_device")

    def iterations(self):
        it = np.zeros(self.n_samples, dtype=np.int32)
        r = np.zeros(self.n_samples)
        self._check(self.L.rom_get_iterations(self.h, _ptr(it, _i32p), _ptr(r)),
                    "rom_get_iterations")
        return it, r

    def balance(self):
        """(net leakage, relative balance error, min phi) of each sample's last sweep."""
        lk = np.zeros(self.n_samples)
        bal = np.zeros(self.n_samples)
        mn = np.zeros(self.n_samples)
        self._check(self.L.rom_get_balance(self.h, _ptr(lk), _ptr(bal), _ptr(mn)),
                    "rom_get_balance")
        return lk, bal, mn

    def partial_sum(self):
        s = np.zeros(self._shape())
        n = ctypes.c_int64(0)
        self._check(self.L.rom_get_partial_sum(self.h, _ptr(s), ctypes.byref(n)),
                    "rom_get_partial_sum")
        return s, int(n.value)
