"""The C-ABI library loads and exports every entry point include/rom.h declares;
its host-only calls (quadratures, version, defaults) work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rom.h")


def _lib():
    from paper_2407_12527_gb300 import build, rom
    build.build()
    return rom.lib()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rom_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported():
    L = _lib()
    names = header_functions()
    assert len(names) >= 20
    from paper_2407_12527_gb300 import rom
    for n in names:
        assert hasattr(L, n), f"{n} declared in rom.h but not exported"
        assert n in rom.SIGNATURES, f"{n} has no binding signature"


def test_version_and_defaults():
    L = _lib()
    assert b"sm_103a" in L.rom_version()
    from paper_2407_12527_gb300 import default_options
    o = default_options()
    assert o.scheme == 0 and o.max_iter == 10000 and o.tol == 1e-6 and o.fixed_iters == 0


@pytest.mark.parametrize("kind,n1,n2,maker", [
    ("uniform", 1, 0, lambda: O.quad_uniform_xy(1)),
    ("uniform", 7, 0, lambda: O.quad_uniform_xy(7)),
    ("gauss", 1, 0, lambda: O.quad_gauss_xy(1)),
    ("gauss", 9, 0, lambda: O.quad_gauss_xy(9)),
    ("gauss", 40, 0, lambda: O.quad_gauss_xy(40)),
    ("product_gl", 4, 8, lambda: O.quad_product_gl_xy(4, 8)),
])
def test_library_quadrature_matches_oracle(kind, n1, n2, maker):
    from paper_2407_12527_gb300 import quadrature_xy
    dirs, w = quadrature_xy(kind, n1, n2)
    o = maker()
    np.testing.assert_allclose(dirs[:, 0], o.c, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dirs[:, 1], o.s, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dirs[:, 2], o.zeta, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(w, o.w, rtol=1e-11)


def test_quadrature_rejects_bad_arguments():
    L = _lib()
    m = ctypes.c_int32(0)
    assert L.rom_quadrature_xy(9, 3, 0, None, None, ctypes.byref(m)) < 0
    assert L.rom_quadrature_xy(0, 0, 0, None, None, ctypes.byref(m)) < 0
    assert L.rom_quadrature_xy(2, 3, 0, None, None, ctypes.byref(m)) < 0


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2407_12527_gb300 import RomContext, RomError
    with pytest.raises(RomError):
        RomContext(0)
