"""GB300-native hot path of the Random Ordinate Method (Li, Tang & Yang, arXiv 2407.12527).

The method's steps run in the CUDA library ``librom_gb300.so`` (sources in
``csrc/``, C ABI in ``include/rom.h``); :mod:`.rom` is its ctypes binding.
"""
from .rom import (RomContext, RomError, default_options, lib, quadrature_xy,  # noqa: F401
                  KERNEL, QUAD, SCHEME, FACES, KERNEL_FLAG_NORMALIZE, KERNEL_FLAG_RAW)

__all__ = ["RomContext", "RomError", "default_options", "lib", "quadrature_xy"]
