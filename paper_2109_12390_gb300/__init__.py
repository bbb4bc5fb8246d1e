"""GB300-native (sm_103a) hot path of MPM model reduction with an implicit neural decoder.

The compute runs in ``_lib/libmpmrom.so`` (CUDA kernels under ``csrc/``,
C ABI in ``include/mpmrom.h``); this package only marshals arguments.
"""
from . import _abi  # noqa: F401

__all__ = ["build", "mpm"]


def build(verbose=False):
    from .build import build as _build
    return _build(verbose=verbose)
