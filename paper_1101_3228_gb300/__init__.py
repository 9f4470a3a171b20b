"""GB300-native Quantization Tree forward step (Pages & Wilbertz, arXiv:1101.3228).

The compute path is libqt (C ABI in include/qt.h, CUDA kernels under csrc/);
``binding`` is its thin ctypes binding and ``build`` compiles it for sm_103a.
"""
from . import build  # noqa: F401

__all__ = ["build", "binding"]
