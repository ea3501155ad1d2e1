"""GB300-native cross-spectrum FRB search (arxiv 1801.02391): libfrbx + Python binding.

The compute path is the CUDA library ``libfrbx`` (``csrc/``, C ABI in
``include/frbx.h``); ``paper_1801_02391_gb300.frbx`` is its ctypes binding.
Build with ``paper_1801_02391_gb300.build()``.
"""
from . import _build  # noqa: F401


def build(force: bool = False) -> str:
    return _build.build(force=force)
