"""Binding of libfrbx_peaks (include/frbx_peaks.h): peak-rate probes of the current GPU, the
roofline denominators the bench measures itself (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import _build

KINDS = {"fp32_fma": 0, "fp32_fma2": 1, "bf16_mma": 2, "fp8_mma": 3}
SIGNATURES = {"frbx_peak_probe": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p])}
_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB_PEAKS):
            raise OSError(f"libfrbx_peaks not built ({_build.LIB_PEAKS} missing)")
        lib = ctypes.CDLL(_build.LIB_PEAKS)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def probe(kind: str, iters: int, stream=None) -> tuple[float, float]:
    """(TFLOP/s, ms) of one probe launch on the current device."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    sp = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    rc = load().frbx_peak_probe(KINDS[kind], int(iters), ctypes.byref(tf), ctypes.byref(ms), sp)
    if rc != 0:
        raise RuntimeError(f"frbx_peak_probe({kind}) failed with {rc}")
    return tf.value, ms.value
