"""ctypes loader for the FP64 C part of the oracle (test infrastructure only).

The shared object is compiled from ``frbx_oracle.c`` with plain gcc
(-O2 -ffp-contract=off -fopenmp) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frbx_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.oracle_fit_list.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                         ctypes.c_int, P, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P,
                                         ctypes.c_int64, P, P, P, P, P, ctypes.c_int]
        _lib.oracle_fit_list.restype = ctypes.c_int
        _lib.oracle_triple_sum.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                           ctypes.c_int, P, P]
        _lib.oracle_triple_sum.restype = None
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def fit_list(vis, n_bl, T, N, J, dk, flag, rot_re, rot_im, g, Ls, Lm, allow_m, allow_q, seg,
             want_grid=False, n_threads=0):
    n = seg.shape[0]
    amp = np.empty(n, np.float64)
    amp2 = np.empty(n, np.float64)
    m = np.empty(n, np.int32)
    q = np.empty(n, np.int32)
    grid = np.empty((n, Ls, Lm), np.complex128) if want_grid else None
    flag = np.ascontiguousarray(flag, np.uint8)
    am = None if allow_m is None else np.ascontiguousarray(allow_m, np.uint8)
    aq = None if allow_q is None else np.ascontiguousarray(allow_q, np.uint8)
    rc = lib().oracle_fit_list(_p(vis), n_bl, T, N, J, _p(dk), dk.shape[0], _p(flag), _p(rot_re),
                               _p(rot_im), _p(g), Ls, Lm, _p(am), _p(aq), _p(seg), n, _p(amp),
                               _p(m), _p(q), _p(amp2), _p(grid), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_fit_list: a segment reads outside the cube")
    return amp, m, q, amp2, grid


def triple_sum(x, N, J, flag, g, Ls, Lm):
    xr = np.ascontiguousarray(x.real, np.float64)
    xi = np.ascontiguousarray(x.imag, np.float64)
    gr = np.empty(Ls * Lm)
    gi = np.empty(Ls * Lm)
    lib().oracle_triple_sum(_p(xr), _p(xi), N, J, _p(np.ascontiguousarray(flag, np.uint8)),
                            _p(np.ascontiguousarray(g, np.int32)), Ls, Lm, _p(gr), _p(gi))
    return (gr + 1j * gi).reshape(Ls, Lm)


def num_threads() -> int:
    return int(lib().oracle_num_threads())
