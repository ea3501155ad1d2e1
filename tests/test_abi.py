"""The C ABI library builds, loads and exports what include/frbx.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1801_02391_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "frbx.h")


@pytest.fixture(scope="module")
def frbx():
    _build.build()
    from paper_1801_02391_gb300 import frbx as f
    f.load()
    return f


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(frbx_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_exported(frbx):
    names = declared_functions()
    assert len(names) >= 11
    lib = frbx.load()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(frbx.SIGNATURES) == names


def test_struct_layouts_match_header(frbx, tmp_path):
    """sizeof / offsetof of every ABI struct, compiled from the header with gcc, equal the
    ctypes and numpy layouts the binding uses."""
    structs = {"frbx_setup": frbx.frbx_setup, "frbx_params": frbx.frbx_params, "frbx_seg": frbx.frbx_seg,
               "frbx_event": frbx.frbx_event, "frbx_cand": frbx.frbx_cand, "frbx_group": frbx.frbx_group,
               "frbx_results": frbx.frbx_results, "frbx_scan": frbx.frbx_scan,
               "frbx_batch_stats": frbx.frbx_batch_stats, "frbx_limits": frbx.frbx_limits}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
    assert int(out["frbx_seg"]) == frbx.SEG_DTYPE.itemsize
    assert int(out["frbx_event"]) == frbx.EVENT_DTYPE.itemsize
    assert int(out["frbx_cand"]) == frbx.CAND_DTYPE.itemsize
    assert int(out["frbx_group"]) == frbx.GROUP_DTYPE.itemsize
    for fname in frbx.CAND_DTYPE.names:
        assert frbx.CAND_DTYPE.fields[fname][1] == getattr(frbx.frbx_cand, fname).offset


def test_default_params_are_the_papers(frbx):
    p = frbx.frbx_default_params()
    assert p.threshold == 3.0 and p.nwin_min == 3 and p.n_combo == 0
    assert p.sbd_win_ns[0] > p.sbd_win_ns[1] and p.mbd_win_ns[0] > p.mbd_win_ns[1]


def test_series_layout(frbx):
    off, tot = frbx.frbx_series_layout(20, [1, 4, 24])
    assert list(off) == [0, 20, 29] and tot == 29
    with pytest.raises(frbx.FrbxError):
        frbx.frbx_series_layout(20, [0])


def test_create_rejects_bad_setups_before_touching_the_gpu(frbx):
    lib = frbx.load()
    h = ctypes.c_void_p()
    f0 = np.array([1400.0, 1432.0])
    good = dict(n_chan=2, n_point=32, f0_mhz=f0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                f_bw_mhz=32.0, t_ap_ms=1.0)
    for bad in (dict(n_chan=0), dict(n_point=1), dict(f_bw_mhz=-1.0), dict(t_ap_ms=0.0),
                dict(f_ref_dm_mhz=1000.0), dict(sbd_pad=3), dict(mbd_pad=-1)):
        s = frbx.frbx_setup(**{**good, **bad})
        rc = lib.frbx_create(ctypes.byref(s), ctypes.byref(h))
        assert rc in (frbx.FRBX_EINVAL, frbx.FRBX_EUNSUPPORTED), bad
        assert not h.value
    s = frbx.frbx_setup(**{**good, "f0_mhz": np.array([1400.0, 1432.0004]).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))})
    assert lib.frbx_create(ctypes.byref(s), ctypes.byref(h)) == frbx.FRBX_EINVAL
    assert lib.frbx_create(None, ctypes.byref(h)) == frbx.FRBX_EINVAL
    assert lib.frbx_last_error(None) == b"null handle"
    lib.frbx_destroy(None)


def test_limits_entry_points_reject_null_and_negative_without_a_gpu(frbx):
    lib = frbx.load()
    lim = frbx.frbx_limits()
    assert lib.frbx_set_limits(None, ctypes.byref(lim)) == frbx.FRBX_EINVAL
    assert lib.frbx_get_limits(None, ctypes.byref(lim)) == frbx.FRBX_EINVAL
    assert lib.frbx_scratch_bytes(None) == -1


def test_peak_probe_library_exports_its_header(frbx):
    from paper_1801_02391_gb300 import peaks
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "frbx_peaks.h")).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(frbx_[a-z_]+)\s*\(", text)))
    lib = peaks.load()
    assert names == sorted(peaks.SIGNATURES)
    for n in names:
        assert hasattr(lib, n), n
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.frbx_peak_probe(9, 1, ctypes.byref(tf), ctypes.byref(ms), None) == -1  # rejected before any CUDA call


def test_fp64_host_code_built_without_contraction():
    """Host code that computes FP64 tables is compiled with -ffp-contract=off, so the shift
    table inputs are identical on x86 and Arm hosts."""
    assert "-fPIC,-ffp-contract=off" in _build.NVCC_FLAGS
