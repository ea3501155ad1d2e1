"""frbx_fit_segments_noalloc: the segment fit without any device allocation.

It is for callers that must not allocate device memory when they call the library (memory
reserved up front by a real-time back end, a framework's caching allocator, or code that
must not risk the device-wide synchronisation of cudaMalloc / cudaFree).  Its scratch is a
fixed array inside the library.  Checked here through the C ABI against frbx_fit_segments
(the allocating entry point) with the FP32 tolerances of the parity tests, on two calls in a
row with different inputs, so nothing left in the shared array from the first call leaks
into the second.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import reference as R
from paper_1801_02391_gb300 import _build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build.build()
    from paper_1801_02391_gb300 import frbx as f
    f.load()
    return f


def _setup_struct(frbx, wl, keep):
    f0 = np.ascontiguousarray(wl.f0_mhz, np.float64)
    fl = None if wl.flags is None else np.ascontiguousarray(wl.flags, np.uint8)
    keep += [f0, fl]
    return frbx.frbx_setup(n_chan=len(f0), n_point=wl.n_point, f0_mhz=frbx._ptr(f0, ctypes.c_double),
                           f_bw_mhz=wl.f_bw_mhz, t_ap_ms=wl.t_ap_ms, f_ref_dm_mhz=0.0,
                           flag=frbx._ptr(fl, ctypes.c_uint8), sbd_pad=wl.sbd_pad, mbd_pad=wl.mbd_pad)


def _noalloc(frbx, wl, vis_dev, segs):
    import torch
    keep = []
    s = _setup_struct(frbx, wl, keep)
    dm = np.ascontiguousarray(wl.dms, np.float64)
    sg = np.ascontiguousarray(segs, np.int32)
    out = torch.zeros(sg.shape[0] * 2, dtype=torch.float32, device="cuda")   # frbx_seg = 8 bytes
    rc = frbx.load().frbx_fit_segments_noalloc(ctypes.byref(s), ctypes.c_void_p(vis_dev.data_ptr()), wl.n_bl, wl.T,
                                               frbx._ptr(dm, ctypes.c_double), len(dm),
                                               frbx._ptr(sg, ctypes.c_int32), sg.shape[0],
                                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == frbx.FRBX_OK, rc
    return np.frombuffer(out.cpu().numpy().tobytes(), dtype=frbx.SEG_DTYPE)


def _rows(wl, n, seed):
    st = R.setup_from_workload(wl)
    dk_max = R.shift_table(st, wl.dms).max(axis=1)
    rng = np.random.default_rng(seed)
    rows = []
    while len(rows) < n:
        b, d = int(rng.integers(0, wl.n_bl)), int(rng.integers(0, len(wl.dms)))
        l = int(rng.choice(wl.windows))
        nv = R.n_valid(wl.T, l, int(dk_max[d]))
        if nv > 0:
            rows.append((b, d, l, int(rng.integers(0, nv)) * R.window_step(l)))
    return np.array(rows, np.int32)


def _compare(a, b):
    np.testing.assert_allclose(a["amp"], b["amp"], rtol=1e-4)
    same = (a["sbd_idx"] == b["sbd_idx"]) & (a["mbd_idx"] == b["mbd_idx"])
    assert same.mean() > 0.99


def test_noalloc_matches_allocating_entry_point_twice(frbx):
    import torch
    cases = []
    wl1 = synth.make_small(T=600, dms=[0.0, 300.0, 557.0])
    wl2 = synth.make_vgos(T=200, n_bl=2)
    wl2.dms = np.array([0.0, 50.0, 120.0])
    for wl, seed in ((wl1, 1), (wl2, 2)):
        vis = synth.generate(wl)
        vis_dev = torch.from_numpy(vis).cuda()
        segs = _rows(wl, 150, seed)
        ref = frbx.Handle.from_workload(wl).fit_segments(vis_dev, wl.dms, segs, kernel=1)
        got = _noalloc(frbx, wl, vis_dev, segs)
        _compare(got, ref)
        cases.append(got)
    assert cases[0].shape == (150,) and cases[1].shape == (150,)


def test_noalloc_rejects_rows_outside_the_cube(frbx):
    import torch
    wl = synth.make_small(T=64, dms=[0.0, 100.0])
    vis_dev = torch.from_numpy(synth.generate(wl)).cuda()
    keep = []
    s = _setup_struct(frbx, wl, keep)
    dm = np.ascontiguousarray(wl.dms, np.float64)
    sg = np.array([[0, 1, 4, 60]], np.int32)
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    rc = frbx.load().frbx_fit_segments_noalloc(ctypes.byref(s), ctypes.c_void_p(vis_dev.data_ptr()), wl.n_bl, wl.T,
                                               frbx._ptr(dm, ctypes.c_double), 2, frbx._ptr(sg, ctypes.c_int32), 1,
                                               ctypes.c_void_p(out.data_ptr()), None)
    assert rc == frbx.FRBX_EINVAL
