"""frbx_fit_segments_noalloc: the segment fit without any device allocation.

It is for callers that must not allocate device memory when they call the library (memory
reserved up front by a real-time back end, a framework's caching allocator, or code that
must not risk the device-wide synchronisation of cudaMalloc / cudaFree).  Its scratch is a
fixed array inside the library.  Checked here through the C ABI, on two calls in a row (a
large setup first, then a small one, so the second call reads next to what the first left in
the shared array): bit for bit against frbx_fit_segments with the same direct-DFT kernel on a
handle of the same setup (channel delays, initial phases and flags included), against the
FP64 oracle with the parity tests' rules, and with the device's free memory unchanged across
calls once the first call has loaded the library on the device.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import reference as R
from paper_1801_02391_gb300 import _build
from tests.gpu_helpers import assert_fit_match

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


def _setup_struct(frbx, wl, keep, cal=None):
    cal = cal or {}
    f0 = np.ascontiguousarray(wl.f0_mhz, np.float64)
    fl = None if wl.flags is None else np.ascontiguousarray(wl.flags, np.uint8)
    dt = None if "chan_delay_ns" not in cal else np.ascontiguousarray(cal["chan_delay_ns"], np.float64)
    dp = None if "chan_phase_rad" not in cal else np.ascontiguousarray(cal["chan_phase_rad"], np.float64)
    keep += [f0, fl, dt, dp]
    return frbx.frbx_setup(n_chan=len(f0), n_point=wl.n_point, f0_mhz=frbx._ptr(f0, ctypes.c_double),
                           f_bw_mhz=wl.f_bw_mhz, t_ap_ms=wl.t_ap_ms, f_ref_dm_mhz=0.0,
                           chan_delay_ns=frbx._ptr(dt, ctypes.c_double), chan_phase_rad=frbx._ptr(dp, ctypes.c_double),
                           flag=frbx._ptr(fl, ctypes.c_uint8), sbd_pad=wl.sbd_pad, mbd_pad=wl.mbd_pad)


def _call(frbx, wl, vis_dev, segs, out, cal=None):
    """One call of the entry point through the C ABI (out: a preallocated CUDA tensor)."""
    keep = []
    s = _setup_struct(frbx, wl, keep, cal)
    dm = np.ascontiguousarray(wl.dms, np.float64)
    sg = np.ascontiguousarray(segs, np.int32)
    return frbx.load().frbx_fit_segments_noalloc(ctypes.byref(s), ctypes.c_void_p(vis_dev.data_ptr()), wl.n_bl, wl.T,
                                                 frbx._ptr(dm, ctypes.c_double), len(dm),
                                                 frbx._ptr(sg, ctypes.c_int32), sg.shape[0],
                                                 ctypes.c_void_p(out.data_ptr()), None)


def _as_segs(frbx, out):
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


def test_noalloc_matches_allocating_entry_point_and_oracle_twice(frbx):
    import torch
    # large setup first (VGOS-like, 2048 points, calibration and flags), then a small one
    wl1 = synth.make_vgos(T=200, n_bl=2)
    wl1.dms = np.array([0.0, 50.0, 120.0])
    rng = np.random.default_rng(17)
    cal1 = dict(chan_delay_ns=rng.uniform(-5, 5, wl1.n_chan), chan_phase_rad=rng.uniform(-3, 3, wl1.n_chan))
    wl2 = synth.make_small(T=600, dms=[0.0, 300.0, 557.0])
    cases = [(wl1, cal1, _rows(wl1, 160, 1)), (wl2, {}, _rows(wl2, 150, 2))]
    inputs = []
    for wl, cal, segs in cases:
        vis = synth.generate(wl)
        out = torch.zeros(segs.shape[0] * 2, dtype=torch.float32, device="cuda")  # frbx_seg = 8 bytes
        inputs.append((wl, cal, segs, vis, torch.from_numpy(vis).cuda(), out))
    # the first call on the device may load the library's device code (and its array)
    wl, cal, segs, vis, vis_dev, out = inputs[0]
    assert _call(frbx, wl, vis_dev, segs[:0], out, cal) == frbx.FRBX_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = []
    for wl, cal, segs, vis, vis_dev, out in inputs:
        assert _call(frbx, wl, vis_dev, segs, out, cal) == frbx.FRBX_OK
        got.append(_as_segs(frbx, out))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "a call allocated device memory"
    for (wl, cal, segs, vis, vis_dev, out), g in zip(inputs, got):
        ref = frbx.Handle.from_workload(wl, **cal).fit_segments(vis_dev, wl.dms, segs, kernel=1)
        assert np.array_equal(g, ref), "differs from frbx_fit_segments(kernel=1) on the same setup"
        st = R.setup_from_workload(wl, **cal)
        dk = R.shift_table(st, wl.dms)
        assert_fit_match(st, vis, dk, segs, g, R.fit_segments(st, vis, dk, segs))


def test_noalloc_rejects_rows_outside_the_cube_and_oversized_calls(frbx):
    import torch
    wl = synth.make_small(T=64, dms=[0.0, 100.0])
    vis_dev = torch.from_numpy(synth.generate(wl)).cuda()
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    assert _call(frbx, wl, vis_dev, np.array([[0, 1, 4, 60]], np.int32), out) == frbx.FRBX_EINVAL
    # a shift table beyond the fixed array: 2048 DM trials x 256 points x 4 bytes = 2 MiB fits,
    # 20000 trials (20 MiB) does not
    big = synth.make_small(T=64, dms=np.linspace(0.0, 10.0, 20000))
    assert _call(frbx, big, vis_dev, np.array([[0, 0, 2, 0]], np.int32), out) == frbx.FRBX_EINVAL
    assert _call(frbx, wl, vis_dev, np.array([[0, 0, 2, 0]], np.int32), out) == frbx.FRBX_OK
