"""Python binding of libfrbx (ctypes): argument marshalling only.

Every function named ``frbx_*`` here is the C entry point of the same name in
``include/frbx.h``; :class:`Handle` wraps them for numpy arrays and torch
tensors (device pointers are taken from ``tensor.data_ptr()``).  All compute
runs in the library's CUDA kernels; if the shared library is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FRBX_OK, FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA, FRBX_ETRUNC, FRBX_ETIMEOUT, FRBX_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETRUNC", -5: "ETIMEOUT", -6: "EUNSUPPORTED"}

c_i32, c_i64, c_f32, c_f64, c_u64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p
P = ctypes.POINTER


class FrbxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"frbx error {_NAMES.get(code, code)}: {msg}")
        self.code = code


class frbx_setup(ctypes.Structure):
    _fields_ = [("n_chan", c_i32), ("n_point", c_i32), ("f0_mhz", P(c_f64)), ("f_bw_mhz", c_f64),
                ("t_ap_ms", c_f64), ("f_ref_dm_mhz", c_f64), ("chan_delay_ns", P(c_f64)),
                ("chan_phase_rad", P(c_f64)), ("flag", P(ctypes.c_uint8)), ("sbd_pad", c_i32),
                ("mbd_pad", c_i32)]


class frbx_params(ctypes.Structure):
    _fields_ = [("threshold", c_f32), ("nwin_min", c_i32), ("sbd_win_ns", c_f64 * 2),
                ("mbd_win_ns", c_f64 * 2), ("combos", P(c_u64)), ("n_combo", c_i32), ("kernel", c_i32)]


class frbx_seg(ctypes.Structure):
    _fields_ = [("amp", c_f32), ("sbd_idx", ctypes.c_uint16), ("mbd_idx", ctypes.c_uint16)]


SEG_DTYPE = np.dtype([("amp", np.float32), ("sbd_idx", np.uint16), ("mbd_idx", np.uint16)])


class frbx_event(ctypes.Structure):
    _fields_ = [("series", c_i32), ("dm_idx", c_i32), ("win_idx", c_i32), ("k0", c_i32), ("amp", c_f32),
                ("pnorm", c_f32), ("sbd_idx", ctypes.c_uint16), ("mbd_idx", ctypes.c_uint16)]


EVENT_DTYPE = np.dtype([("series", np.int32), ("dm_idx", np.int32), ("win_idx", np.int32), ("k0", np.int32),
                        ("amp", np.float32), ("pnorm", np.float32), ("sbd_idx", np.uint16), ("mbd_idx", np.uint16)])


class frbx_cand(ctypes.Structure):
    _fields_ = [("series", c_i32), ("dm_idx", c_i32), ("win_idx", c_i32), ("width", c_i32), ("k0", c_i32),
                ("sbd_idx", c_i32), ("mbd_idx", c_i32), ("n_win", c_i32), ("group", c_i32), ("amp", c_f32),
                ("pnorm", c_f32), ("reserved", c_i32), ("t_s", c_f64), ("sbd_ns", c_f64), ("mbd_ns", c_f64),
                ("dm", c_f64)]


CAND_DTYPE = np.dtype([("series", np.int32), ("dm_idx", np.int32), ("win_idx", np.int32), ("width", np.int32),
                       ("k0", np.int32), ("sbd_idx", np.int32), ("mbd_idx", np.int32), ("n_win", np.int32),
                       ("group", np.int32), ("amp", np.float32), ("pnorm", np.float32), ("reserved", np.int32),
                       ("t_s", np.float64), ("sbd_ns", np.float64), ("mbd_ns", np.float64), ("dm", np.float64)])


class frbx_group(ctypes.Structure):
    _fields_ = [("bl_mask", c_u64), ("n_baselines", c_i32), ("n_pulses", c_i32)]


GROUP_DTYPE = np.dtype([("bl_mask", np.uint64), ("n_baselines", np.int32), ("n_pulses", np.int32)])


class frbx_results(ctypes.Structure):
    _fields_ = [("pulses", c_vp), ("pulses_cap", c_i64), ("pulses_count", c_i64),
                ("groups", c_vp), ("groups_cap", c_i64), ("groups_count", c_i64),
                ("combined", c_vp), ("combined_cap", c_i64), ("combined_count", c_i64),
                ("pulses_dm", c_vp), ("pulses_dm_cap", c_i64), ("pulses_dm_count", c_i64),
                ("events", c_vp), ("events_cap", c_i64), ("events_count", c_i64),
                ("series", c_vp), ("pnorm", c_vp), ("series_on_device", c_i32), ("reserved", c_i32),
                ("series_cap", c_i64), ("series_count", c_i64), ("events_baseline_count", c_i64)]


class frbx_scan(ctypes.Structure):
    _fields_ = [("setup", c_vp), ("vis_dev", c_vp), ("n_bl", c_i32), ("T", c_i32)]


class frbx_batch_stats(ctypes.Structure):
    _fields_ = [("graph_captures", c_i32), ("graph_replays", c_i32), ("n_setups", c_i32),
                ("time_tile", c_i32 * 16), ("reserved", c_i32), ("fit_ms", c_f64), ("launches", c_i64)]


class frbx_limits(ctypes.Structure):
    _fields_ = [("tree_chunk_bytes", c_i64), ("wait_cycles", c_i64), ("scratch_cap_bytes", c_i64),
                ("hold_producers", c_i32), ("reserved", c_i32)]


assert ctypes.sizeof(frbx_cand) == CAND_DTYPE.itemsize == 80
assert ctypes.sizeof(frbx_event) == EVENT_DTYPE.itemsize == 28

# Every entry point of include/frbx.h with its ctypes signature.
SIGNATURES = {
    "frbx_default_params": (None, [P(frbx_params)]),
    "frbx_create": (c_i32, [P(frbx_setup), P(c_vp)]),
    "frbx_destroy": (None, [c_vp]),
    "frbx_last_error": (ctypes.c_char_p, [c_vp]),
    "frbx_grid_info": (c_i32, [c_vp, P(c_i32), P(c_i32), P(c_f64), P(c_i32)]),
    "frbx_shift_table": (c_i32, [c_vp, P(c_f64), c_i32, P(c_i32), c_vp]),
    "frbx_series_layout": (c_i64, [c_i32, P(c_i32), c_i32, P(c_i64)]),
    "frbx_search": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, P(c_f64), c_i32, P(c_i32), c_i32,
                            P(frbx_params), P(frbx_results), c_vp]),
    "frbx_fit_segments": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, P(c_f64), c_i32, P(c_i32), c_i64,
                                  P(frbx_params), c_vp, c_vp]),
    "frbx_last_launch_count": (c_i64, [c_vp]),
    "frbx_last_stage_times": (c_i32, [c_vp, P(c_f64), c_i32]),
    "frbx_refine_power": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "frbx_refine_adjoint": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "frbx_calibrate": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, c_i32, c_i32, P(c_f64), P(c_f64), P(c_f64),
                               P(c_f64), c_vp]),
    "frbx_fit_segments_noalloc": (c_i32, [P(frbx_setup), c_vp, c_i32, c_i32, P(c_f64), c_i32, P(c_i32), c_i64,
                                          c_vp, c_vp]),
    "frbx_batch_create": (c_i32, [P(c_vp)]),
    "frbx_batch_destroy": (None, [c_vp]),
    "frbx_batch_last_error": (ctypes.c_char_p, [c_vp]),
    "frbx_batch_info": (c_i32, [c_vp, P(frbx_batch_stats)]),
    "frbx_search_batch": (c_i32, [c_vp, P(frbx_scan), c_i32, P(c_f64), c_i32, P(c_i32), c_i32, P(frbx_params),
                                  P(frbx_results), c_vp]),
    "frbx_set_limits": (c_i32, [c_vp, P(frbx_limits)]),
    "frbx_get_limits": (c_i32, [c_vp, P(frbx_limits)]),
    "frbx_scratch_bytes": (c_i64, [c_vp]),
    "frbx_extract_events": (c_i32, [c_vp, c_i64, c_i32, c_i32, c_i32, P(c_i32), c_i32, c_i32, c_i32, c_i32,
                                    c_vp, c_i64, P(c_i64), c_vp, c_i64, P(c_i64), c_vp, c_i64, P(c_i64)]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfrbx (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        p = path or _build.LIB
        if not os.path.exists(p):
            raise OSError(f"libfrbx not built ({p} missing); run paper_1801_02391_gb300._build.build()")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(P(ctype))


def _check(h, rc):
    if rc != FRBX_OK:
        raise FrbxError(rc, load().frbx_last_error(h).decode())


# thin module-level aliases with the C names
def frbx_default_params():
    p = frbx_params()
    load().frbx_default_params(ctypes.byref(p))
    return p


def frbx_series_layout(T, windows):
    w = np.ascontiguousarray(windows, np.int32)
    off = np.zeros(len(w), np.int64)
    tot = load().frbx_series_layout(int(T), _ptr(w, c_i32), len(w), _ptr(off, c_i64))
    if tot < 0:
        raise FrbxError(int(tot), "bad layout arguments")
    return off, int(tot)


def frbx_extract_events(events, n_series, T, n_dm, windows, Lm, nwin_min=3, cross_match=True):
    """Host extraction (steps b-d, DM merge, cross-matching) of a sorted event array
    (EVENT_DTYPE).  Returns (pulses, groups, pre_merge) structured arrays."""
    ev = np.ascontiguousarray(events, EVENT_DTYPE)
    win = np.ascontiguousarray(windows, np.int32)
    caps = [max(16, ev.size)] * 3
    for _ in range(2):
        pul = np.zeros(caps[0], CAND_DTYPE)
        grp = np.zeros(caps[1], GROUP_DTYPE)
        pre = np.zeros(caps[2], CAND_DTYPE)
        n = [c_i64(), c_i64(), c_i64()]
        rc = load().frbx_extract_events(ev.ctypes.data_as(c_vp) if ev.size else None, ev.size, int(n_series), int(T),
                                        int(n_dm), _ptr(win, c_i32), len(win), int(Lm), int(nwin_min),
                                        1 if cross_match else 0, pul.ctypes.data_as(c_vp), pul.size,
                                        ctypes.byref(n[0]), grp.ctypes.data_as(c_vp), grp.size, ctypes.byref(n[1]),
                                        pre.ctypes.data_as(c_vp), pre.size, ctypes.byref(n[2]))
        if rc == FRBX_ETRUNC:
            caps = [max(c, v.value) for c, v in zip(caps, n)]
            continue
        if rc != FRBX_OK:
            raise FrbxError(rc, "frbx_extract_events rejected its arguments")
        return pul[:n[0].value].copy(), grp[:n[1].value].copy(), pre[:n[2].value].copy()
    raise FrbxError(FRBX_ETRUNC, "output sizes kept growing")


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _vis_arg(vis):
    """(pointer, on_device, keepalive, shape) of a complex64 cube [n_bl][T][C]."""
    try:
        import torch
        if isinstance(vis, torch.Tensor):
            t = vis
            if t.dtype == torch.complex64:
                pass
            elif t.dtype == torch.float32 and t.shape[-1] == 2:
                t = torch.view_as_complex(t)
            else:
                raise TypeError("vis must be complex64 (or float32 [..., 2])")
            if not t.is_contiguous():
                raise ValueError("vis must be contiguous")
            return ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, t, tuple(t.shape)
    except ImportError:
        pass
    a = np.ascontiguousarray(vis, np.complex64)
    return a.ctypes.data_as(c_vp), 0, a, a.shape


_RESULT_KINDS = (("pulses", "CAND"), ("groups", "GROUP"), ("combined", "CAND"), ("pulses_dm", "CAND"),
                 ("events", "EVENT"))


def _default_caps(caps, want_events, want_pre_merge):
    caps = dict(caps or {})
    caps.setdefault("pulses", 1 << 16)
    caps.setdefault("groups", 1 << 16)
    caps.setdefault("combined", 1 << 16)
    caps.setdefault("pulses_dm", 1 << 18 if want_pre_merge else 0)
    caps.setdefault("events", 1 << 20 if want_events else 0)
    return caps


def _result_buffers(caps):
    """Host output arrays of the sizes in caps and a frbx_results pointing at them."""
    dt = {"CAND": CAND_DTYPE, "GROUP": GROUP_DTYPE, "EVENT": EVENT_DTYPE}
    bufs = {k: np.zeros(caps[k], dt[kind]) for k, kind in _RESULT_KINDS}
    r = frbx_results()
    for k, arr in bufs.items():
        setattr(r, k, arr.ctypes.data_as(c_vp) if arr.size else None)
        setattr(r, k + "_cap", arr.size)
    return bufs, r


def _collect(bufs, r):
    out = {k: bufs[k][:int(getattr(r, k + "_count"))].copy() if bufs[k].size else None for k in bufs}
    out["counts"] = {k: int(getattr(r, k + "_count")) for k in bufs}
    out["counts"]["events_baseline"] = int(r.events_baseline_count)
    return out


class Handle:
    """One observing setup on the current CUDA device (frbx_create / frbx_destroy)."""

    def __init__(self, f0_mhz, n_point, f_bw_mhz, t_ap_ms, f_ref_dm_mhz=0.0, chan_delay_ns=None,
                 chan_phase_rad=None, flag=None, sbd_pad=2, mbd_pad=2):
        lib = load()
        self._f0 = np.ascontiguousarray(f0_mhz, np.float64)
        self._dt = None if chan_delay_ns is None else np.ascontiguousarray(chan_delay_ns, np.float64)
        self._dp = None if chan_phase_rad is None else np.ascontiguousarray(chan_phase_rad, np.float64)
        self._fl = None if flag is None else np.ascontiguousarray(flag, np.uint8)
        s = frbx_setup(n_chan=len(self._f0), n_point=int(n_point), f0_mhz=_ptr(self._f0, c_f64),
                       f_bw_mhz=float(f_bw_mhz), t_ap_ms=float(t_ap_ms), f_ref_dm_mhz=float(f_ref_dm_mhz),
                       chan_delay_ns=_ptr(self._dt, c_f64), chan_phase_rad=_ptr(self._dp, c_f64),
                       flag=_ptr(self._fl, ctypes.c_uint8), sbd_pad=int(sbd_pad), mbd_pad=int(mbd_pad))
        h = c_vp()
        rc = lib.frbx_create(ctypes.byref(s), ctypes.byref(h))
        if rc != FRBX_OK:
            raise FrbxError(rc, "frbx_create rejected the setup")
        self.h = h
        self.n_chan, self.n_point = len(self._f0), int(n_point)
        self.C = self.n_chan * self.n_point
        self.Ls, self.Lm, self.df_grid_mhz, self.g = self.grid_info()

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.f0_mhz, wl.n_point, wl.f_bw_mhz, wl.t_ap_ms, flag=wl.flags, sbd_pad=wl.sbd_pad,
                   mbd_pad=wl.mbd_pad, **kw)

    def close(self):
        if getattr(self, "h", None):
            load().frbx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return load().frbx_last_error(self.h).decode()

    def launch_count(self) -> int:
        return int(load().frbx_last_launch_count(self.h))

    def set_limits(self, tree_chunk_bytes=0, wait_cycles=0, scratch_cap_bytes=0, hold_producers=0):
        """frbx_set_limits: zero in a field means its default (frbx_limits in include/frbx.h)."""
        lim = frbx_limits(tree_chunk_bytes=int(tree_chunk_bytes), wait_cycles=int(wait_cycles),
                          scratch_cap_bytes=int(scratch_cap_bytes), hold_producers=int(hold_producers))
        _check(self.h, load().frbx_set_limits(self.h, ctypes.byref(lim)))

    def get_limits(self) -> dict:
        lim = frbx_limits()
        _check(self.h, load().frbx_get_limits(self.h, ctypes.byref(lim)))
        return {k: int(getattr(lim, k)) for k, _ in frbx_limits._fields_ if k != "reserved"}

    def scratch_bytes(self) -> int:
        return int(load().frbx_scratch_bytes(self.h))

    STAGES = ("shift_table", "fit", "normalise_baselines", "normalise_combos", "host_extract",
              "tree_sbd_kernels", "tree_mbd_kernels", "tree_chunks", "tree_tensor")

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last search (CUDA events on its stream)."""
        out = np.zeros(9, np.float64)
        n = load().frbx_last_stage_times(self.h, _ptr(out, c_f64), 9)
        if n < 0:
            raise FrbxError(n, "frbx_last_stage_times")
        return dict(zip(self.STAGES, out.tolist()))

    def grid_info(self):
        Ls, Lm, df = c_i32(), c_i32(), c_f64()
        g = np.zeros(self.n_chan, np.int32)
        _check(self.h, load().frbx_grid_info(self.h, ctypes.byref(Ls), ctypes.byref(Lm), ctypes.byref(df),
                                             _ptr(g, c_i32)))
        return Ls.value, Lm.value, df.value, g

    def _params(self, threshold=3.0, nwin_min=3, sbd_win_ns=None, mbd_win_ns=None, combos=(), kernel=0):
        p = frbx_default_params()
        p.threshold = float(threshold)
        p.nwin_min = int(nwin_min)
        if sbd_win_ns is not None:
            p.sbd_win_ns[0], p.sbd_win_ns[1] = float(sbd_win_ns[0]), float(sbd_win_ns[1])
        if mbd_win_ns is not None:
            p.mbd_win_ns[0], p.mbd_win_ns[1] = float(mbd_win_ns[0]), float(mbd_win_ns[1])
        cm = np.ascontiguousarray(np.asarray(combos, dtype=np.uint64).reshape(-1))
        p.combos = _ptr(cm, c_u64) if cm.size else None
        p.n_combo = int(cm.size)
        p.kernel = int(kernel)
        return p, cm

    def shift_table(self, dms, stream=None):
        dm = np.ascontiguousarray(dms, np.float64)
        out = np.zeros((len(dm), self.C), np.int32)
        _check(self.h, load().frbx_shift_table(self.h, _ptr(dm, c_f64), len(dm), _ptr(out, c_i32),
                                               _stream_ptr(stream)))
        return out

    def calibrate(self, vis, k0, l, stream=None):
        """Appendix A: (sbd_ns [n_bl], mbd_ns [n_bl], delay_ns [n_bl][N], phase_rad [n_bl][N])."""
        vp, on_dev, keep, shape = _vis_arg(vis)
        n_bl, T, C = shape
        sbd = np.zeros(n_bl)
        mbd = np.zeros(n_bl)
        dl = np.zeros((n_bl, self.n_chan))
        ph = np.zeros((n_bl, self.n_chan))
        _check(self.h, load().frbx_calibrate(self.h, vp, on_dev, n_bl, T, int(k0), int(l), _ptr(sbd, c_f64),
                                             _ptr(mbd, c_f64), _ptr(dl, c_f64), _ptr(ph, c_f64), _stream_ptr(stream)))
        return sbd, mbd, dl, ph

    def fit_segments(self, vis, dms, segs, kernel=0, sbd_win_ns=None, mbd_win_ns=None, stream=None):
        vp, on_dev, keep, shape = _vis_arg(vis)
        n_bl, T, C = shape
        assert C == self.C
        dm = np.ascontiguousarray(dms, np.float64)
        sg = np.ascontiguousarray(segs, np.int32).reshape(-1, 4)
        out = np.zeros(sg.shape[0], SEG_DTYPE)
        p, cm = self._params(sbd_win_ns=sbd_win_ns, mbd_win_ns=mbd_win_ns, kernel=kernel)
        _check(self.h, load().frbx_fit_segments(self.h, vp, on_dev, n_bl, T, _ptr(dm, c_f64), len(dm),
                                                _ptr(sg, c_i32), sg.shape[0], ctypes.byref(p),
                                                out.ctypes.data_as(c_vp), _stream_ptr(stream)))
        return out

    def search(self, vis, dms, windows, threshold=3.0, nwin_min=3, combos=(), sbd_win_ns=None,
               mbd_win_ns=None, kernel=0, want_series=False, want_events=False, want_pre_merge=False,
               series_out=None, pnorm_out=None, caps=None, stream=None):
        """Run frbx_search.  Returns a dict of numpy structured arrays.  If an output is
        truncated the call is repeated once with the sizes the library reported.
        series_out / pnorm_out may be CUDA tensors (then the series stay on the device)."""
        vp, on_dev, keep, shape = _vis_arg(vis)
        n_bl, T, C = shape
        assert C == self.C, "cube does not match the setup"
        dm = np.ascontiguousarray(dms, np.float64)
        win = np.ascontiguousarray(windows, np.int32)
        p, cm = self._params(threshold, nwin_min, sbd_win_ns, mbd_win_ns, combos, kernel)
        _, S_tot = frbx_series_layout(T, win)
        n_series = n_bl * len(dm) * S_tot
        caps = _default_caps(caps, want_events, want_pre_merge)
        for attempt in range(2):
            bufs, r = _result_buffers(caps)
            ser_host = pn_host = None
            if series_out is not None or pnorm_out is not None:
                r.series_on_device = 1
                r.series = ctypes.c_void_p(series_out.data_ptr()) if series_out is not None else None
                r.pnorm = ctypes.c_void_p(pnorm_out.data_ptr()) if pnorm_out is not None else None
                r.series_cap = n_series
            elif want_series:
                ser_host = np.zeros(n_series, SEG_DTYPE)
                pn_host = np.zeros(n_series, np.float32)
                r.series = ser_host.ctypes.data_as(c_vp)
                r.pnorm = pn_host.ctypes.data_as(c_vp)
                r.series_on_device = 0
                r.series_cap = n_series
            rc = load().frbx_search(self.h, vp, on_dev, n_bl, T, _ptr(dm, c_f64), len(dm), _ptr(win, c_i32),
                                    len(win), ctypes.byref(p), ctypes.byref(r), _stream_ptr(stream))
            if rc == FRBX_ETRUNC and attempt == 0:
                for k in bufs:
                    if bufs[k].size:
                        caps[k] = max(caps[k], int(getattr(r, k + "_count")))
                continue
            _check(self.h, rc)
            break
        out = _collect(bufs, r)
        out["S_tot"] = S_tot
        out["launches"] = self.launch_count()
        if ser_host is not None:
            out["series"] = ser_host.reshape(n_bl, len(dm), S_tot)
            out["pnorm"] = pn_host.reshape(n_bl, len(dm), S_tot)
        return out


class Batch:
    """Batched search over many device-resident scans (frbx_batch_* / frbx_search_batch).

    The object keeps the captured fit graph and the tuned time tiles between calls: a second
    call with scans of the same shapes in the same buffers replays the graph."""

    def __init__(self):
        b = c_vp()
        rc = load().frbx_batch_create(ctypes.byref(b))
        if rc != FRBX_OK:
            raise FrbxError(rc, "frbx_batch_create failed")
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            load().frbx_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return load().frbx_batch_last_error(self.b).decode()

    def info(self) -> dict:
        st = frbx_batch_stats()
        rc = load().frbx_batch_info(self.b, ctypes.byref(st))
        if rc != FRBX_OK:
            raise FrbxError(rc, "frbx_batch_info")
        return {"graph_captures": st.graph_captures, "graph_replays": st.graph_replays,
                "time_tile": list(st.time_tile[:st.n_setups]), "fit_ms": st.fit_ms, "launches": st.launches}

    def search(self, scans, dms, windows, threshold=3.0, nwin_min=3, combos=(), sbd_win_ns=None,
               mbd_win_ns=None, kernel=0, want_series=False, want_events=False, want_pre_merge=False,
               caps=None, stream=None):
        """scans: sequence of (Handle, complex64 CUDA tensor [n_bl][T][C]).  Returns one dict per
        scan, as Handle.search does."""
        lib = load()
        keep = []
        arr = (frbx_scan * len(scans))()
        shapes = []
        for i, (h, vis) in enumerate(scans):
            vp, on_dev, k, shape = _vis_arg(vis)
            if not on_dev:
                raise ValueError("batched scans must be CUDA tensors")
            assert shape[2] == h.C, "cube does not match its setup"
            keep.append(k)
            arr[i].setup = h.h
            arr[i].vis_dev = vp
            arr[i].n_bl, arr[i].T = shape[0], shape[1]
            shapes.append(shape)
        dm = np.ascontiguousarray(dms, np.float64)
        win = np.ascontiguousarray(windows, np.int32)
        p, cm = scans[0][0]._params(threshold, nwin_min, sbd_win_ns, mbd_win_ns, combos, kernel)
        caps_l = [_default_caps(caps, want_events, want_pre_merge) for _ in scans]
        for attempt in range(2):
            res = (frbx_results * len(scans))()
            bufs_l, ser_l = [], []
            for i, (n_bl, T, _) in enumerate(shapes):
                bufs, r = _result_buffers(caps_l[i])
                ser = None
                if want_series:
                    _, S_tot = frbx_series_layout(T, win)
                    n = n_bl * len(dm) * S_tot
                    ser = (np.zeros(n, SEG_DTYPE), np.zeros(n, np.float32), S_tot)
                    r.series = ser[0].ctypes.data_as(c_vp)
                    r.pnorm = ser[1].ctypes.data_as(c_vp)
                    r.series_cap = n
                res[i] = r
                bufs_l.append(bufs)
                ser_l.append(ser)
            rc = lib.frbx_search_batch(self.b, arr, len(scans), _ptr(dm, c_f64), len(dm), _ptr(win, c_i32), len(win),
                                       ctypes.byref(p), res, _stream_ptr(stream))
            if rc == FRBX_ETRUNC and attempt == 0:
                for i in range(len(scans)):
                    for k in bufs_l[i]:
                        if bufs_l[i][k].size:
                            caps_l[i][k] = max(caps_l[i][k], int(getattr(res[i], k + "_count")))
                continue
            if rc != FRBX_OK:
                raise FrbxError(rc, self.last_error())
            break
        outs = []
        for i, (n_bl, T, _) in enumerate(shapes):
            o = _collect(bufs_l[i], res[i])
            if ser_l[i] is not None:
                S_tot = ser_l[i][2]
                o["S_tot"] = S_tot
                o["series"] = ser_l[i][0].reshape(n_bl, len(dm), S_tot)
                o["pnorm"] = ser_l[i][1].reshape(n_bl, len(dm), S_tot)
            outs.append(o)
        return outs


# ------------------------------------------------------------------ refinement (autograd)
def _dp(t):
    return ctypes.c_void_p(t.data_ptr())


def refine_power(handle, vis_dev, params, width, stream=None):
    """P [n_cand] (float32), G [n_cand][n_bl][2] and edge status for CUDA tensors
    params (float64 [n_cand][2 + 3 n_bl]) and width (int32 [n_cand])."""
    import torch
    n_bl, T, _ = vis_dev.shape
    n = params.shape[0]
    power = torch.empty(n, dtype=torch.float32, device=params.device)
    g = torch.empty((n, n_bl, 2), dtype=torch.float32, device=params.device)
    status = torch.empty(n, dtype=torch.int32, device=params.device)
    _check(handle.h, load().frbx_refine_power(handle.h, _dp(vis_dev), n_bl, T, _dp(params), _dp(width), n,
                                              _dp(power), _dp(g), _dp(status), _stream_ptr(stream)))
    return power, g, status


def refine_adjoint(handle, vis_dev, params, width, g, dpower, stream=None):
    import torch
    n_bl, T, _ = vis_dev.shape
    n = params.shape[0]
    dparams = torch.empty((n, 2 + 3 * n_bl), dtype=torch.float32, device=params.device)
    _check(handle.h, load().frbx_refine_adjoint(handle.h, _dp(vis_dev), n_bl, T, _dp(params), _dp(width), n,
                                                _dp(g), _dp(dpower.contiguous()), _dp(dparams), _stream_ptr(stream)))
    return dparams


def coherent_power_fn():
    """torch.autograd.Function whose forward is frbx_refine_power and whose backward is the
    hand-written adjoint kernel frbx_refine_adjoint (argument marshalling only)."""
    import torch

    class CoherentPower(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, handle, vis_dev, width):
            p = params.detach().contiguous()
            power, g, status = refine_power(handle, vis_dev, p, width)
            ctx.save_for_backward(p, g)
            ctx.handle, ctx.vis, ctx.width = handle, vis_dev, width
            ctx.status = status
            return power

        @staticmethod
        def backward(ctx, dpower):
            p, g = ctx.saved_tensors
            dparams = refine_adjoint(ctx.handle, ctx.vis, p, ctx.width, g, dpower.float())
            return dparams.to(p.dtype), None, None, None

    return CoherentPower
