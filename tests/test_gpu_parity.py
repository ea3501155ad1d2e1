"""CUDA path (libfrbx through the C ABI) against the FP64 oracle, on the same seeded inputs."""
import numpy as np
import pytest

import synth
from oracle import reference as R
from paper_1801_02391_gb300 import _build
from tests.gpu_helpers import AMP_RTOL, assert_fit_match, p_band

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


def to_dev(vis):
    import torch
    return torch.from_numpy(np.ascontiguousarray(vis)).cuda()


def valid_segments(rng, wl, dk_max, n, windows=None):
    windows = windows or wl.windows
    rows = []
    for _ in range(20 * n):
        b = int(rng.integers(0, wl.n_bl))
        d = int(rng.integers(0, len(wl.dms)))
        l = int(windows[rng.integers(0, len(windows))])
        nv = R.n_valid(wl.T, l, int(dk_max[d]))
        if nv <= 0:
            continue
        rows.append((b, d, l, int(rng.integers(0, nv)) * R.window_step(l)))
        if len(rows) == n:
            break
    return np.array(rows, np.int32)


# ------------------------------------------------------------------ Eq. 1-2
@pytest.mark.parametrize("maker", ["small", "vgos", "tiny"])
def test_shift_table_bit_exact(frbx, maker):
    wl = {"small": lambda: synth.make_small(T=64), "vgos": lambda: synth.make_vgos(T=64, n_bl=1),
          "tiny": lambda: synth.make_tiny(dms=np.linspace(0, 3000, 37))}[maker]()
    st = R.setup_from_workload(wl)
    h = frbx.Handle.from_workload(wl)
    np.testing.assert_array_equal(h.shift_table(wl.dms), R.shift_table(st, wl.dms))
    assert (h.Ls, h.Lm) == (st.Ls, st.Lm) and h.df_grid_mhz == st.df_grid_mhz
    np.testing.assert_array_equal(h.g, st.g)


# ------------------------------------------------------------------ Eq. 3 + Eq. 5 + Sec. 5.1
def _fit_case(frbx, wl, kernel, n=300, seed=0, sbd=None, mbd=None, handle_kw=None, setup_kw=None):
    st = R.setup_from_workload(wl, **(setup_kw or {}))
    vis = synth.generate(wl)
    dk = R.shift_table(st, wl.dms)
    segs = valid_segments(np.random.default_rng(seed), wl, dk.max(axis=1), n)
    assert segs.shape[0] == n
    h = frbx.Handle.from_workload(wl, **(handle_kw or {}))
    gpu = h.fit_segments(to_dev(vis), wl.dms, segs, kernel=kernel, sbd_win_ns=sbd, mbd_win_ns=mbd)
    am, aq = R.window_masks(st, sbd, mbd)
    ref = R.fit_segments(st, vis, dk, segs, am, aq)
    return assert_fit_match(st, vis, dk, segs, gpu, ref, (am, aq))


def test_fit_small_setup_direct(frbx):
    wl = synth.make_small(T=700, dms=[0.0, 250.0, 557.0, 560.0])
    _fit_case(frbx, wl, kernel=1, n=400)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_vgos_setup(frbx, kernel):
    wl = synth.make_vgos(T=300, n_bl=2)
    wl.dms = np.array([0.0, 40.0, 100.0, 150.0])
    _fit_case(frbx, wl, kernel=kernel, n=120 if kernel == 1 else 400)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_uneven_channel_grid(frbx, kernel):
    """16 channels on an uneven grid (g up to ~40, Lm = 128), several CTA tiles + ragged tail."""
    wl = synth.make_tiny(n_chan=16, n_point=32, T=200, n_bl=3, dms=(0.0, 60.0, 200.0), windows=(1, 2, 4, 8),
                         f0=800.0 + 16.0 * np.array([0, 1, 3, 4, 7, 9, 12, 13, 17, 20, 22, 27, 30, 33, 38, 40]))
    _fit_case(frbx, wl, kernel=kernel, n=333, seed=1)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_short_channels_padded_fft(frbx, kernel):
    """J = 16 < 32 points per channel: the FFT kernel zero-pads the SBD inner sum."""
    wl = synth.make_tiny(n_chan=5, n_point=16, T=150, n_bl=2, dms=(0.0, 90.0), windows=(1, 3, 6),
                         f0=900.0 + 8.0 * np.array([0, 2, 5, 6, 11]), f_bw=8.0)
    _fit_case(frbx, wl, kernel=kernel, n=150, seed=2)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_crowded_residue_classes(frbx, kernel):
    """Channels whose MBD grid indices collide modulo 32 (g = 0, 32, 64, 96 share a class):
    the FFT kernel's inner sum over up to four channels per class."""
    wl = synth.make_tiny(n_chan=7, n_point=32, T=120, n_bl=2, dms=(0.0, 50.0), windows=(1, 2, 4),
                         f0=500.0 + 4.0 * np.array([0, 32, 64, 96, 1, 33, 70]), f_bw=4.0)
    _fit_case(frbx, wl, kernel=kernel, n=120, seed=4)


def test_fit_tiny_irregular_direct(frbx):
    wl = synth.make_tiny(seed_offset=3)
    _fit_case(frbx, wl, kernel=0, n=100, seed=3)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_calibration_and_flags(frbx, kernel):
    """Channel delays / initial phases of Eq. 5 and flagged points."""
    wl = synth.make_vgos(T=120, n_bl=1)
    wl.dms = np.array([0.0, 30.0])
    rng = np.random.default_rng(9)
    cal = dict(chan_delay_ns=rng.uniform(-5, 5, wl.n_chan), chan_phase_rad=rng.uniform(-3, 3, wl.n_chan))
    _fit_case(frbx, wl, kernel=kernel, n=80, handle_kw=cal, setup_kw=cal)


@pytest.mark.parametrize("kernel", [1, 2])
def test_fit_delay_windows(frbx, kernel):
    wl = synth.make_vgos(T=120, n_bl=1)
    wl.dms = np.array([0.0, 30.0])
    _fit_case(frbx, wl, kernel=kernel, n=80, sbd=(-64.0, 64.0), mbd=(-5.0, 10.0))


def test_fft_kernel_rejects_small_mbd_grid(frbx):
    wl = synth.make_small(T=64, dms=[0.0])
    h = frbx.Handle.from_workload(wl)
    with pytest.raises(frbx.FrbxError) as e:
        h.fit_segments(to_dev(synth.generate(wl)), wl.dms, np.array([[0, 0, 2, 0]], np.int32), kernel=2)
    assert e.value.code == frbx.FRBX_EUNSUPPORTED


def test_fit_rejects_out_of_range_rows(frbx):
    wl = synth.make_small(T=64, dms=[0.0, 100.0])
    h = frbx.Handle.from_workload(wl)
    vis = to_dev(synth.generate(wl))
    for row in ([0, 1, 4, 60], [3, 0, 2, 0], [0, 2, 2, 0], [0, 0, 0, 0], [0, 0, 2, -1]):
        with pytest.raises(frbx.FrbxError) as e:
            h.fit_segments(vis, wl.dms, np.array([row], np.int32))
        assert e.value.code == frbx.FRBX_EINVAL


# ------------------------------------------------------------------ whole search
def _series_rows(T, windows, dk_max, n_bl):
    segs, idx, S_tot = R.all_segments(T, n_bl, windows, dk_max)
    return segs, idx, S_tot


def compare_search(frbx, wl, st, vis, res_o, out, combos):
    n_bl, n_dm = wl.n_bl, len(wl.dms)
    S_tot = out["S_tot"]
    assert S_tot == res_o.S_tot
    ser = out["series"]
    # segment fits: valid slots agree, amplitudes / cells per the tie rule
    valid_o = ~np.isnan(res_o.amp)
    assert np.array_equal(ser["amp"] >= 0, valid_o)
    dk = res_o.dk
    segs, idx, _ = _series_rows(wl.T, wl.windows, res_o.dk_max, n_bl)
    flat = ser.reshape(-1)[idx]
    ref = (res_o.amp.reshape(-1)[idx], res_o.m.reshape(-1)[idx], res_o.q.reshape(-1)[idx], res_o.amp2.reshape(-1)[idx])
    n_tie = assert_fit_match(st, vis, dk, segs, flat, ref)
    # normalised power
    offs, _ = R.slot_offsets(wl.T, wl.windows)
    Po = res_o.P
    mean_over_std = np.zeros_like(Po)
    for d in range(n_dm):
        for w, l in enumerate(wl.windows):
            nv = R.n_valid(wl.T, l, int(res_o.dk_max[d]))
            if nv:
                a = res_o.amp[:, d, offs[w]:offs[w] + nv]
                mean_over_std[:, d, offs[w]:offs[w] + nv] = (a.mean(axis=1) / a.std(axis=1))[:, None]
    band = p_band(np.nan_to_num(Po), mean_over_std)
    Pg = out["pnorm"]
    assert np.all(np.abs(Pg[valid_o] - Po[valid_o]) <= band[valid_o])
    # threshold crossings (the baselines' come first)
    ev = out["events"]
    gb = ev[:out["counts"]["events_baseline"]]
    okeys = {(s, d, c.w, c.k0): c for (s, d), lst in res_o.events.items() for c in lst}
    gb_keys = {(int(e["series"]), int(e["dm_idx"]), int(e["win_idx"]), int(e["k0"])) for e in gb}
    assert len(gb_keys) == len(gb)
    flips = gb_keys ^ set(okeys)
    for k in flips:
        s, d, w, k0 = k
        j = offs[w] + k0 // R.window_step(wl.windows[w])
        assert abs(Po[s, d, j] - 3.0) <= band[s, d, j], f"event {k} differs away from the threshold"
    for e in gb:
        k = (int(e["series"]), int(e["dm_idx"]), int(e["win_idx"]), int(e["k0"]))
        if k in okeys:
            c = okeys[k]
            assert (int(e["sbd_idx"]), int(e["mbd_idx"])) == (c.m, c.q) or n_tie
            assert abs(e["amp"] - c.amp) <= AMP_RTOL * c.amp
    n_b = len(okeys)
    affected = {(s, d) for (s, d, w, k0) in flips}
    # pulses before and after the DM merge, cross-match groups
    pre = out["pulses_dm"]
    o_pre = [p for b in range(n_bl) for d in range(n_dm) for p in res_o.pulses_dm[(b, d)] if (b, d) not in affected]
    g_pre = [p for p in pre if (int(p["series"]), int(p["dm_idx"])) not in affected]
    assert [(int(p["series"]), int(p["dm_idx"]), int(p["win_idx"]), int(p["k0"]), int(p["n_win"])) for p in g_pre] == \
        [(p.series, p.d, p.w, p.k0, p.n_win) for p in o_pre]
    if not affected:
        o_m = [p for b in range(n_bl) for p in res_o.pulses[b]]
        g_m = out["pulses"]
        assert [(int(p["series"]), int(p["dm_idx"]), int(p["win_idx"]), int(p["k0"]), int(p["n_win"]), int(p["group"]))
                for p in g_m] == [(p.series, p.d, p.w, p.k0, p.n_win, p.group) for p in o_m]
        np.testing.assert_allclose(g_m["pnorm"], [p.p for p in o_m], atol=1e-3)
        np.testing.assert_allclose(g_m["dm"], [wl.dms[p.d] for p in o_m])
        np.testing.assert_allclose(g_m["t_s"], [p.k0 * wl.t_ap_ms * 1e-3 for p in o_m])
        sbd_ax, mbd_ax = R.delay_axes(st)
        np.testing.assert_allclose(g_m["sbd_ns"], [sbd_ax[p.m] for p in o_m])
        np.testing.assert_allclose(g_m["mbd_ns"], [mbd_ax[p.q] for p in o_m])
        grp = out["groups"]
        assert [(int(g["bl_mask"]), int(g["n_baselines"]), int(g["n_pulses"])) for g in grp] == \
            [(g["mask"], g["n_baselines"], len(g["members"])) for g in res_o.groups]
    # power summation scheme
    if combos:
        o_c = [p for ci in range(len(combos)) for p in res_o.combined[ci]]
        g_c = out["combined"]
        assert [(int(p["series"]), int(p["dm_idx"]), int(p["win_idx"]), int(p["k0"]), int(p["n_win"])) for p in g_c] == \
            [(p.series, p.d, p.w, p.k0, p.n_win) for p in o_c]
        np.testing.assert_allclose(g_c["amp"], [p.amp for p in o_c], rtol=AMP_RTOL)
    return dict(ties=n_tie, flips=len(flips), events=n_b)


def test_search_small_workload_full_size(frbx):
    """The small workload at full size (3 baselines x 101 DMs x 4096 APs x 256 points):
    every segment, P value, crossing, pulse, group and combined pulse against the oracle."""
    wl = synth.make_small()
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    combos = [0b111, 0b011, 0b101, 0b110]
    res_o = R.search(st, vis, wl.dms, wl.windows, combos=combos)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, combos=combos, want_series=True, want_events=True,
                   want_pre_merge=True)
    stats = compare_search(frbx, wl, st, vis, res_o, out, combos)
    assert stats["events"] > 1000
    # the injected pulse is found on all three baselines at DM 560
    best = [max((p for p in out["pulses"] if p["series"] == b), key=lambda p: p["pnorm"]) for b in range(3)]
    assert all(wl.dms[p["dm_idx"]] == 560.0 for p in best)
    assert len({int(p["group"]) for p in best}) == 1


def test_search_host_and_device_input_agree(frbx):
    wl = synth.make_small(T=900, dms=np.arange(500.0, 601.0, 20.0))
    vis = synth.generate(wl)
    h = frbx.Handle.from_workload(wl)
    a = h.search(vis, wl.dms, wl.windows, combos=[7], want_series=True)
    b = h.search(to_dev(vis), wl.dms, wl.windows, combos=[7], want_series=True)
    assert np.array_equal(a["series"], b["series"]) and np.array_equal(a["pulses"], b["pulses"])
    assert a["launches"] >= 6


@pytest.mark.parametrize("kernel", [1, 2])
def test_search_vgos_reduced(frbx, kernel):
    """VGOS-like setup (4 bands x 8 x 64 points, flags, 6 windows) at reduced T / DM count:
    the whole search element by element with both fit kernels."""
    wl = synth.make_vgos(T=1500, n_bl=3, n_dm=6)
    wl.dms = np.array([0.0, 100.0, 400.0, 900.0, 1200.0, 1700.0])
    for p in wl.pulses:
        p.t0_bin = int(p.t0_bin % 200 + 50)
        p.dm = float(wl.dms[2])
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    combos = [0b111, 0b011]
    res_o = R.search(st, vis, wl.dms, wl.windows, combos=combos)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, combos=combos, want_series=True, want_events=True,
                   want_pre_merge=True, kernel=kernel)
    compare_search(frbx, wl, st, vis, res_o, out, combos)


def test_search_edge_cases(frbx):
    # scan shorter than every window: nothing to fit, empty outputs
    wl = synth.make_tiny(T=3, windows=(4, 8), pulse=False)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(synth.generate(wl)), wl.dms, wl.windows, want_series=True, combos=[3])
    assert out["S_tot"] == 0 and out["pulses"].size == 0 and out["combined"].size == 0
    # every DM sweeps past the scan: series exist but no valid segment
    wl = synth.make_tiny(T=40, dms=(5000.0, 9000.0), windows=(1, 2), pulse=False)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(synth.generate(wl)), wl.dms, wl.windows, want_series=True)
    assert out["S_tot"] > 0 and np.all(out["series"]["amp"] == -1.0) and out["counts"]["events"] == 0
    # one baseline, one DM, one window of length 1
    wl = synth.make_tiny(T=50, n_bl=1, dms=(0.0,), windows=(1,))
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, want_series=True, want_events=True, want_pre_merge=True,
                   nwin_min=1)
    res_o = R.search(st, vis, wl.dms, wl.windows, nwin_min=1)
    compare_search(frbx, wl, st, vis, res_o, out, [])


def test_search_rejects_bad_arguments(frbx):
    wl = synth.make_tiny(T=40)
    h = frbx.Handle.from_workload(wl)
    vis = to_dev(synth.generate(wl))
    for kw in (dict(windows=[2, 2]), dict(windows=[0]), dict(dms=[-1.0]), dict(combos=[1 << 5]),
               dict(sbd_win_ns=(1e6, 2e6)), dict(windows=list(range(1, 18)))):
        args = dict(dms=wl.dms, windows=wl.windows)
        args.update(kw)
        with pytest.raises(frbx.FrbxError) as e:
            h.search(vis, args.pop("dms"), args.pop("windows"), **args)
        assert e.value.code == frbx.FRBX_EINVAL
    # a cube pointer that is not 8-byte aligned is refused before any launch
    import ctypes
    import torch
    from paper_1801_02391_gb300.frbx import _ptr, c_f64, c_i32, frbx_default_params, frbx_results, load
    raw = torch.zeros(vis.numel() * 2 + 2, dtype=torch.float32, device="cuda")
    dm = np.ascontiguousarray(wl.dms)
    win = np.ascontiguousarray(wl.windows, np.int32)
    r, p = frbx_results(), frbx_default_params()
    rc = load().frbx_search(h.h, ctypes.c_void_p(raw.data_ptr() + 4), 1, wl.n_bl, wl.T, _ptr(dm, c_f64), len(dm),
                            _ptr(win, c_i32), len(win), ctypes.byref(p), ctypes.byref(r), None)
    assert rc == frbx.FRBX_EINVAL and "aligned" in h.last_error()


def test_search_truncation_reports_sizes(frbx):
    wl = synth.make_small(T=900, dms=np.arange(540.0, 581.0, 10.0))
    vis = to_dev(synth.generate(wl))
    h = frbx.Handle.from_workload(wl)
    full = h.search(vis, wl.dms, wl.windows, want_events=True)
    n = full["counts"]["events"]
    assert n > 2
    small = h.search(vis, wl.dms, wl.windows, want_events=True, caps={"events": 2})
    assert small["counts"]["events"] == n and np.array_equal(small["events"], full["events"])
