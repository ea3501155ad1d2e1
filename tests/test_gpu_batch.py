"""Batched search (frbx_search_batch): many scans of uneven length on several setups in one
persistent, graph-captured fit.  Every scan must come out exactly as frbx_search gives it
(same kernels, same arithmetic, only the work order differs), and a small batch is checked
against the FP64 oracle directly."""
import numpy as np
import pytest

import synth
from oracle import reference as R
from tests.test_gpu_parity import compare_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frbx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_02391_gb300 import _build
    _build.build()
    from paper_1801_02391_gb300 import frbx as f
    f.load()
    return f


def to_dev(vis):
    import torch
    return torch.from_numpy(np.ascontiguousarray(vis)).cuda()


DMS = np.linspace(0.0, 600.0, 13)


def _scans():
    """Small-like (8 x 32 points, 4 windows) and VGOS-like (32 x 64 points, flags) scans of
    uneven length and baseline count, interleaved."""
    small = [synth.make_small(T=1500, dms=DMS), synth.make_small(T=1111, n_bl=2, dms=DMS, seed_offset=3)]
    vg = []
    for T, n_bl, off in ((700, 2, 0), (333, 2, 5)):
        wl = synth.make_vgos(T=T, n_bl=n_bl, n_dm=len(DMS), seed_offset=off)
        wl.dms = DMS.copy()
        for p in wl.pulses:
            p.t0_bin = int(p.t0_bin % max(1, T - 200) + 20)
        if vg:  # one VGOS setup: the second scan takes the first one's flags
            wl.flags = vg[0].flags.copy()
            wl.rfi_points = list(vg[0].rfi_points)
        vg.append(wl)
    return [small[0], vg[0], small[1], vg[1]]


def _same(a, b):
    assert np.array_equal(a["series"], b["series"])
    assert np.array_equal(a["pnorm"], b["pnorm"])
    for k in ("pulses", "groups", "combined", "pulses_dm", "events"):
        if a[k] is None:
            assert b[k] is None
        else:
            assert np.array_equal(a[k], b[k]), k
    assert a["counts"] == b["counts"]


@pytest.mark.parametrize("kernel", [0, 1])
def test_batch_equals_per_scan_search(frbx, kernel):
    """kernel 0: the VGOS-like scans take the window-tree fit, the small ones the per-segment
    direct fit, in one captured graph; kernel 1: the persistent per-segment fit everywhere."""
    wls = _scans()
    windows = [1, 2, 4, 8]
    hs = {}
    for wl in wls:  # one handle per setup, shared by its scans
        hs.setdefault(wl.name, frbx.Handle.from_workload(wl))
    vis = [to_dev(synth.generate(wl)) for wl in wls]
    scans = [(hs[wl.name], v) for wl, v in zip(wls, vis)]
    kw = dict(combos=[0b1, 0b11], want_series=True, want_events=True, want_pre_merge=True, kernel=kernel)
    with frbx.Batch() as b:
        out = b.search(scans, DMS, windows, **kw)
        info = b.info()
        assert info["graph_captures"] == 1 and info["graph_replays"] == 0
        # per-segment tiles 32 / 64 / 128, window-tree tiles 512 / 1024 / 2048, each measured
        assert len(info["time_tile"]) == 2 and all(t in (32, 64, 128, 512, 1024, 2048) for t in info["time_tile"])
        assert info["fit_ms"] > 0 and info["launches"] >= 2 + 4 * 2
        # the same shapes in the same buffers: the fit graph is replayed, results unchanged
        again = b.search(scans, DMS, windows, **kw)
        info = b.info()
        assert info["graph_captures"] == 1 and info["graph_replays"] == 1
        for o, o2 in zip(out, again):
            _same(o, o2)
        # new data in the same buffers: replayed, and the results follow the data
        vis[1].mul_(2.0)
        out2 = b.search(scans, DMS, windows, **kw)
        info = b.info()
        assert info["graph_captures"] == 1 and info["graph_replays"] == 2
        ok = out[1]["series"]["amp"] >= 0
        np.testing.assert_allclose(out2[1]["series"]["amp"][ok], 2.0 * out[1]["series"]["amp"][ok], rtol=1e-6)
        _same(out2[0], out[0])
        # another DM grid changes the work: re-captured
        b.search(scans, DMS[:7], windows, **kw)
        assert b.info()["graph_captures"] == 2
    # every scan exactly as frbx_search gives it (same kernels, same arithmetic)
    for (h, v), o in zip(scans, out2):
        _same(o, h.search(v, DMS, windows, **kw))


@pytest.mark.parametrize("kernel,sbd,mbd", [(4, None, None), (6, None, None), (6, (-64.0, 64.0), None),
                                            (6, (40.0, 300.0), (10.0, 12.5)), (4, (40.0, 300.0), (10.0, 12.5))])
def test_batch_window_tree_only(frbx, kernel, sbd, mbd):
    """Window-tree kernels (4: CUDA cores, 6: tensor cores) on VGOS-like scans of three
    lengths, one spanning several time tiles, against frbx_search with the same kernel, on the
    whole grid and with delay search windows; replay with new data."""
    wls = []
    for T, off in ((2300, 0), (700, 5), (1200, 9)):
        wl = synth.make_vgos(T=T, n_bl=2, n_dm=len(DMS), seed_offset=off)
        wl.dms = DMS.copy()
        if wls:
            wl.flags = wls[0].flags.copy()
            wl.rfi_points = list(wls[0].rfi_points)
        wls.append(wl)
    h = frbx.Handle.from_workload(wls[0])
    vis = [to_dev(synth.generate(wl)) for wl in wls]
    kw = dict(combos=[0b11], want_series=True, want_events=True, kernel=kernel, sbd_win_ns=sbd, mbd_win_ns=mbd)
    with frbx.Batch() as b:
        out = b.search([(h, v) for v in vis], DMS, [1, 2, 4, 8, 16], **kw)
        vis[0].mul_(0.5)  # same buffers, new data: the captured graph is replayed
        out2 = b.search([(h, v) for v in vis], DMS, [1, 2, 4, 8, 16], **kw)
        assert b.info()["graph_captures"] == 1 and b.info()["graph_replays"] == 1
        assert b.info()["time_tile"][0] in (512, 1024, 2048)  # measured; the results do not depend on it
        ok = out[0]["series"]["amp"] >= 0
        np.testing.assert_allclose(out2[0]["series"]["amp"][ok], 0.5 * out[0]["series"]["amp"][ok], rtol=1e-6)
        _same(out2[1], out[1])
        for v, o in zip(vis, out2):
            _same(o, h.search(v, DMS, [1, 2, 4, 8, 16], **kw))


def test_batch_against_oracle(frbx):
    """Two tiny scans of different length and one small scan through the batch, each compared
    with the FP64 oracle's search element by element."""
    t0 = synth.make_tiny(T=150, n_bl=2, dms=(0.0, 150.0, 400.0))
    # the two tiny scans share one setup: same channel grid, other data
    wls = [t0, synth.make_tiny(T=97, n_bl=2, dms=(0.0, 150.0, 400.0), seed_offset=2, f0=t0.f0_mhz),
           synth.make_small(T=700, dms=(0.0, 150.0, 400.0))]
    windows = [1, 2, 4]
    dms = np.array([0.0, 150.0, 400.0])
    for wl in wls:
        wl.windows = windows
        wl.dms = dms
    h_tiny = frbx.Handle.from_workload(wls[0])
    h_small = frbx.Handle.from_workload(wls[2])
    vis = [synth.generate(wl) for wl in wls]
    with frbx.Batch() as b:
        out = b.search([(h_tiny, to_dev(vis[0])), (h_tiny, to_dev(vis[1])), (h_small, to_dev(vis[2]))], dms,
                       windows, combos=[3], want_series=True, want_events=True, want_pre_merge=True)
    for wl, v, o in zip(wls, vis, out):
        st = R.setup_from_workload(wl)
        res_o = R.search(st, v, dms, windows, combos=[3])
        compare_search(frbx, wl, st, v, res_o, o, [3])


def test_batch_edge_cases_and_errors(frbx):
    wl = synth.make_tiny(T=60, pulse=False)
    h = frbx.Handle.from_workload(wl)
    v = to_dev(synth.generate(wl))
    short = synth.make_tiny(T=3, pulse=False)  # shorter than every window: empty series
    vs = to_dev(synth.generate(short))
    with frbx.Batch() as b:
        out = b.search([(h, v), (h, vs)], wl.dms, [4, 8], want_series=True)
        ref = h.search(v, wl.dms, [4, 8], want_series=True)
        _same(out[0], ref)
        assert out[1]["S_tot"] == 0 and out[1]["pulses"].size == 0
        for kw in (dict(windows=[2, 2]), dict(windows=[0]), dict(dms=[-1.0]), dict(combos=[1 << 5]),
                   dict(kernel=3)):
            args = dict(dms=wl.dms, windows=[1, 2])
            args.update(kw)
            with pytest.raises(frbx.FrbxError) as e:
                b.search([(h, v)], args.pop("dms"), args.pop("windows"), **args)
            assert e.value.code == frbx.FRBX_EINVAL
        # a combination mask naming a baseline that one scan lacks is refused
        one = synth.make_tiny(T=60, n_bl=1, pulse=False)
        with pytest.raises(frbx.FrbxError) as e:
            b.search([(h, v), (h, to_dev(synth.generate(one)))], wl.dms, [1, 2], combos=[3])
        assert e.value.code == frbx.FRBX_EINVAL and "scan 1" in b.last_error()


def test_batch_truncation_retries(frbx):
    wl = synth.make_small(T=900, dms=np.arange(540.0, 581.0, 10.0))
    h = frbx.Handle.from_workload(wl)
    v = to_dev(synth.generate(wl))
    full = h.search(v, wl.dms, wl.windows, want_events=True)
    with frbx.Batch() as b:
        out = b.search([(h, v), (h, v)], wl.dms, wl.windows, want_events=True, caps={"events": 2})
    for o in out:
        assert o["counts"]["events"] == full["counts"]["events"]
        assert np.array_equal(o["events"], full["events"])
