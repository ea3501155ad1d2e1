"""Window-tree fits: every window of a power-of-two set is built from one-AP delay-resolution
matrices by the additivity of Sec. 5.1, G_{k0,l} + G_{k0+l,l} = G_{k0,2l}.  Kernel 4 runs the
MBD transform on the CUDA cores in FP32; kernel 6 (the automatic choice where it applies)
runs it on the tensor cores as a three-term split-BF16 GEMM with FP32 accumulation (about
1e-5 relative).  Both are compared with the FP64 oracle element by element, to the FP32
tolerance, on several grid shapes (Lm/32 = 16, 8 and 1 MBD column classes, and Lm = 16), window sets with
and without gaps, more than one time tile, delay windows and scans that DM trials sweep past."""
import numpy as np
import pytest

import synth
from oracle import reference as R
from tests.gpu_helpers import assert_fit_match
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


def _vgos(T=1300, n_bl=2, dms=(0.0, 100.0, 400.0, 1700.0)):
    wl = synth.make_vgos(T=T, n_bl=n_bl, n_dm=len(dms))
    wl.dms = np.array(dms)
    for p in wl.pulses:
        p.t0_bin = int(p.t0_bin % 200 + 50)
        p.dm = float(wl.dms[min(2, len(dms) - 1)])
    return wl


def _run(frbx, wl, windows, combos=(3,), kernel=4, **kw):
    wl.windows = list(windows)
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    res_o = R.search(st, vis, wl.dms, wl.windows, combos=list(combos))
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, combos=list(combos), want_series=True, want_events=True,
                   want_pre_merge=True, kernel=kernel, **kw)
    compare_search(frbx, wl, st, vis, res_o, out, list(combos))
    return h, out


@pytest.mark.parametrize("kernel", [4, 6])
@pytest.mark.parametrize("windows", [[1, 2, 4, 8, 16, 32], [2, 4, 8, 16], [1, 4, 16], [8], [64, 1]])
def test_tree_search_matches_oracle(frbx, windows, kernel):
    # T = 1300 spans two time tiles of 1024 APs; DM 1700 leaves about 400 APs of valid sweep
    _run(frbx, _vgos(), windows, kernel=kernel)


def test_tree_is_the_automatic_choice(frbx):
    wl = _vgos(T=700, n_bl=2, dms=(0.0, 400.0))
    wl.windows = [1, 2, 4, 8]
    vis = to_dev(synth.generate(wl))
    h = frbx.Handle.from_workload(wl)
    auto = h.search(vis, wl.dms, wl.windows, want_series=True)
    assert h.stage_times()["tree_chunks"] > 0
    tc = h.search(vis, wl.dms, wl.windows, want_series=True, kernel=6)
    assert np.array_equal(auto["series"], tc["series"])
    seg = h.search(vis, wl.dms, wl.windows, want_series=True, kernel=2)
    ok = seg["series"]["amp"] >= 0
    for k in (4, 6):
        tree = h.search(vis, wl.dms, wl.windows, want_series=True, kernel=k)
        assert np.array_equal(ok, tree["series"]["amp"] >= 0)
        rel = np.abs(tree["series"]["amp"][ok] - seg["series"]["amp"][ok]) / seg["series"]["amp"][ok]
        print(f"kernel {k} vs per-segment FFT: max rel {rel.max():.2e}, median {np.median(rel):.2e}")
        assert rel.max() <= 1e-4


def test_tree_two_band_grid(frbx):
    """Two VGOS bands (16 x 64 points): Lm = 256, eight SBD rows per block."""
    wl = synth._batch_setup("c1024", 41, 1100, 2, [0.0, 300.0, 900.0])
    wl.tau_g_ns = np.array([12.0, 31.0])
    wl.rate_mhz = np.array([1.0, -2.0])
    wl.phase0 = np.array([0.3, 2.0])
    wl.pulses = [synth.Pulse(dm=300.0, t0_bin=200, width=3, snr=25.0)]
    _run(frbx, wl, [2, 4, 8, 16], combos=(3, 1))
    _run(frbx, wl, [2, 4, 8, 16], combos=(3, 1), kernel=6)


def test_tree_single_column_class_grid(frbx):
    """4 channels x 32 points with channel offsets {0, 3, 7, 12} x 16 MHz: Lm = 32, so one MBD
    column class and all 64 SBD rows in one block."""
    wl = synth.make_tiny(n_chan=4, n_point=32, T=400, n_bl=2, dms=(0.0, 50.0, 200.0), windows=(1, 2, 4, 8),
                         f0=800.0 + 16.0 * np.array([0, 3, 7, 12]))
    h, _ = _run(frbx, wl, [1, 2, 4, 8])
    assert (h.Ls, h.Lm) == (64, 32)


@pytest.mark.parametrize("windows", [[2, 4, 8, 16], [1, 2, 4, 8, 16, 32, 64], [4]])
def test_tree_sixteen_cell_mbd(frbx, windows):
    """The S-band setup (8 channels x 32 points at 32 MHz spacing): Lm = 16, so one thread holds
    a whole SBD row (16 MBD cells, the even half of the 32-point structure) and 64 rows fill
    half a block.  The automatic choice is this tree; it matches the oracle element by element
    and agrees with the per-segment direct fit (kernel 1)."""
    wl = synth.make_small(T=1400, dms=np.arange(530.0, 591.0, 20.0))
    h, out = _run(frbx, wl, windows, combos=(7, 3))
    assert (h.Ls, h.Lm) == (64, 16)
    vis = to_dev(synth.generate(wl))
    auto = h.search(vis, wl.dms, windows, want_series=True)
    assert h.stage_times()["tree_chunks"] > 0 and h.stage_times()["tree_tensor"] == 0
    assert np.array_equal(auto["series"], out["series"])
    seg = h.search(vis, wl.dms, windows, want_series=True, kernel=1)
    ok = seg["series"]["amp"] >= 0
    assert np.array_equal(ok, out["series"]["amp"] >= 0)
    rel = np.abs(out["series"]["amp"][ok] - seg["series"]["amp"][ok]) / seg["series"]["amp"][ok]
    assert rel.max() <= 1e-4


@pytest.mark.parametrize("sbd,mbd", [(None, None), ((-100.0, 150.0), (-10.0, 12.0)), ((300.0, 900.0), (5.0, 20.0))])
def test_tree_sixteen_cell_mbd_full_block(frbx, sbd, mbd):
    """8 channels x 64 points: Ls = 128 and Lm = 16, every thread of the block a row; with and
    without SBD / MBD search windows (a window wrapping around zero delay and one that skips
    the first SBD rows)."""
    wl = synth.make_tiny(n_chan=8, n_point=64, T=900, n_bl=2, dms=(0.0, 20.0, 60.0), windows=(1, 2, 4, 8),
                         f0=1400.0 + 32.0 * np.arange(8))
    st = R.setup_from_workload(wl)
    assert (st.Ls, st.Lm) == (128, 16)
    vis = synth.generate(wl)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, want_series=True, kernel=4, sbd_win_ns=sbd, mbd_win_ns=mbd)
    dk = R.shift_table(st, wl.dms)
    segs, idx, _ = R.all_segments(wl.T, wl.n_bl, wl.windows, dk.max(axis=1))
    am, aq = R.window_masks(st, sbd, mbd)
    ref = R.fit_segments(st, vis, dk, segs, am, aq)
    flat = out["series"].reshape(-1)[idx]
    assert (flat["amp"] >= 0).all()
    assert_fit_match(st, vis, dk, segs, flat, ref, (am, aq))
    assert am[flat["sbd_idx"].astype(int)].all() and aq[flat["mbd_idx"].astype(int)].all()


@pytest.mark.parametrize("kernel", [4, 6])
@pytest.mark.parametrize("sbd,mbd", [((-100.0, 150.0), (-2.0, 3.0)), ((-64.0, 64.0), None),
                                     ((40.0, 300.0), (10.0, 12.5)), (None, (-1.0, 30.0))])
def test_tree_delay_windows(frbx, kernel, sbd, mbd):
    """SBD / MBD search windows: rows and cells outside them are excluded from the maximum.
    Kernel 4 skips blocks of SBD rows; kernel 6 rotates the SBD rows of its A tiles so the
    searched ones come first (windows wrapping around row 0 or not, starting off a multiple of
    8), masks cells of partly searched MBD column blocks and skips the others."""
    wl = _vgos(T=600, n_bl=2, dms=(0.0, 400.0))
    wl.windows = [1, 2, 4, 8]
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, want_series=True, kernel=kernel, sbd_win_ns=sbd, mbd_win_ns=mbd)
    assert h.stage_times()["tree_tensor"] == (1 if kernel == 6 else 0)
    dk = R.shift_table(st, wl.dms)
    segs, idx, _ = R.all_segments(wl.T, wl.n_bl, wl.windows, dk.max(axis=1))
    am, aq = R.window_masks(st, sbd, mbd)
    ref = R.fit_segments(st, vis, dk, segs, am, aq)
    flat = out["series"].reshape(-1)[idx]
    assert (flat["amp"] >= 0).all()
    assert_fit_match(st, vis, dk, segs, flat, ref, (am, aq))
    m = flat["sbd_idx"].astype(int)
    assert am[m].all() and aq[flat["mbd_idx"].astype(int)].all()


@pytest.mark.parametrize("sbd,pack", [((-64.0, 64.0), 4), ((-300.0, 400.0), 2), ((-600.0, 700.0), 1)])
def test_tree_packed_delay_windows(frbx, sbd, pack):
    """Delay windows whose searched SBD rows fit 32 (or 64) rotated tile rows: the SBD pass keeps
    those rows of each AP and one tensor-core CTA stacks the pieces of four (or two) time tiles.
    2600 APs make three time tiles of 1024 (the last one short and the fourth of the group
    empty); DM 1700 sweeps past the second.  A window of 83 rows takes the whole-tile form."""
    wl = _vgos(T=2600, n_bl=1, dms=(0.0, 1700.0))
    wl.windows = [1, 2, 4, 8, 16, 32]
    st = R.setup_from_workload(wl)
    am, aq = R.window_masks(st, sbd, None)
    m = np.flatnonzero(am)
    lo = int(m[0]) if not (am[0] and am[-1]) else int(np.flatnonzero(am == 0)[-1]) + 1
    nq = ((lo % 8) + int(am.sum()) + 31) // 32  # 32-row quarters holding the searched rows
    assert {1: 4, 2: 2}.get(nq, 1) == pack
    vis = synth.generate(wl)
    h = frbx.Handle.from_workload(wl)
    out = h.search(to_dev(vis), wl.dms, wl.windows, want_series=True, kernel=6, sbd_win_ns=sbd)
    assert h.stage_times()["tree_tensor"] == 1
    dk = R.shift_table(st, wl.dms)
    segs, idx, _ = R.all_segments(wl.T, wl.n_bl, wl.windows, dk.max(axis=1))
    ref = R.fit_segments(st, vis, dk, segs, am, aq)
    flat = out["series"].reshape(-1)[idx]
    assert (flat["amp"] >= 0).all()
    assert_fit_match(st, vis, dk, segs, flat, ref, (am, aq))
    assert am[flat["sbd_idx"].astype(int)].all()


def test_tree_scan_swept_past(frbx):
    """DM trials whose sweep exceeds the scan have no valid segment; the rest are fitted."""
    wl = _vgos(T=300, n_bl=1, dms=(0.0, 2000.0))
    h, out = _run(frbx, wl, [1, 2, 4], combos=(1,))
    assert np.all(out["series"]["amp"][0, 1] == -1.0) and np.all(out["series"]["amp"][0, 0] >= 0)


def test_tree_rejects_other_windows(frbx):
    wl = _vgos(T=300, n_bl=1, dms=(0.0,))
    h = frbx.Handle.from_workload(wl)
    for k in (4, 6):
        with pytest.raises(frbx.FrbxError) as e:
            h.search(to_dev(synth.generate(wl)), wl.dms, [3, 6], kernel=k)
        assert e.value.code == frbx.FRBX_EUNSUPPORTED
    # the automatic choice falls back to the per-segment fit for such windows
    out = h.search(to_dev(synth.generate(wl)), wl.dms, [3, 6], want_series=True)
    assert (out["series"]["amp"] >= 0).any()


@pytest.mark.parametrize("windows", [[1, 2, 4, 8, 16, 32, 64], [2, 8, 32]])
def test_tree_tensor_cores_two_k_atoms(frbx, windows):
    """64 contiguous channels x 64 points: K = 2N = 128, two 64-wide K atoms per MMA row and
    64 KB A tiles.  Windows up to 32 APs keep every anchor in tensor memory and a three-deep
    A ring; windows of 64 APs put the deepest anchor level in shared memory, which leaves
    room for a two-deep ring only."""
    wl = synth.make_tiny(n_chan=64, n_point=64, T=420, n_bl=1, dms=(0.0, 8.0), windows=windows,
                         f0=800.0 + 16.0 * np.arange(64))
    wl.pulses = [synth.Pulse(dm=8.0, t0_bin=150, width=4, snr=25.0)]
    h, _ = _run(frbx, wl, windows, combos=(1,), kernel=6)
    assert (h.Ls, h.Lm) == (128, 128)
    assert h.stage_times()["tree_tensor"] == 1


def test_tree_rejects_shapes_beyond_shared_memory(frbx):
    """64 channels x 256 points: Ls = 512 SBD rows, so one AP of SBD output (256 KB) exceeds
    shared memory.  The window trees refuse the shape up front (no failed launch), and so does
    the automatic choice, since no per-segment fit holds it either."""
    wl = synth.make_tiny(n_chan=64, n_point=256, T=40, n_bl=1, dms=(0.0,), windows=(1, 2),
                         f0=800.0 + 16.0 * np.arange(64), pulse=False)
    h = frbx.Handle.from_workload(wl)
    assert h.Ls == 512
    vis = to_dev(synth.generate(wl))
    for k in (4, 6):
        with pytest.raises(frbx.FrbxError) as e:
            h.search(vis, wl.dms, [1, 2], kernel=k)
        assert e.value.code == frbx.FRBX_EUNSUPPORTED
    with pytest.raises(frbx.FrbxError) as e:
        h.search(vis, wl.dms, [1, 2])
    assert e.value.code == frbx.FRBX_EUNSUPPORTED
