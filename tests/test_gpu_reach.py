"""Parity of the default path at full reach: the chunked window-tree fit across many chunks,
and the full VGOS-shaped search (15 baselines x 512 DM trials x 20000 APs x 2048 points),
against the FP64 oracle.

Every slot of a segment series must equal Eq. 5's maximum on the Sec. 5.1 grid for its
(baseline, DM, window, k0), whichever chunk, buffer set and time tile computed it.  The
window-tree fit splits the (baseline, DM) series into chunks that alternate between two
scratch sets on two streams (the SBD pass of chunk i + 2 reuses the set of chunk i once its
MBD pass is done), so these tests force many chunks (a small chunk budget through
frbx_set_limits) and, at full size, sample slots spread over all chunks, DM trials, windows
and both edges of the 1024-AP time tiles."""
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


def _vgos_cut(T=1300, n_bl=3, dms=(0.0, 100.0, 400.0, 900.0)):
    wl = synth.make_vgos(T=T, n_bl=n_bl, n_dm=len(dms))
    wl.dms = np.array(dms)
    for p in wl.pulses:
        p.t0_bin = int(p.t0_bin % 200 + 50)
        p.dm = float(wl.dms[2])
    wl.windows = [1, 2, 4, 8, 16, 32]
    return wl


@pytest.fixture(scope="module")
def cut_case():
    wl = _vgos_cut()
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    return wl, st, vis, R.search(st, vis, wl.dms, wl.windows, combos=[7])


@pytest.mark.parametrize("kernel", [4, 6])
@pytest.mark.parametrize("series_per_chunk", [1, 3])
def test_tree_many_chunks_matches_oracle(frbx, cut_case, kernel, series_per_chunk):
    """12 series in 12 or 4 chunks: both scratch sets reused several times, chunk edges inside
    a baseline, two time tiles per series; every slot, event and pulse against the oracle."""
    wl, st, vis, res_o = cut_case
    h = frbx.Handle.from_workload(wl)
    # bytes per series of one scratch set: the one-AP matrices of its T APs (32 KB per AP for
    # this setup in both the FP32 rows and the split tiles), plus a margin for the FP32 tree's
    # deep anchors (about 1 MB per series here)
    per_series = wl.T * h.Ls * wl.n_chan * 8 + (2 << 20)
    h.set_limits(tree_chunk_bytes=series_per_chunk * per_series)
    out = h.search(to_dev(vis), wl.dms, wl.windows, combos=[7], want_series=True, want_events=True,
                   want_pre_merge=True, kernel=kernel)
    n_ser = wl.n_bl * len(wl.dms)
    assert h.stage_times()["tree_chunks"] == -(-n_ser // series_per_chunk) >= 4
    compare_search(frbx, wl, st, vis, res_o, out, [7])
    # the same handle back on its default budget gives bit-identical series
    h.set_limits()
    one = h.search(to_dev(vis), wl.dms, wl.windows, combos=[7], want_series=True, kernel=kernel)
    assert h.stage_times()["tree_chunks"] == 1
    assert np.array_equal(one["series"], out["series"])


@pytest.mark.parametrize("kernel", [0, 4, 2])
def test_host_input_copy_overlaps_the_fit(frbx, cut_case, kernel):
    """Host input: the cube is copied one baseline after another beside the fit, and each chunk
    of the window tree waits only for the baselines it reads.  With one series per chunk, every
    chunk after the first runs while later baselines may still be in flight; the series, events
    and pulses must equal those of the same search on a device copy of the cube, for the tree
    (kernels 0, 4) and for a per-segment fit (kernel 2), which waits for the whole copy."""
    wl, st, vis, res_o = cut_case
    h = frbx.Handle.from_workload(wl)
    per_series = wl.T * h.Ls * wl.n_chan * 8 + (2 << 20)
    h.set_limits(tree_chunk_bytes=per_series)
    dev = h.search(to_dev(vis), wl.dms, wl.windows, combos=[7], want_series=True, want_events=True,
                   want_pre_merge=True, kernel=kernel)
    pinned = __import__("torch").from_numpy(np.ascontiguousarray(vis)).pin_memory()
    for host in (pinned, np.ascontiguousarray(vis)):  # pinned, then pageable host memory
        out = h.search(host, wl.dms, wl.windows, combos=[7], want_series=True, want_events=True,
                       want_pre_merge=True, kernel=kernel)
        if kernel != 2:
            assert h.stage_times()["tree_chunks"] == wl.n_bl * len(wl.dms)
        assert np.array_equal(out["series"], dev["series"])
        assert np.array_equal(out["events"], dev["events"])
        assert np.array_equal(out["pulses"], dev["pulses"])
        assert np.array_equal(out["pulses_dm"], dev["pulses_dm"])
    if kernel == 0:  # and the oracle agrees with all of it
        compare_search(frbx, wl, st, vis, res_o, dev, [7])


def _sample_slots(wl, dk_max, ser, n_series, rng, tile=1024):
    """Rows (bl, d, l, k0) and series slots spread over the ordered series list (the chunk
    order), every window, the first and last valid segments and both edges of each time tile."""
    offs, _ = R.slot_offsets(wl.T, wl.windows)
    picks = np.unique(np.linspace(0, len(ser) - 1, n_series).round().astype(int))
    rows, slots = [], []
    for i in picks:
        b, d = ser[i]
        for w, l in enumerate(wl.windows):
            step = R.window_step(l)
            nv = R.n_valid(wl.T, l, int(dk_max[d]))
            if nv <= 0:
                continue
            cand = {0, nv - 1}
            for t0 in range(tile, (nv - 1) * step + 1, tile):
                for k0 in (t0 - step, t0):
                    cand.add(k0 // step)
            cand.update(int(x) for x in rng.integers(0, nv, 2))
            for s in sorted(c for c in cand if 0 <= c < nv):
                rows.append((b, d, l, s * step))
                slots.append(((b * len(wl.dms) + d), int(offs[w]) + s))
    return np.array(rows, np.int32), slots


def test_full_vgos_search_sampled_slots_match_oracle(frbx):
    """The bench workload through frbx_search with the default kernel and chunk plan (hundreds
    of chunks): >= 2000 slots against the oracle's fit of the same segments, and every valid
    slot filled (amp >= 0), every invalid one empty."""
    import torch
    wl = synth.make_vgos()
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    dk = R.shift_table(st, wl.dms)
    dk_max = dk.max(axis=1)
    h = frbx.Handle.from_workload(wl)
    vis_dev = to_dev(vis)
    _, S_tot = R.slot_offsets(wl.T, wl.windows)
    n_el = wl.n_bl * len(wl.dms) * S_tot
    ser_dev = torch.empty(n_el * 2, dtype=torch.float32, device="cuda")  # frbx_seg: 8 bytes
    out = h.search(vis_dev, wl.dms, wl.windows, combos=[(1 << wl.n_bl) - 1], series_out=ser_dev)
    stages = h.stage_times()
    assert stages["tree_tensor"] == 1 and stages["tree_chunks"] >= 200, stages
    assert out["counts"]["pulses"] > 0
    amp = ser_dev.view(wl.n_bl * len(wl.dms), S_tot, 2)[:, :, 0]
    # valid slots: s < n_valid(T, l, dk_max[d]) in each window's block of the series
    offs, _ = R.slot_offsets(wl.T, wl.windows)
    ends = list(offs[1:]) + [S_tot]
    counts = torch.stack([(amp[:, int(o):int(e)] >= 0).sum(dim=1) for o, e in zip(offs, ends)], dim=1)
    expect = np.array([[R.n_valid(wl.T, l, int(x)) for l in wl.windows] for x in dk_max])
    np.testing.assert_array_equal(counts.cpu().numpy(), np.tile(expect, (wl.n_bl, 1)))
    # sampled slots against the oracle (series ordered baseline-major, as the chunk plan is)
    ser = [(b, d) for b in range(wl.n_bl) for d in range(len(wl.dms)) if wl.T - int(dk_max[d]) >= 1]
    rows, slots = _sample_slots(wl, dk_max, ser, 48, np.random.default_rng(20000))
    assert rows.shape[0] >= 2000, rows.shape
    raw = ser_dev.view(torch.int32).view(wl.n_bl * len(wl.dms), S_tot, 2)
    si = torch.tensor([s for s, _ in slots], device="cuda")
    ti = torch.tensor([t for _, t in slots], device="cuda")
    picked = raw[si, ti].cpu().numpy()
    gpu = np.zeros(len(slots), frbx.SEG_DTYPE)
    gpu["amp"] = picked[:, 0].view(np.float32)
    gpu["sbd_idx"] = (picked[:, 1].view(np.uint32) & 0xFFFF).astype(np.uint16)
    gpu["mbd_idx"] = (picked[:, 1].view(np.uint32) >> 16).astype(np.uint16)
    ref = R.fit_segments(st, vis, dk, rows)
    n_tie = assert_fit_match(st, vis, dk, rows, gpu, ref)
    print(f"full vgos: {rows.shape[0]} sampled slots over {len(np.unique(si.cpu().numpy()))} series, "
          f"{int(stages['tree_chunks'])} chunks, {n_tie} near-tie argmax differences")
    del vis_dev, ser_dev, raw, amp
    torch.cuda.empty_cache()
