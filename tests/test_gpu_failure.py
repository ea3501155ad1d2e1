"""Failure paths of the library, exercised without any GPU fault.

* Bounded waits: the tensor-core kernels (the window tree's k_tree_mma, the per-segment
  k_fit_mma) give up a pipeline wait after frbx_limits.wait_cycles.  With hold_producers the
  producer role issues nothing, so a consumer's wait runs out for certain: the call must return
  FRBX_ETIMEOUT (no fault, nothing left in flight), and the next call on the same handle, with
  the defaults back, must give the correct results.
* Allocation failure: a scratch cap below what a call needs makes the call return FRBX_ENOMEM
  before it launches anything that needs the memory; the handle stays usable.
* A short but sufficient wait limit changes nothing in the results.
"""
import numpy as np
import pytest

import synth
from oracle import reference as R
from tests.gpu_helpers import assert_fit_match

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


@pytest.fixture(scope="module")
def vgos_case():
    wl = synth.make_vgos(T=700, n_bl=2, n_dm=3)
    wl.dms = np.array([0.0, 150.0, 400.0])
    wl.windows = [1, 2, 4, 8]
    for p in wl.pulses:
        p.t0_bin = int(p.t0_bin % 200 + 50)
        p.dm = 150.0
    return wl, synth.generate(wl)


def test_tree_tensor_core_wait_runs_out_then_recovers(frbx, vgos_case):
    wl, vis = vgos_case
    vis_dev = to_dev(vis)
    h = frbx.Handle.from_workload(wl)
    ref = h.search(vis_dev, wl.dms, wl.windows, want_series=True, kernel=6)
    h.set_limits(wait_cycles=2_000_000, hold_producers=1)  # about 1 ms per wait
    with pytest.raises(frbx.FrbxError) as ei:
        h.search(vis_dev, wl.dms, wl.windows, want_series=True, kernel=6)
    assert ei.value.code == frbx.FRBX_ETIMEOUT
    assert "bounded wait" in h.last_error()
    h.set_limits()
    again = h.search(vis_dev, wl.dms, wl.windows, want_series=True, kernel=6)
    assert np.array_equal(again["series"], ref["series"])
    assert [tuple(p) for p in again["pulses"]] == [tuple(p) for p in ref["pulses"]]


def test_segment_tensor_core_wait_runs_out_then_recovers(frbx):
    wl = synth.make_small(T=400, dms=[0.0, 300.0, 557.0])
    vis = synth.generate(wl)
    vis_dev = to_dev(vis)
    st = R.setup_from_workload(wl)
    dk = R.shift_table(st, wl.dms)
    rng = np.random.default_rng(5)
    rows = []
    while len(rows) < 200:
        d = int(rng.integers(0, 3))
        l = int(rng.choice(wl.windows))
        nv = R.n_valid(wl.T, l, int(dk[d].max()))
        if nv > 0:
            rows.append((int(rng.integers(0, wl.n_bl)), d, l, int(rng.integers(0, nv)) * R.window_step(l)))
    rows = np.array(rows, np.int32)
    h = frbx.Handle.from_workload(wl)
    for k in (3, 5):
        h.set_limits(wait_cycles=2_000_000, hold_producers=1)
        with pytest.raises(frbx.FrbxError) as ei:
            h.fit_segments(vis_dev, wl.dms, rows, kernel=k)
        assert ei.value.code == frbx.FRBX_ETIMEOUT
    h.set_limits()
    # the per-segment BF16 form, checked as its own tests check it (per-result error bound)
    got = h.fit_segments(vis_dev, wl.dms, rows, kernel=3)
    ref = R.fit_segments(st, vis, dk, rows)
    rel = np.abs(got["amp"] - ref[0]) / ref[0]
    assert rel.max() < 8e-3
    direct = h.fit_segments(vis_dev, wl.dms, rows, kernel=1)
    assert_fit_match(st, vis, dk, rows, direct, ref)


def test_short_wait_limit_that_suffices_changes_nothing(frbx, vgos_case):
    wl, vis = vgos_case
    vis_dev = to_dev(vis)
    h = frbx.Handle.from_workload(wl)
    ref = h.search(vis_dev, wl.dms, wl.windows, want_series=True, kernel=6)
    h.set_limits(wait_cycles=50_000_000)  # about 25 ms: far above any wait of a healthy run
    got = h.search(vis_dev, wl.dms, wl.windows, want_series=True, kernel=6)
    assert np.array_equal(got["series"], ref["series"])
    assert h.get_limits()["wait_cycles"] == 50_000_000


def test_scratch_cap_gives_enomem_then_recovers(frbx, vgos_case):
    wl, vis = vgos_case
    vis_dev = to_dev(vis)
    h = frbx.Handle.from_workload(wl)
    h.set_limits(scratch_cap_bytes=1 << 20)  # 1 MiB: less than the segment series alone
    with pytest.raises(frbx.FrbxError) as ei:
        h.search(vis_dev, wl.dms, wl.windows, want_series=True)
    assert ei.value.code == frbx.FRBX_ENOMEM
    assert 0 <= h.scratch_bytes() <= 1 << 20
    # from host memory too: the cube copy is scratch as well
    with pytest.raises(frbx.FrbxError) as ei:
        h.search(vis, wl.dms, wl.windows)
    assert ei.value.code == frbx.FRBX_ENOMEM
    h.set_limits()
    got = h.search(vis_dev, wl.dms, wl.windows, want_series=True)
    fresh = frbx.Handle.from_workload(wl).search(vis_dev, wl.dms, wl.windows, want_series=True)
    assert np.array_equal(got["series"], fresh["series"])
    assert h.scratch_bytes() > 1 << 20
    with pytest.raises(frbx.FrbxError) as ei:
        h.set_limits(wait_cycles=-1)
    assert ei.value.code == frbx.FRBX_EINVAL
