"""Appendix A extraction on the GPU (frbx_calibrate) against the FP64 oracle, and the
calibrated search recovering full coherence."""
import math

import numpy as np
import pytest

import synth
from oracle import calib as K
from oracle import reference as R
from paper_1801_02391_gb300 import _build
from tests.test_oracle_calib import _calibrator

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


@pytest.mark.parametrize("maker,noise", [("small", 0.0), ("small", 0.5), ("vgos", 0.5)])
def test_calibrate_matches_oracle(frbx, maker, noise):
    import torch
    wl = synth.make_small(T=64) if maker == "small" else synth.make_vgos(T=64, n_bl=1)
    st = R.setup_from_workload(wl)
    rng = np.random.default_rng(12)
    T = 1500
    vis = np.stack([_calibrator(st, T, 15.625 * 2 + b, rng.uniform(-3, 3, st.N), rng.uniform(-3, 3, st.N),
                                noise=noise, seed=b) for b in range(2)])
    h = frbx.Handle.from_workload(wl)
    sbd, mbd, dl, ph = h.calibrate(torch.from_numpy(vis).cuda(), 100, 1200)
    for b in range(2):
        osbd, ombd, odl, oph = K.calibrate(st, vis[b], 100, 1200)
        assert (sbd[b], mbd[b]) == (osbd, ombd)
        np.testing.assert_allclose(dl[b], odl, atol=1e-4)
        np.testing.assert_allclose(np.angle(np.exp(1j * (ph[b] - oph))), 0.0, atol=1e-4)


def test_calibrated_handle_restores_coherence(frbx):
    """Eq. 5 with the extracted (dtau0, dphi0): the GPU fit of the calibrator reaches the fully
    coherent amplitude; without them it does not."""
    import torch
    wl = synth.make_small(T=64)
    st = R.setup_from_workload(wl)
    rng = np.random.default_rng(5)
    vis = _calibrator(st, 200, 31.25, rng.uniform(-3, 3, st.N), rng.uniform(-3, 3, st.N))[None]
    vd = torch.from_numpy(vis).cuda()
    h = frbx.Handle.from_workload(wl)
    sbd, mbd, dl, ph = h.calibrate(vd, 0, 200)
    hc = frbx.Handle(wl.f0_mhz, wl.n_point, wl.f_bw_mhz, wl.t_ap_ms, chan_delay_ns=dl[0], chan_phase_rad=ph[0])
    seg = np.array([[0, 0, 64, 10]], np.int32)
    full = st.N * (st.J - 1) * 64
    assert hc.fit_segments(vd, [0.0], seg)["amp"][0] == pytest.approx(full, rel=2e-4)
    assert h.fit_segments(vd, [0.0], seg)["amp"][0] < 0.97 * full
