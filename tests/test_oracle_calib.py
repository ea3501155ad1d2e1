"""Pins of the Appendix A extraction oracle (channel delays and initial phases)."""
import math

import numpy as np
import pytest

import synth
from oracle import calib as K
from oracle import reference as R


def _calibrator(st, T, tau_ns, d_ns, p_rad, noise=0.0, seed=0):
    f = st.f
    fj = np.tile((np.arange(st.J) * st.f_bw_mhz) / st.J, st.N)
    dn = np.repeat(d_ns, st.J)
    pn = np.repeat(p_rad, st.J)
    ph = 2 * math.pi * ((f - st.f0_mhz.min()) * tau_ns + (fj - st.f_bw_mhz / 2) * dn) * 1e-3 + pn
    vis = np.repeat(np.exp(1j * ph)[None, :], T, axis=0)
    if noise:
        rng = np.random.default_rng(seed)
        vis = vis + noise * (rng.standard_normal(vis.shape) + 1j * rng.standard_normal(vis.shape)) / math.sqrt(2)
    return vis.astype(np.complex64)


def test_recovers_channel_delays_and_flattens_the_phase():
    """Noise-free calibrator with per-channel delays and phases: the extracted (dtau0, dphi0)
    plugged into Eq. 5 give the fully coherent |G| = N (J - 1) l at the grid peak, while the
    uncalibrated fit loses power (the 5-10 % loss of Sec. 2.3 for delays of a few ns)."""
    wl = synth.make_small(T=64)
    st = R.setup_from_workload(wl)
    rng = np.random.default_rng(4)
    d = rng.uniform(-3, 3, st.N)
    p = rng.uniform(-3, 3, st.N)
    tau = 15.625 * 2   # on the SBD grid and a multiple of the MBD step
    vis = _calibrator(st, 64, tau, d, p)
    sbd, mbd, delays, phases = K.calibrate(st, vis, 0, 40)
    assert sbd == pytest.approx(tau)
    np.testing.assert_allclose(delays, d, atol=1e-6)
    st_cal = R.make_setup(wl.f0_mhz, st.J, st.f_bw_mhz, st.t_ap_ms, chan_delay_ns=delays, chan_phase_rad=phases)
    seg = np.array([[0, 0, 40, 0]], np.int32)
    a_cal = R.fit_segments(st_cal, vis[None], np.zeros((1, st.C), np.int32), seg)[0][0]
    a_raw = R.fit_segments(st, vis[None], np.zeros((1, st.C), np.int32), seg)[0][0]
    full = st.N * (st.J - 1) * 40
    assert a_cal == pytest.approx(full, rel=2e-4)
    assert a_raw < 0.97 * full


def test_noisy_calibrator_high_snr():
    wl = synth.make_small(T=2000)
    st = R.setup_from_workload(wl)
    rng = np.random.default_rng(9)
    d = rng.uniform(-2, 2, st.N)
    p = rng.uniform(-3, 3, st.N)
    vis = _calibrator(st, 2000, 7.8125 * 3, d, p, noise=0.5, seed=1)   # channel SNR ~ 500
    sbd, mbd, delays, phases = K.calibrate(st, vis, 0, 2000)
    # residual common delay (tau - sbd) is shared by all channels; differences are pinned
    np.testing.assert_allclose(np.diff(delays), np.diff(d), atol=0.1)
