"""Pins of the refinement oracle (coherent power of Eq. 4 with continuous DM / time)."""
import math

import numpy as np
import pytest

import synth
from oracle import reference as R
from oracle import refine as F


def _wl():
    wl = synth.make_small(T=160, n_bl=2, dms=[0.0, 100.0])
    wl.pulses = []
    return wl


def test_reduces_to_the_grid_transform():
    """DM 0, integer t0, zero rate: the interpolation is the identity and P of one baseline is
    |G|^2 of the grid transform at the cell of (tau_s, tau_m) (Eq. 5 on the Sec. 5.1 grid)."""
    wl = _wl()
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    dk = R.shift_table(st, [0.0])
    seg = np.array([[0, 0, 4, 37]], np.int32)
    _, _, _, _, grid = R.fit_segments(st, vis[:1], dk, seg, want_grid=True)
    sbd, mbd = R.delay_axes(st)
    for m, q in ((0, 0), (3, 5), (60, 11)):
        th = np.array([0.0, 37.0, sbd[m], mbd[q], 0.0])
        P, _ = F.coherent_power(st, vis[:1], th, 4, want_grad=False)
        assert P == pytest.approx(abs(grid[0, m, q]) ** 2, rel=1e-10)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    """Analytic gradient vs central differences: h = 1e-3 of each parameter's grid step
    (relative 1e-2: on noise the interpolated data are rough along time, so the DM and time
    differences carry an O(h^2) truncation error of a few 1e-3) and h = 1e-4 of it
    (relative 1e-4)."""
    wl = _wl()
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    rng = np.random.default_rng(seed)
    scales = F.grid_scales(st, 10.0)
    th = np.array([rng.uniform(20, 80), rng.uniform(30, 60)] +
                  [v for _ in range(wl.n_bl) for v in (rng.uniform(-40, 40), rng.uniform(-10, 10), rng.uniform(-0.5, 0.5))])
    P, g = F.coherent_power(st, vis, th, 8)
    steps = [scales[0], scales[1]] + [s for _ in range(wl.n_bl) for s in scales[2:]]
    for k, s in enumerate(steps):
        for hf, rel in ((1e-3, 1e-2), (1e-4, 1e-4)):
            h = hf * s
            e = np.zeros_like(th)
            e[k] = h
            fd = (F.coherent_power(st, vis, th + e, 8, want_grad=False)[0] -
                  F.coherent_power(st, vis, th - e, 8, want_grad=False)[0]) / (2 * h)
            assert g[k] == pytest.approx(fd, rel=rel, abs=1e-6 * P / s)


def test_tone_peak_at_true_offgrid_delays_and_rate():
    """A noise-free tone with off-grid delays and a fringe rate: P is stationary (gradient ~ 0)
    at the true (tau_s, tau_m, rho) and equals (N (J-1) l)^2 there."""
    wl = _wl()
    st = R.setup_from_workload(wl)
    T, l, t0 = 160, 6, 50.0
    tau, rho = 23.7, 0.3  # ns, ns/s
    f = st.f
    f0n = np.repeat(st.f0_mhz, st.J)
    k = np.arange(T)[:, None]
    ph = 2 * math.pi * ((f - st.f0_mhz.min()) * tau * 1e-3 + f0n * rho * st.t_ap_ms * k * 1e-6)
    vis = np.exp(1j * ph)[None]
    th = np.array([0.0, t0, tau, tau, rho])
    P, g = F.coherent_power(st, vis, th, l)
    assert P == pytest.approx((st.N * (st.J - 1) * l) ** 2, rel=1e-9)
    scales = F.grid_scales(st, 10.0)
    assert abs(g[2]) * scales[2] < 1e-9 * P and abs(g[3]) * scales[3] < 1e-9 * P and abs(g[4]) * scales[4] < 1e-9 * P
    P2, _ = F.coherent_power(st, vis, th + np.array([0, 0, 3.0, 0, 0]), l)
    assert P2 < P


def test_dm_and_time_peak_on_a_dispersed_pulse():
    """A dispersed Gaussian pulse (sigma 3 APs): P at the true DM and window start exceeds P one
    DM step or one AP away, and the DM / time gradient vanishes there."""
    wl = _wl()
    st = R.setup_from_workload(wl)
    T, dm_true, w, sig = 400, 140.0, 8, 3.0
    c_top = 100.0 + (w - 1) / 2.0
    u = c_top + dm_true * R.K_DM * (1 / st.f ** 2 - 1 / st.f_ref_dm_mhz ** 2) / st.t_ap_ms
    k = np.arange(T)[:, None]
    vis = np.exp(-0.5 * ((k - u[None, :]) / sig) ** 2)[None] + 0j
    th0 = np.array([dm_true, 100.0, 0, 0, 0.0])
    best, g = F.coherent_power(st, vis, th0, w)
    for d in ((10.0, 0.0), (-10.0, 0.0), (0.0, 1.0), (0.0, -1.0)):
        assert F.coherent_power(st, vis, th0 + np.array([d[0], d[1], 0, 0, 0.0]), w, want_grad=False)[0] < best
    assert abs(g[0]) * 10.0 < 1e-3 * best and abs(g[1]) < 1e-3 * best
