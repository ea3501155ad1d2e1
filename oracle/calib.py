"""FP64 oracle of the initial-phase / channel-delay extraction of Appendix A.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Steps for one baseline, following the appendix:
 a. start with zero channel delays and initial phases;
 b. build one long time segment of the calibrator (Eq. 3 with DM 0: the plain sum of the
    APs [k0, k0 + l));
 c. fringe-fit it on the grid (Eq. 5, Sec. 5.1) for the common SBD and MBD; then per channel
    - the channel delay: the delay tau_n that maximises |sum_{j>=1} S(n,j) exp(-i 2 pi f_j SBD)
      exp(-i 2 pi (f_j - f_bw/2) tau_n)| -- "fitting S exp(-i 2 pi f_j SBD)" read as a
      per-channel delay search: a DFT over j zero-padded to 8 J points, a three-point
      parabolic interpolation of |.|^2 around the peak, then Newton steps on the continuous
      channel power (NEWTON_STEPS iterations, stopped where the curvature is not negative);
    - the initial phase: the argument of the channel sum with the common SBD, MBD and the
      channel delay removed.
The outputs plug into Eq. 5 as (dtau0_n, dphi0_n).
"""
from __future__ import annotations

import math

import numpy as np

from . import reference as R

PAD = 8
NEWTON_STEPS = 8


def newton_delay(z, omega, tau):
    """Maximise |sum_j z_j exp(-i omega_j tau)|^2 near tau by Newton steps."""
    for _ in range(NEWTON_STEPS):
        e = np.exp(-1j * omega * tau)
        D = (z * e).sum()
        D1 = (-1j * omega * z * e).sum()
        D2 = (-(omega ** 2) * z * e).sum()
        f1 = 2 * (np.conj(D) * D1).real
        f2 = 2 * (abs(D1) ** 2 + (np.conj(D) * D2).real)
        if not f2 < 0:
            break
        tau = tau - f1 / f2
    return tau


def parabolic_offset(ym1, y0, yp1):
    """Vertex offset (in bins) of the parabola through three equally spaced samples."""
    den = ym1 - 2 * y0 + yp1
    return 0.0 if den == 0 else 0.5 * (ym1 - yp1) / den


def calibrate(st: R.Setup, vis_bl: np.ndarray, k0: int, l: int):
    """vis_bl: [T][C] complex of one baseline.  Returns (sbd_ns, mbd_ns, delay_ns[N], phase_rad[N])."""
    X = vis_bl[k0:k0 + l].astype(np.complex128).sum(axis=0)
    # (c) common fringe fit on the grid, without calibration
    zero = R.make_setup(st.f0_mhz, st.J, st.f_bw_mhz, st.t_ap_ms, flag=st.flag, sbd_pad=st.Ls // st.J,
                        mbd_pad=st.Lm // max(1, R._nextpow2(int(st.g.max()) + 1)))
    cube = X.astype(np.complex64)[None, None, :]
    # the grid fit of the complex64 segment; the sum itself was taken in FP64 above
    a, m, q, _, grid = R.fit_segments(zero, cube, np.zeros((1, st.C), np.int32), np.array([[0, 0, 1, 0]], np.int32),
                                      want_grid=True)
    sbd_ax, mbd_ax = R.delay_axes(st)
    sbd, mbd = float(sbd_ax[m[0]]), float(mbd_ax[q[0]])
    J, N = st.J, st.N
    fj = (np.arange(J) * st.f_bw_mhz) / J
    delays = np.zeros(N)
    phases = np.zeros(N)
    used = (np.arange(J) >= 1)
    for n in range(N):
        w = used & (st.flag[n * J:(n + 1) * J] == 0)
        z = X[n * J:(n + 1) * J] * np.exp(-2j * math.pi * fj * sbd * 1e-3) * w
        L = PAD * J
        # the delay search: D(p) = sum_j z_j exp(-2 pi i (f_j - f_bw/2) tau_p), tau_p on a grid of
        # J / (L f_bw) us; evaluated directly (the common factor exp(i pi f_bw tau) has modulus 1)
        step_ns = (J * 1000.0) / (L * st.f_bw_mhz)
        p = np.arange(L)
        sp = np.where(p < L // 2, p, p - L)
        taus = sp * step_ns
        D = np.exp(-2j * math.pi * np.outer(taus, fj - st.f_bw_mhz / 2) * 1e-3) @ z
        pw = np.abs(D) ** 2
        k = int(np.argmax(pw))
        off = parabolic_offset(pw[(k - 1) % L], pw[k], pw[(k + 1) % L])
        omega = 2 * math.pi * (fj - st.f_bw_mhz / 2) * 1e-3
        tau_n = newton_delay(z, omega, (sp[k] + off) * step_ns)
        delays[n] = tau_n
        ph = 2 * math.pi * (fj * sbd + (st.f0_mhz[n] - st.f0_mhz.min()) * mbd + (fj - st.f_bw_mhz / 2) * tau_n) * 1e-3
        phases[n] = float(np.angle((X[n * J:(n + 1) * J] * w * np.exp(-1j * ph)).sum()))
    return sbd, mbd, delays, phases
