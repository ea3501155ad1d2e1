"""FP64 oracle of the candidate refinement (continuous DM, time, delays and rate).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For one candidate and baseline b, the delay-resolution function of Eq. 4 with its
delay-rate term kept, over a window of l APs whose start follows the dispersion sweep
continuously instead of Eq. 2's rounding:

    u(n, j)  = t0 + 4.15e6 DM (f^-2 - f_ref^-2) / t_ap          (APs, Eq. 1 without rounding)
    X(n,j,i) = sum_{m=-1..2} w_m(phi) S(n, j, k + m),  k = floor(u + i), phi = u + i - k
               (cubic Catmull-Rom fractional-delay interpolation, C1 in phi)
    Phi      = 2 pi [ f_j tau_s + (f0_n - f0_min) tau_m ] * 1e-3
             + 2 pi f0_n rho t_ap (u + i) * 1e-6               (MHz, ns, ns/s, ms, APs)
    G_b      = sum_n sum_{j>=1} c(n,j) sum_{i<l} X(n,j,i) exp(-i Phi)
    P        = sum_b |G_b|^2                                      (summed coherent power)

Parameters per candidate: DM and t0 shared by all baselines; tau_s, tau_m, rho per baseline
(layout [dm, t0, (tau_s, tau_m, rho) x n_bl]).  c(n, j) is the calibration rotation and
weight of Eq. 5 (zero for j = 0 and flagged points).  The gradient is the derivative of
this definition, dP/dtheta = sum_b 2 Re(conj(G_b) dG_b/dtheta).
"""
from __future__ import annotations

import math

import numpy as np

from .reference import K_DM, Setup


def catmull_rom(phi):
    """Weights of taps k-1, k, k+1, k+2 and their derivatives in phi."""
    p2, p3 = phi * phi, phi * phi * phi
    w = np.stack([(-p3 + 2 * p2 - phi) / 2, (3 * p3 - 5 * p2 + 2) / 2, (-3 * p3 + 4 * p2 + phi) / 2,
                  (p3 - p2) / 2])
    dw = np.stack([(-3 * p2 + 4 * phi - 1) / 2, (9 * p2 - 10 * phi) / 2, (-9 * p2 + 8 * phi + 1) / 2,
                   (3 * p2 - 2 * phi) / 2])
    return w, dw


def n_params(n_bl: int) -> int:
    return 2 + 3 * n_bl


def _weights(st: Setup):
    used = np.ones(st.C, bool)
    used[0::st.J] = False
    used &= st.flag == 0
    return np.where(used, st.rot, 0.0)


def coherent_power(st: Setup, vis: np.ndarray, params, width: int, want_grad=True):
    """P and dP/dparams for one candidate.  vis: [n_bl][T][C] complex."""
    vis = np.asarray(vis)
    n_bl, T, C = vis.shape
    th = np.asarray(params, dtype=np.float64)
    dm, t0 = th[0], th[1]
    cw = _weights(st)
    f = st.f
    f0n = np.repeat(st.f0_mhz, st.J)
    fj = np.tile((np.arange(st.J) * st.f_bw_mhz) / st.J, st.N)
    fmbd = f0n - st.f0_mhz.min()
    ddm = K_DM * (1.0 / (f * f) - 1.0 / (st.f_ref_dm_mhz * st.f_ref_dm_mhz)) / st.t_ap_ms   # du/dDM
    u = t0 + dm * ddm
    P = 0.0
    grad = np.zeros(th.shape)
    cols = np.arange(C)
    for b in range(n_bl):
        tau_s, tau_m, rho = th[2 + 3 * b: 5 + 3 * b]
        G = 0j
        A_s = A_m = A_r = A_t0 = A_dm = 0j
        for i in range(width):
            x = u + i
            k = np.floor(x).astype(np.int64)
            phi = x - k
            if k.min() - 1 < 0 or k.max() + 2 > T - 1:
                raise ValueError("candidate window reaches outside the cube")
            w, dw = catmull_rom(phi)
            taps = np.stack([vis[b, k + m, cols] for m in (-1, 0, 1, 2)])
            xs = (w * taps).sum(axis=0)
            dxs = (dw * taps).sum(axis=0)
            ph = 2 * math.pi * ((fj * tau_s + fmbd * tau_m) * 1e-3 + f0n * rho * st.t_ap_ms * x * 1e-6)
            e = np.exp(-1j * ph)
            term = cw * xs * e
            G += term.sum()
            if want_grad:
                A_s += (term * (-2j * math.pi * fj * 1e-3)).sum()
                A_m += (term * (-2j * math.pi * fmbd * 1e-3)).sum()
                A_r += (term * (-2j * math.pi * f0n * st.t_ap_ms * x * 1e-6)).sum()
                du = cw * dxs * e + term * (-2j * math.pi * f0n * rho * st.t_ap_ms * 1e-6)
                A_t0 += du.sum()
                A_dm += (du * ddm).sum()
        P += abs(G) ** 2
        if want_grad:
            g = np.conj(G)
            grad[0] += 2 * (g * A_dm).real
            grad[1] += 2 * (g * A_t0).real
            grad[2 + 3 * b] = 2 * (g * A_s).real
            grad[3 + 3 * b] = 2 * (g * A_m).real
            grad[4 + 3 * b] = 2 * (g * A_r).real
    return P, grad


def grid_scales(st: Setup, dm_step: float):
    """Natural step of each parameter type: DM grid step, 1 AP, SBD and MBD grid steps, and
    the delay rate that turns the phase by one cycle across 1000 APs at the top channel."""
    sbd_step = (st.J * 1000.0) / (st.Ls * st.f_bw_mhz)
    mbd_step = 1000.0 / (st.Lm * st.df_grid_mhz)
    rho_step = 1e6 / (st.f0_mhz.max() * st.t_ap_ms * 1000.0)
    return dm_step, 1.0, sbd_step, mbd_step, rho_step
