"""Candidate refinement on the GPU (frbx_refine_power / frbx_refine_adjoint, FP32 with FP64
delay and phase arguments) against the FP64 oracle of oracle/refine.py.

Tolerances: P relative 1e-4 (FP32 sums of ~8k terms); gradients relative 2e-3 of the largest
component of the same parameter type (FP32 sums of terms with large cancellation)."""
import math

import numpy as np
import pytest

import synth
from oracle import reference as R
from oracle import refine as F
from paper_1801_02391_gb300 import _build

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


def _setup(seed=0, off_grid=True):
    wl = synth.make_small(T=1200, dms=[500.0, 560.0])
    rng = np.random.default_rng(seed)
    if off_grid:
        wl.pulses[0].dm = 553.7
        wl.pulses[0].t0_bin = 400
        wl.pulses[0].snr = 40.0
    return wl, R.setup_from_workload(wl), synth.generate(wl), rng


def _random_params(rng, wl, n):
    th = np.zeros((n, 2 + 3 * wl.n_bl))
    th[:, 0] = rng.uniform(0.0, 600.0, n)
    th[:, 1] = rng.uniform(20.0, 400.0, n)
    th[:, 2::3] = rng.uniform(-60, 60, (n, wl.n_bl))
    th[:, 3::3] = rng.uniform(-15, 15, (n, wl.n_bl))
    th[:, 4::3] = rng.uniform(-1, 1, (n, wl.n_bl))
    return th


def test_power_and_adjoint_match_the_oracle(frbx):
    import torch
    wl, st, vis, rng = _setup()
    n = 24
    th = _random_params(rng, wl, n)
    width = rng.choice([2, 4, 8, 16], n).astype(np.int32)
    h = frbx.Handle.from_workload(wl)
    vd = torch.from_numpy(vis).cuda()
    pt = torch.from_numpy(th).cuda()
    wt = torch.from_numpy(width).cuda()
    power, g, status = frbx.refine_power(h, vd, pt, wt)
    assert int(status.sum()) == 0
    dpar = frbx.refine_adjoint(h, vd, pt, wt, g, torch.ones(n, device="cuda")).cpu().numpy()
    P = power.cpu().numpy()
    ref = [F.coherent_power(st, vis, th[i], int(width[i])) for i in range(n)]
    Po = np.array([r[0] for r in ref])
    Go = np.array([r[1] for r in ref])
    np.testing.assert_allclose(P, Po, rtol=1e-4)
    for k in range(Go.shape[1]):
        scale = np.abs(Go[:, k]).max()
        np.testing.assert_allclose(dpar[:, k], Go[:, k], atol=2e-3 * scale)


def test_adjoint_matches_central_differences(frbx):
    """GPU gradient vs central differences of the FP64 definition, h = 1e-3 of the grid step."""
    import torch
    wl, st, vis, rng = _setup(seed=3)
    th = _random_params(rng, wl, 1)[0]
    h = frbx.Handle.from_workload(wl)
    vd = torch.from_numpy(vis).cuda()
    pt = torch.from_numpy(th[None]).cuda()
    wt = torch.tensor([8], dtype=torch.int32, device="cuda")
    power, g, _ = frbx.refine_power(h, vd, pt, wt)
    dpar = frbx.refine_adjoint(h, vd, pt, wt, g, torch.ones(1, device="cuda")).cpu().numpy()[0]
    scales = F.grid_scales(st, 10.0)
    steps = [scales[0], scales[1]] + [s for _ in range(wl.n_bl) for s in scales[2:]]
    P0 = float(power[0])
    for k, s in enumerate(steps):
        e = np.zeros_like(th)
        e[k] = 1e-3 * s
        fd = (F.coherent_power(st, vis, th + e, 8, want_grad=False)[0] -
              F.coherent_power(st, vis, th - e, 8, want_grad=False)[0]) / (2e-3 * s)
        assert dpar[k] == pytest.approx(fd, rel=1e-2, abs=2e-4 * P0 / s)


def test_autograd_gradient_ascent_moves_to_the_offgrid_pulse(frbx):
    """Through torch.autograd (forward kernel + hand-written adjoint), Adam on the candidate
    parameters raises the summed coherent power of the injected off-grid pulse and brings DM,
    SBD and MBD closer to the injected values than the grid start."""
    import torch
    wl, st, vis, rng = _setup()
    p = wl.pulses[0]
    sbd_ax, mbd_ax = R.delay_axes(st)
    # grid start: DM 560, window of 2 starting one AP early, delays at the nearest grid cells
    th0 = [560.0, float(p.t0_bin - 1)]
    for b in range(wl.n_bl):
        tau = wl.tau_g_ns[b]
        ms = sbd_ax[np.argmin(np.abs(sbd_ax - tau))]
        wrapped = (tau + st.t_ambig_ns / 2) % st.t_ambig_ns - st.t_ambig_ns / 2
        mq = mbd_ax[np.argmin(np.abs(mbd_ax - wrapped))]
        th0 += [ms, mq, 0.0]
    h = frbx.Handle.from_workload(wl)
    vd = torch.from_numpy(vis).cuda()
    wt = torch.tensor([p.width], dtype=torch.int32, device="cuda")
    scales = np.array([10.0, 1.0] + [s for _ in range(wl.n_bl) for s in F.grid_scales(st, 10.0)[2:]])
    z = torch.zeros((1, len(th0)), dtype=torch.float64, device="cuda", requires_grad=True)  # steps of grid units
    base = torch.tensor([th0], dtype=torch.float64, device="cuda")
    sc = torch.from_numpy(scales).cuda()
    fn = frbx.coherent_power_fn()
    opt = torch.optim.Adam([z], lr=0.05)
    P_start = None
    for it in range(150):
        opt.zero_grad()
        P = fn.apply(base + z * sc, h, vd, wt)
        if P_start is None:
            P_start = float(P)
        (-P.sum() / P_start).backward()
        opt.step()
    th = (base + z * sc).detach().cpu().numpy()[0]
    P_end = float(fn.apply(base + z * sc, h, vd, wt))
    assert P_end > 1.05 * P_start
    assert abs(th[0] - p.dm) < abs(th0[0] - p.dm)
    for b in range(wl.n_bl):
        tau = wl.tau_g_ns[b]
        assert abs(th[2 + 3 * b] - tau) <= abs(th0[2 + 3 * b] - tau) + 0.5
        wrapped = (tau - th[3 + 3 * b] + st.t_ambig_ns / 2) % st.t_ambig_ns - st.t_ambig_ns / 2
        assert abs(wrapped) < 0.5 * mbd_ax[1]
