"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints (tests/golden), closed forms, invariants, special cases that reduce
to a library routine, and brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import reference as R
from oracle import _clib


def _golden(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- worked numbers
def test_worked_numbers_eq7_eq11(golden_dir):
    """Eq. 7 (T1, T2) and Eq. 11 (T3, T4) reproduce the values printed in Sec. 4 and 5.3."""
    g = {r[0]: (float(r[1]), float(r[2])) for r in _golden(golden_dir, "worked_numbers.txt")}
    noise = R.radiometer_noise_jy(800.0, 560.0, 96e6, 4.096e-3)
    assert noise == pytest.approx(g["eq7_noise_jy_shur"][0], rel=g["eq7_noise_jy_shur"][1])
    # invert Eq. 7 for T at SEFD 2000 Jy (both ends), B = 0.5 GHz, same noise level
    t_vgos_ms = 2000.0 * 2000.0 / (2 * 0.5e9 * noise ** 2) * 1e3
    assert t_vgos_ms == pytest.approx(g["eq7_vgos_window_ms"][0], rel=g["eq7_vgos_window_ms"][1])
    assert round(noise * 7.0, 1) == pytest.approx(g["eq7_vgos_fluence_jyms"][0], rel=g["eq7_vgos_fluence_jyms"][1])
    res1 = R.dm_resolution(4.096, 2192.0, 2288.0)
    assert res1 == pytest.approx(g["eq11_dmres_psrf02"][0], rel=g["eq11_dmres_psrf02"][1])
    res2 = R.dm_resolution(8.0, 2200.0, 2700.0)
    assert res2 == pytest.approx(g["eq11_dmres_vgos"][0], rel=g["eq11_dmres_vgos"][1])
    assert round(2000.0 / res2) == int(g["eq11_vgos_bins"][0])


def test_eq1_constant_matches_eq11():
    """Eq. 11's 2.41e-7 is 1/4.15e6 of Eq. 1: a DM step of DM_res sweeps exactly one minimum
    window across the band through the shift table (4.096 ms = 4 APs of 1.024 ms)."""
    assert R.K_DM * 2.41e-7 == pytest.approx(1.0, abs=2e-4)
    st = R.make_setup([2192.0], 2, 96.0, 1.024)   # points at 2192 and 2240 MHz; f_ref given below
    st = R.make_setup([2192.0], 2, 96.0, 1.024, f_ref_dm_mhz=2288.0)
    dk = R.shift_table(st, [R.dm_resolution(4.096, 2192.0, 2288.0)])
    assert dk[0, 0] == 4


def test_shift_table_hand_value():
    """Eq. 1-2 by hand: DM 557, f = 1400 MHz, f_ref = 1655 MHz (top point of the small setup),
    t_ap 1 ms: 4.15e6 * 557 * (1/1400^2 - 1/1655^2) = 335.43 ms -> dk = 335."""
    wl = synth.make_small(T=64)
    st = R.setup_from_workload(wl)
    assert st.f_ref_dm_mhz == 1655.0
    dk = R.shift_table(st, [557.0])
    assert dk[0, 0] == 335
    assert dk[0, -1] == 0


def test_shift_table_invariants():
    """DM 0 gives identity shifts; the top point never moves; dk grows with DM and with 1/f."""
    wl = synth.make_vgos(T=64, n_bl=1, n_dm=16)
    st = R.setup_from_workload(wl)
    dk = R.shift_table(st, wl.dms)
    assert np.all(dk[0] == 0)
    top = int(np.argmax(st.f))
    assert np.all(dk[:, top] == 0)
    assert np.all(np.diff(dk, axis=0) >= 0)
    order = np.argsort(st.f)
    assert np.all(np.diff(dk[:, order], axis=1) <= 0)
    # largest delay: DM 2000 at 3000 MHz vs 10688-ish MHz top, 0.5 ms APs ~ 1699 APs
    assert 1690 <= dk[-1].max() <= 1705


def test_shift_table_rounds_half_up():
    """Eq. 2 is floor(0.5 + x): x = 0.5 gives 1 and x = 2.5 gives 3 (round-half-even would
    give 0 and 2).  Points at 1 and 2 MHz make every FP64 step exact."""
    for t_ap, want in ((6225000.0, 1), (1245000.0, 3), (1245000.0 * 1.0001, 2)):
        st = R.make_setup([1.0], 2, 2.0, t_ap, f_ref_dm_mhz=2.0)
        assert R.shift_table(st, [1.0])[0, 0] == want    # 4.15e6 * 0.75 / t_ap = 0.5, 2.5, 2.4998


# ---------------------------------------------------------------- time grid (T5)
def test_tab4_times_on_half_overlap_grid(golden_dir):
    """Tab. 4 times are segment starts: 10 s + k0 * 1.024 ms with k0 on the half-overlap grid
    k0 = m * (l/2) of the listed width (Sec. 2.4.1, Sec. 3.2)."""
    for scan, bl, t, ph, width_ms, p in _golden(golden_dir, "tab4_three_baseline_pulses.txt"):
        l = float(width_ms) / 1.024
        assert abs(l - round(l)) < 1e-9
        l = int(round(l))
        assert l in (4, 8, 16, 24, 32)
        k0 = (float(t) - 10.0) / 1.024e-3
        assert abs(k0 - round(k0)) < 1e-6
        assert int(round(k0)) % R.window_step(l) == 0


# ---------------------------------------------------------------- counting (T6)
def test_tab3_counting_semantics(golden_dir):
    """Tab. 3 pair columns count groups containing both baselines (triples included): the
    paper's totals 16 (exactly two baselines) and 15 (in phase) follow only from that reading,
    and coincidence_counts reproduces every row from groups built under it."""
    rows = [[int(v) for v in r] for r in _golden(golden_dir, "tab3_crossmatch_counts.txt")]
    two_all = sum(r[7] + r[9] + r[11] - 3 * r[13] for r in rows)
    two_in = sum(r[8] + r[10] + r[12] - 3 * r[14] for r in rows)
    assert (two_all, two_in) == (16, 15)
    assert sum(r[13] for r in rows) == 4 and sum(r[14] for r in rows) == 4
    for r in rows:
        tri = r[13]
        pairs = {(0, 1): r[7] - tri, (0, 2): r[9] - tri, (1, 2): r[11] - tri}
        groups = [{"mask": 0b111}] * tri
        for (a, b), n in pairs.items():
            groups += [{"mask": (1 << a) | (1 << b)}] * n
        singles = {b: r[1 + 2 * b] for b in range(3)}
        count = R.coincidence_counts(groups, singles)
        assert [count((0,)), count((1,)), count((2,)), count((0, 1)), count((0, 2)), count((1, 2)),
                count((0, 1, 2))] == [r[1], r[3], r[5], r[7], r[9], r[11], r[13]]


# ---------------------------------------------------------------- transform pins
def _one_segment_cube(x_c):
    return np.asarray(x_c, np.complex64).reshape(1, 1, -1)


def _fit_spectrum(st, spec, want_grid=True, allow=(None, None)):
    vis = _one_segment_cube(spec)
    dk = np.zeros((1, st.C), np.int32)
    seg = np.array([[0, 0, 1, 0]], np.int32)
    return R.fit_segments(st, vis, dk, seg, allow[0], allow[1], want_grid=want_grid)


@pytest.mark.parametrize("m0", [0, 1, 3, 7, 60])
def test_pure_tone_on_grid(m0):
    """A tone exp(2 pi i (f - f0_0) tau) with tau on both grids gives |G| = N (J-1) exactly at
    (m, q) = (tau Ls f_bw / J, tau Lm df_grid) mod (Ls, Lm) (Eq. 5, Sec. 5.1)."""
    wl = synth.make_small(T=64)
    st = R.setup_from_workload(wl)
    tau = 15.625 * m0   # SBD step 15.625 ns; a multiple of the MBD step 1.953125 ns
    spec = synth.pure_tone_segment(wl, tau)
    amp, m, q, amp2, grid = _fit_spectrum(st, spec)
    assert amp[0] == pytest.approx(st.N * (st.J - 1), rel=1e-6)
    assert m[0] == (m0 % st.Ls)
    assert q[0] == (8 * m0) % st.Lm


@pytest.mark.parametrize("tau", [7.3, -23.9, 41.05])
def test_off_grid_tone_dirichlet_closed_form(tau):
    """Off grid, |G(m,q)| = |sum_{j=1}^{J-1} e^{2 pi i j (f_bw/J tau - m/Ls)}| *
    |sum_n e^{2 pi i g_n (df tau - q/Lm)}| (product of Dirichlet kernels), every cell."""
    wl = synth.make_small(T=64)
    st = R.setup_from_workload(wl)
    spec = synth.pure_tone_segment(wl, tau)
    _, _, _, _, grid = _fit_spectrum(st, spec)
    t = tau * 1e-3
    j = np.arange(1, st.J)
    m = np.arange(st.Ls)
    ds = np.abs(np.exp(2j * np.pi * np.outer(st.f_bw_mhz / st.J * t - m / st.Ls, j)).sum(axis=1))
    q = np.arange(st.Lm)
    dm_ = np.abs(np.exp(2j * np.pi * np.outer(st.df_grid_mhz * t - q / st.Lm, st.g)).sum(axis=1))
    want = np.outer(ds, dm_)
    np.testing.assert_allclose(np.abs(grid[0]), want, rtol=1e-5, atol=1e-4)


def test_parseval_full_grid():
    """sum_{m,q} |G|^2 = Ls Lm sum_{n, j>=1, unflagged} |X|^2 when the g_n are distinct."""
    wl = synth.make_vgos(T=4, n_bl=1, n_dm=1)
    st = R.setup_from_workload(wl)
    rng = np.random.default_rng(5)
    spec = (rng.standard_normal(st.C) + 1j * rng.standard_normal(st.C)).astype(np.complex64)
    _, _, _, _, grid = _fit_spectrum(st, spec)
    used = np.ones((st.N, st.J), bool)
    used[:, 0] = False
    used &= st.flag.reshape(st.N, st.J) == 0
    x = spec.astype(np.complex128).reshape(st.N, st.J)
    lhs = (np.abs(grid[0]) ** 2).sum()
    rhs = st.Ls * st.Lm * (np.abs(x[used]) ** 2).sum()
    assert lhs == pytest.approx(rhs, rel=1e-10)


def test_matches_numpy_fft2_on_zero_padded_grid():
    """G(m,q) = fft2(Z)[q, m] with Z[g_n, j] = X(n, j) (j >= 1) zero-padded to [Lm][Ls]."""
    st = R.make_setup([800.0, 848.0, 880.0, 816.0], 8, 16.0, 1.0)   # uneven grid, g = 0,3,5,1
    assert list(st.g) == [0, 3, 5, 1] and st.Lm == 16 and st.Ls == 16
    rng = np.random.default_rng(11)
    spec = (rng.standard_normal(st.C) + 1j * rng.standard_normal(st.C)).astype(np.complex64)
    _, _, _, _, grid = _fit_spectrum(st, spec)
    Z = np.zeros((st.Lm, st.Ls), np.complex128)
    x = spec.astype(np.complex128).reshape(st.N, st.J)
    for n in range(st.N):
        Z[st.g[n], 1:st.J] += x[n, 1:]
    F = np.fft.fft2(Z)
    np.testing.assert_allclose(grid[0], F.T, rtol=1e-10, atol=1e-10)


def test_factored_sum_equals_literal_triple_sum():
    """The oracle's j-then-n evaluation equals the literal triple sum of Eq. 5 (tiny input,
    with a flagged point and a calibration rotation)."""
    flag = np.zeros(3 * 6, np.uint8)
    flag[8] = 1
    st = R.make_setup([500.0, 532.0, 596.0], 6, 16.0, 1.0, chan_delay_ns=[3.0, -5.0, 1.5],
                      chan_phase_rad=[0.3, -1.1, 2.0], flag=flag)
    rng = np.random.default_rng(3)
    spec = (rng.standard_normal(st.C) + 1j * rng.standard_normal(st.C)).astype(np.complex64)
    amp, m, q, amp2, grid = _fit_spectrum(st, spec)
    x = spec.astype(np.complex128) * st.rot
    lit = _clib.triple_sum(x, st.N, st.J, st.flag, st.g, st.Ls, st.Lm)
    np.testing.assert_allclose(grid[0], lit, rtol=1e-9, atol=1e-9)
    a = np.abs(lit)
    assert amp[0] == pytest.approx(a.max(), rel=1e-12)
    assert (m[0], q[0]) == np.unravel_index(np.argmax(a), a.shape)


def test_j0_and_flagged_points_excluded():
    """Only j >= 1 enters Eq. 5 (Sec. 2.3): a spectrum living on j = 0 and flagged points
    gives G == 0."""
    flag = np.zeros(4 * 8, np.uint8)
    flag[[3, 17]] = 1
    st = R.make_setup([800.0, 816.0, 832.0, 848.0], 8, 16.0, 1.0, flag=flag)
    spec = np.zeros(st.C, np.complex64)
    spec[0::8] = 5.0 + 2.0j
    spec[[3, 17]] = -7.0j
    _, _, _, _, grid = _fit_spectrum(st, spec)
    assert np.abs(grid[0]).max() == 0.0


def test_window_additivity_eq_sec51():
    """G_{k0,l1} + G_{k0+l1,l2} = G_{k0,l1+l2} (Sec. 5.1), through the dedispersion gather."""
    wl = synth.make_small(T=400, n_bl=1, dms=[0.0, 300.0])
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    dk = R.shift_table(st, wl.dms)
    seg = np.array([[0, 1, 3, 5], [0, 1, 4, 8], [0, 1, 7, 5], [0, 0, 2, 9], [0, 0, 6, 11], [0, 0, 8, 9]], np.int32)
    _, _, _, _, grid = R.fit_segments(st, vis, dk, seg, want_grid=True)
    scale = np.abs(grid).max()
    np.testing.assert_allclose(grid[0] + grid[1], grid[2], atol=1e-12 * scale)
    np.testing.assert_allclose(grid[3] + grid[4], grid[5], atol=1e-12 * scale)


def test_dedispersion_identity_at_zero_dm():
    """DM 0 and l = 1: the segment is the raw AP, so |G| of AP k equals the transform of vis[k]."""
    wl = synth.make_small(T=16, n_bl=1, dms=[0.0])
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    dk = R.shift_table(st, wl.dms)
    seg = np.array([[0, 0, 1, 5]], np.int32)
    _, _, _, _, g1 = R.fit_segments(st, vis, dk, seg, want_grid=True)
    _, _, _, _, g2 = _fit_spectrum(st, vis[0, 5])
    np.testing.assert_array_equal(g1, g2)


def test_delay_window_masks():
    """A delay window restricts the maximum to the cells whose SBD / MBD lie inside it."""
    wl = synth.make_small(T=16)
    st = R.setup_from_workload(wl)
    spec = synth.pure_tone_segment(wl, 15.625 * 7)     # peak at SBD 109.4 ns
    am, aq = R.window_masks(st, sbd_win_ns=(-64.0, 64.0), mbd_win_ns=None)
    sbd, mbd = R.delay_axes(st)
    assert sbd[4] == 62.5 and am[4] == 1 and am[5] == 0 and am[-4] == 1 and am[-5] == 0
    amp, m, q, _, grid = _fit_spectrum(st, spec, allow=(am, aq))
    a = np.abs(grid[0])
    a[am == 0, :] = -1
    assert amp[0] == pytest.approx(a.max(), rel=1e-12)
    assert am[m[0]] == 1
    assert mbd[7] == 13.671875 and mbd[8] == -15.625 and st.t_ambig_ns == 31.25


def test_rayleigh_noise_level():
    """Noise only: at a fixed cell |G| is Rayleigh with mean sqrt(pi M)/2, M = l * (#used
    points) (Eq. 7's radiometer scaling); checked loosely on 400 segments."""
    wl = synth.make_small(T=2000, n_bl=1, dms=[0.0])
    wl.pulses, wl.rfi_points = [], []
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    dk = R.shift_table(st, wl.dms)
    l = 4
    seg = np.array([[0, 0, l, 4 * i] for i in range(400)], np.int32)
    _, _, _, _, grid = R.fit_segments(st, vis, dk, seg, want_grid=True)
    M = l * st.N * (st.J - 1)
    mean = np.abs(grid[:, 3, 5]).mean()
    assert mean == pytest.approx(math.sqrt(math.pi * M) / 2, rel=0.08)


# ---------------------------------------------------------------- normalisation
def test_normalised_power_zero_mean_unit_std():
    rng = np.random.default_rng(1)
    T, windows = 100, [1, 4]
    dk_max = np.array([0, 30])
    offs, S = R.slot_offsets(T, windows)
    amp = rng.random((2, 2, S)) + 1.0
    P = R.normalise(amp, T, windows, dk_max)
    for d in range(2):
        for w, l in enumerate(windows):
            nv = R.n_valid(T, l, int(dk_max[d]))
            p = P[:, d, offs[w]:offs[w] + nv]
            np.testing.assert_allclose(p.mean(axis=1), 0.0, atol=1e-12)
            np.testing.assert_allclose(p.std(axis=1), 1.0, rtol=1e-12)
            assert np.all(np.isnan(P[:, d, offs[w] + nv:offs[w] + R.n_slots(T, l)]))


def test_segment_counts():
    """Half overlap: l = 4 on T = 20 gives k0 = 0, 2, ..., 16 (9 segments); a dispersion
    sweep of 5 APs leaves k0 <= 11 (6 segments); l = 1 steps by one."""
    assert R.n_slots(20, 4) == 9
    assert R.n_valid(20, 4, 5) == 6
    assert R.n_slots(20, 1) == 20 and R.n_valid(20, 1, 19) == 1 and R.n_valid(20, 1, 20) == 0
    assert R.window_step(24) == 12 and R.window_step(3) == 1


# ---------------------------------------------------------------- grouping (Sec. 2.4.1)
def C(w, l, k0, p, q=0, d=0, s=0):
    return R.Cand(series=s, d=d, w=w, l=l, k0=k0, amp=1.0, p=p, q=q)


def test_step_b_insertion_first_group_no_merge():
    # largest window first; the bridging event [2, 12) joins the first group only
    items = [C(1, 4, 0, 5.0), C(1, 4, 10, 5.0), C(0, 10, 2, 4.0)]
    groups = R.insert_groups(items)
    assert [[(c.l, c.k0) for c in g] for g in groups] == [[(4, 0), (10, 2)], [(4, 10)]]
    # half-open ranges: [0,4) and [4,8) do not overlap
    groups = R.insert_groups([C(0, 4, 0, 4.0), C(0, 4, 4, 4.0)])
    assert len(groups) == 2


def test_single_baseline_steps_b_to_d():
    windows = [4, 8, 16]
    Lm = 16
    cands = [C(2, 16, 96, 6.0, q=1), C(1, 8, 100, 9.0, q=0), C(1, 8, 104, 7.0, q=15),
             C(0, 4, 104, 8.0, q=8),        # MBD opposite: removed by step c
             C(0, 4, 300, 12.0, q=2), C(1, 8, 296, 4.0, q=3)]   # only 2 windows -> rejected
    pulses = R.single_series_pulses(cands, windows, nwin_min=3, Lm=Lm, use_mbd=True)
    assert len(pulses) == 0   # first group has windows {16, 8} after step c -> 2 < 3
    pulses = R.single_series_pulses(cands, windows, nwin_min=2, Lm=Lm, use_mbd=True)
    assert [(p.l, p.k0, p.n_win) for p in pulses] == [(8, 100, 2), (4, 300, 2)]
    pulses = R.single_series_pulses(cands, windows, nwin_min=3, Lm=Lm, use_mbd=False)
    assert [(p.l, p.k0, p.n_win) for p in pulses] == [(8, 100, 3)]


def test_mbd_circular_mean_wraps():
    """Step c with the ambiguity: q = 15, 0, 1 of Lm = 16 average to ~0, not to 5.3."""
    grp = [C(0, 4, 0, 5.0, q=15), C(0, 4, 2, 5.0, q=0), C(0, 4, 4, 5.0, q=1), C(0, 4, 6, 5.0, q=5)]
    keep = R.mbd_filter(grp, 16)
    assert [c.q for c in keep] == [15, 0, 1]


def test_pick_pulse_ties_first_inserted():
    grp = [C(1, 8, 0, 5.0), C(0, 4, 0, 5.0), C(2, 16, 0, 5.0)]
    p = R.pick_pulse(grp, 3)
    assert (p.l, p.n_win) == (8, 3)


def test_dm_merge_keeps_highest_power_lowest_dm_on_tie():
    by_d = {0: [C(0, 4, 100, 5.0, d=0)], 1: [C(0, 4, 102, 7.0, d=1)], 2: [C(0, 4, 101, 7.0, d=2)],
            3: [C(0, 4, 500, 3.5, d=3)]}
    out = R.dm_merge(by_d)
    assert [(c.d, c.k0) for c in out] == [(1, 102), (3, 500)]


def test_cross_match_groups_by_overlap():
    merged = {0: [C(0, 4, 100, 5.0), C(0, 4, 600, 5.0)], 1: [C(0, 8, 98, 5.0, s=1)],
              2: [C(0, 4, 900, 5.0, s=2), C(0, 4, 103, 5.0, s=2)]}
    groups = R.cross_match(merged)
    assert [(g["mask"], g["n_baselines"]) for g in groups] == [(0b111, 3), (0b001, 1), (0b100, 1)]
    assert merged[2][1].group == 0 and merged[2][0].group == 2


# ---------------------------------------------------------------- end to end
def test_injected_pulse_recovered_at_dm_delay_time():
    """An injected dispersed pulse (DM 557, 2 APs, SNR 20) is found on every baseline at the DM
    trial nearest 557 (560 on the 10-step grid), at the k0 of its arrival on the half-overlap
    grid, with MBD = tau_g mod t_ambig and SBD = tau_g within one grid step; cross-matching
    puts the three detections in one group, and the RFI points make no multi-baseline pulse."""
    dms = np.arange(500.0, 621.0, 10.0)
    wl = synth.make_small(T=4096, dms=dms)
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    res = R.search(st, vis, wl.dms, wl.windows, combos=[0b111])
    t0 = wl.pulses[0].t0_bin
    sbd_ax, mbd_ax = R.delay_axes(st)
    hits = []
    for b in range(wl.n_bl):
        best = max(res.pulses[b], key=lambda p: p.p)
        assert dms[best.d] == 560.0
        assert best.k0 <= t0 < best.k0 + best.l
        tau = wl.tau_g_ns[b]
        wrapped = (tau - mbd_ax[best.q] + st.t_ambig_ns / 2) % st.t_ambig_ns - st.t_ambig_ns / 2
        assert abs(wrapped) <= mbd_ax[1]
        assert abs(sbd_ax[best.m] - tau) <= sbd_ax[1]
        hits.append(best.group)
    assert len(set(hits)) == 1
    assert res.groups[hits[0]]["n_baselines"] == 3
    multi = [g for g in res.groups if g["n_baselines"] >= 2]
    assert len(multi) == 1
    comb = max(res.combined[0], key=lambda p: p.p)
    assert dms[comb.d] == 560.0 and comb.k0 <= t0 < comb.k0 + comb.l
