"""FP64 oracle of the cross-spectrum FRB search (arxiv 1801.02391).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct restatement of
the method that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It shares no code with the library and never imports it.

Every function names the passage it follows.  Where the paper is silent or
ambiguous, the reading taken is stated in the docstring (and listed in the
design notes).  The per-segment transform is in ``frbx_oracle.c`` (FP64 C);
everything else here is numpy (FP64) or pure Python.
"""
from __future__ import annotations

import dataclasses
import math
from functools import reduce

import numpy as np

from . import _clib

K_DM = 4.15e6  # Eq. 1: ms MHz^2, as printed (consistent with 2.41e-7 = 1/4.15e6 of Eq. 11)
TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------------------
# Frequency setup (Eq. 1, Eq. 5, Sec. 2.3)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Setup:
    f0_mhz: np.ndarray      # [N] subband edge frequencies
    n_point: int            # J
    f_bw_mhz: float
    t_ap_ms: float
    f_ref_dm_mhz: float     # reference of Eq. 1
    f: np.ndarray           # [N*J] point frequencies f0_n + f_j
    flag: np.ndarray        # [N*J] uint8, 1 = excluded (j = 0 is excluded separately)
    rot: np.ndarray         # [N*J] complex128 calibration rotation (Eq. 5)
    g: np.ndarray           # [N] int, (f0_n - f0_min) / df_grid
    df_grid_mhz: float
    Ls: int
    Lm: int

    @property
    def N(self):
        return int(self.f0_mhz.shape[0])

    @property
    def J(self):
        return self.n_point

    @property
    def C(self):
        return self.N * self.J

    @property
    def t_ambig_ns(self):
        return 1000.0 / self.df_grid_mhz


def _nextpow2(x: int) -> int:
    p = 1
    while p < x:
        p *= 2
    return p


def make_setup(f0_mhz, n_point, f_bw_mhz, t_ap_ms, f_ref_dm_mhz=0.0, chan_delay_ns=None,
               chan_phase_rad=None, flag=None, sbd_pad=2, mbd_pad=2) -> Setup:
    """Point frequencies, Eq. 1 reference, MBD grid and calibration rotation.

    * f(n, j) = f0_n + j f_bw / J (USB baseband points, j = 0 at the channel edge; Sec. 2.2).
    * f_ref,dm = the highest point frequency when not given ("highest frequency of
      the band", Sec. 2.2), so the top point has zero delay.
    * The MBD grid (Sec. 5.1): df_grid = GCD of the channel offsets f0_n - min f0 (in
      kHz), g_n = offset / df_grid, Lm = mbd_pad * nextpow2(max g + 1); the SBD grid
      is Ls = sbd_pad * J (zero padding, App. B).  The paper gives no grid sizes; they
      are parameters shared by both implementations.
    * Calibration rotation of Eq. 5: exp(-i [2 pi (f_j - f_bw/2) dtau0_n + dphi0_n]).
    """
    f0 = np.asarray(f0_mhz, dtype=np.float64)
    N, J = f0.shape[0], int(n_point)
    j = np.arange(J, dtype=np.float64)
    f = (f0[:, None] + (j[None, :] * f_bw_mhz) / J).reshape(-1)
    fref = float(f.max()) if not f_ref_dm_mhz else float(f_ref_dm_mhz)
    offs_khz = (f0 - f0.min()) * 1000.0
    offs_int = np.rint(offs_khz).astype(np.int64)
    if np.any(np.abs(offs_khz - offs_int) > 1e-3):
        raise ValueError("channel offsets must be whole kHz")
    nz = [int(v) for v in offs_int if v != 0]
    gcd_khz = reduce(math.gcd, nz) if nz else int(round(f_bw_mhz * 1000.0))
    g = (offs_int // gcd_khz).astype(np.int64)
    Lm = int(mbd_pad) * _nextpow2(int(g.max()) + 1)
    Ls = int(sbd_pad) * J
    dtau = np.zeros(N) if chan_delay_ns is None else np.asarray(chan_delay_ns, np.float64)
    dphi = np.zeros(N) if chan_phase_rad is None else np.asarray(chan_phase_rad, np.float64)
    fj = (j * f_bw_mhz) / J
    ph = TWO_PI * (fj[None, :] - f_bw_mhz / 2.0) * dtau[:, None] * 1e-3 + dphi[:, None]
    rot = (np.cos(ph) - 1j * np.sin(ph)).reshape(-1)
    fl = np.zeros(N * J, np.uint8) if flag is None else np.asarray(flag, np.uint8).reshape(-1).copy()
    return Setup(f0_mhz=f0, n_point=J, f_bw_mhz=float(f_bw_mhz), t_ap_ms=float(t_ap_ms),
                 f_ref_dm_mhz=fref, f=f, flag=fl, rot=rot, g=g, df_grid_mhz=gcd_khz / 1000.0,
                 Ls=Ls, Lm=Lm)


def setup_from_workload(wl, **kw) -> Setup:
    return make_setup(wl.f0_mhz, wl.n_point, wl.f_bw_mhz, wl.t_ap_ms, flag=wl.flags,
                      sbd_pad=wl.sbd_pad, mbd_pad=wl.mbd_pad, **kw)


# --------------------------------------------------------------------------------------
# Eq. 1-2: dispersion shift table
# --------------------------------------------------------------------------------------
def shift_table(st: Setup, dms) -> np.ndarray:
    """dk(d, c) = floor(0.5 + dt / t_ap), dt = 4.15e6 DM [f^-2 - f_ref^-2] (Eq. 1, Eq. 2).

    Evaluated op by op in FP64 in this order: a = 4.15e6 * DM; b = 1/(f*f) - 1/(fref*fref);
    dt = a * b; x = dt / t_ap; floor(0.5 + x).
    """
    dms = np.asarray(dms, dtype=np.float64)
    a = K_DM * dms
    b = 1.0 / (st.f * st.f) - 1.0 / (st.f_ref_dm_mhz * st.f_ref_dm_mhz)
    dt = a[:, None] * b[None, :]
    x = dt / st.t_ap_ms
    return np.floor(0.5 + x).astype(np.int32)


# --------------------------------------------------------------------------------------
# Sec. 2.4.1: half-overlapped segment lists
# --------------------------------------------------------------------------------------
def window_step(l: int) -> int:
    """Consecutive segments overlap by half (S_k0, S_{k0+l/2}, ...); l = 1 cannot, step 1."""
    return max(1, l // 2)


def n_slots(T: int, l: int) -> int:
    return (T - l) // window_step(l) + 1 if T >= l else 0


def n_valid(T: int, l: int, dk_max: int) -> int:
    """Segments whose whole dedispersed span lies inside the scan (partial ones dropped)."""
    r = T - dk_max - l
    return r // window_step(l) + 1 if r >= 0 else 0


def slot_offsets(T: int, windows) -> tuple[np.ndarray, int]:
    sizes = [n_slots(T, l) for l in windows]
    offs = np.zeros(len(windows), np.int64)
    if len(windows) > 1:
        offs[1:] = np.cumsum(sizes)[:-1]
    return offs, int(sum(sizes))


# --------------------------------------------------------------------------------------
# Eq. 3 + Eq. 5 + Sec. 5.1 (C, FP64)
# --------------------------------------------------------------------------------------
def delay_axes(st: Setup):
    """SBD / MBD value (ns) of every grid index: s(i) = i (i < L/2) else i - L;
    SBD_m = s(m) J / (Ls f_bw); MBD_q = s(q) / (Lm df_grid)  (Sec. 5.1 grid)."""
    m = np.arange(st.Ls)
    sm = np.where(m < st.Ls // 2, m, m - st.Ls).astype(np.float64)
    q = np.arange(st.Lm)
    sq = np.where(q < st.Lm // 2, q, q - st.Lm).astype(np.float64)
    sbd = ((sm * st.J) * 1000.0) / (st.Ls * st.f_bw_mhz)
    mbd = (sq * 1000.0) / (st.Lm * st.df_grid_mhz)
    return sbd, mbd


def window_masks(st: Setup, sbd_win_ns=None, mbd_win_ns=None):
    """Delay search windows: a cell is searched when lo <= delay <= hi; None = whole grid."""
    sbd, mbd = delay_axes(st)
    am = np.ones(st.Ls, np.uint8) if sbd_win_ns is None else ((sbd >= sbd_win_ns[0]) & (sbd <= sbd_win_ns[1])).astype(np.uint8)
    aq = np.ones(st.Lm, np.uint8) if mbd_win_ns is None else ((mbd >= mbd_win_ns[0]) & (mbd <= mbd_win_ns[1])).astype(np.uint8)
    return am, aq


def fit_segments(st: Setup, vis: np.ndarray, dk: np.ndarray, seg: np.ndarray, allow_m=None,
                 allow_q=None, want_grid=False, n_threads=0):
    """Fit a list of segments (rows of seg = (bl, d, l, k0)).  Returns amp, m, q, amp2 [, grid]."""
    vis = np.ascontiguousarray(vis, dtype=np.complex64)
    n_bl, T, C = vis.shape
    assert C == st.C
    return _clib.fit_list(vis, n_bl, T, st.N, st.J, np.ascontiguousarray(dk, np.int32), st.flag,
                          np.ascontiguousarray(st.rot.real), np.ascontiguousarray(st.rot.imag),
                          st.g.astype(np.int32), st.Ls, st.Lm, allow_m, allow_q,
                          np.ascontiguousarray(seg, np.int32), want_grid, n_threads)


def all_segments(T: int, n_bl: int, windows, dk_max: np.ndarray):
    """Every valid segment in series order [bl][d][window][slot] and its flat series index."""
    offs, S_tot = slot_offsets(T, windows)
    rows, idx = [], []
    n_dm = dk_max.shape[0]
    for b in range(n_bl):
        for d in range(n_dm):
            for w, l in enumerate(windows):
                nv = n_valid(T, l, int(dk_max[d]))
                if nv <= 0:
                    continue
                s = np.arange(nv, dtype=np.int64)
                r = np.empty((nv, 4), np.int32)
                r[:, 0], r[:, 1], r[:, 2], r[:, 3] = b, d, l, s * window_step(l)
                rows.append(r)
                idx.append((b * n_dm + d) * S_tot + offs[w] + s)
    if not rows:
        return np.zeros((0, 4), np.int32), np.zeros(0, np.int64), S_tot
    return np.concatenate(rows), np.concatenate(idx), S_tot


# --------------------------------------------------------------------------------------
# Eq. 6 and the threshold of Sec. 2.4.1
# --------------------------------------------------------------------------------------
def normalise(amp_series: np.ndarray, T: int, windows, dk_max: np.ndarray):
    """P = (|G| - mean|G|) / std|G| per (series, window) over the valid segments (Eq. 6).

    amp_series: [n_series][n_dm][S_tot] (n_series = baselines or combos).  The "given
    time range" is read as the whole scan; std is the population std.  A window with
    std 0 (or no segment) has P = 0.  Invalid slots get P = nan.
    """
    offs, S_tot = slot_offsets(T, windows)
    P = np.full(amp_series.shape, np.nan)
    for d in range(amp_series.shape[1]):
        for w, l in enumerate(windows):
            nv = n_valid(T, l, int(dk_max[d]))
            if nv <= 0:
                continue
            a = amp_series[:, d, offs[w]:offs[w] + nv].astype(np.float64)
            mu = a.mean(axis=1, keepdims=True)
            sd = np.sqrt(((a - mu) ** 2).mean(axis=1, keepdims=True))
            with np.errstate(invalid="ignore", divide="ignore"):
                p = np.where(sd > 0, (a - mu) / np.where(sd > 0, sd, 1.0), 0.0)
            P[:, d, offs[w]:offs[w] + nv] = p
    return P


@dataclasses.dataclass
class Cand:
    series: int      # baseline or combo index
    d: int
    w: int           # window index
    l: int           # window length
    k0: int
    amp: float
    p: float
    m: int = -1
    q: int = -1
    n_win: int = 0
    group: int = -1

    def overlaps(self, o: "Cand") -> bool:
        return self.k0 < o.k0 + o.l and o.k0 < self.k0 + self.l


def events(P: np.ndarray, amp: np.ndarray, m_idx, q_idx, T, windows, dk_max, threshold=3.0):
    """Candidate signals: segments with P > threshold (strict), Sec. 2.4.1 (threshold 3).
    Returned per (series, d) in window order then ascending k0."""
    offs, S_tot = slot_offsets(T, windows)
    out = {}
    for s in range(P.shape[0]):
        for d in range(P.shape[1]):
            lst = []
            for w, l in enumerate(windows):
                nv = n_valid(T, l, int(dk_max[d]))
                for i in range(nv):
                    j = offs[w] + i
                    p = P[s, d, j]
                    if p > threshold:
                        lst.append(Cand(series=s, d=d, w=w, l=l, k0=i * window_step(l), amp=float(amp[s, d, j]),
                                        p=float(p), m=int(m_idx[s, d, j]) if m_idx is not None else -1,
                                        q=int(q_idx[s, d, j]) if q_idx is not None else -1))
            out[(s, d)] = lst
    return out


# --------------------------------------------------------------------------------------
# Sec. 2.4.1 steps b-d, Sec. 2.4.2, Sec. 5.3 DM merge, cross-matching
# --------------------------------------------------------------------------------------
def insert_groups(items):
    """Step b insertion rule: each item joins the first existing group (creation order)
    holding a member whose time range [k0, k0+l) overlaps its own; else it opens a group.
    Groups are never merged."""
    groups = []
    for it in items:
        for grp in groups:
            if any(it.overlaps(o) for o in grp):
                grp.append(it)
                break
        else:
            groups.append([it])
    return groups


def mbd_filter(group, Lm):
    """Step c: circular mean of MBD over the group (period t_ambig, as the paper asks the
    ambiguity be taken into account), then drop members with |wrapped MBD - mean| >=
    t_ambig/4.  In grid units the angle of a member is 2 pi q / Lm."""
    sc = ss = 0.0
    for c in group:
        th = (TWO_PI * c.q) / Lm
        sc += math.cos(th)
        ss += math.sin(th)
    mu = math.atan2(ss, sc)
    keep = []
    for c in group:
        th = (TWO_PI * c.q) / Lm
        if abs(math.remainder(th - mu, TWO_PI)) < math.pi / 2:
            keep.append(c)
    return keep


def pick_pulse(group, nwin_min):
    """Step d: N_win = number of distinct window lengths; if N_win >= N_win,min the member
    of highest normalised power (first inserted on ties) is the pulse."""
    if not group:
        return None
    nw = len({c.l for c in group})
    if nw < nwin_min:
        return None
    best = group[0]
    for c in group[1:]:
        if c.p > best.p:
            best = c
    return dataclasses.replace(best, n_win=nw)


def single_series_pulses(cands, windows, nwin_min, Lm, use_mbd):
    """Steps b-d for one (series, DM): windows largest first, ascending k0 within a window."""
    order = sorted(range(len(windows)), key=lambda w: -windows[w])
    items = []
    for w in order:
        items.extend(sorted((c for c in cands if c.w == w), key=lambda c: c.k0))
    pulses = []
    for grp in insert_groups(items):
        if use_mbd:
            grp = mbd_filter(grp, Lm)
        p = pick_pulse(grp, nwin_min)
        if p is not None:
            pulses.append(p)
    return pulses


def dm_merge(pulses_by_d):
    """Sec. 5.3 coarse search: a pulse seen in several DM bins keeps the bin of highest
    power.  Pulses (DM ascending, then discovery order) are grouped by time overlap with
    the step-b rule; each group keeps its highest-P pulse (lowest DM on ties)."""
    items = [p for d in sorted(pulses_by_d) for p in pulses_by_d[d]]
    out = []
    for grp in insert_groups(items):
        best = grp[0]
        for c in grp[1:]:
            if c.p > best.p:
                best = c
        out.append(best)
    return out


def cross_match(merged_by_bl):
    """Sec. 2.4.1 cross matching: baselines ascending, pulses by ascending start; a pulse
    joins the first group holding an overlapping pulse; the group's baseline set is
    reported.  Returns (groups as lists of (bl, index)), and sets group ids in place."""
    items = []
    for b in sorted(merged_by_bl):
        lst = merged_by_bl[b]
        for i in sorted(range(len(lst)), key=lambda i: lst[i].k0):
            items.append((b, i, lst[i]))
    groups = []
    for b, i, c in items:
        for grp in groups:
            if any(c.overlaps(o) for (_, _, o) in grp):
                grp.append((b, i, c))
                break
        else:
            groups.append([(b, i, c)])
    out = []
    for gi, grp in enumerate(groups):
        for (_, _, c) in grp:
            c.group = gi
        mask = 0
        for (b, _, _) in grp:
            mask |= 1 << b
        out.append({"mask": mask, "n_baselines": bin(mask).count("1"), "members": [(b, i) for (b, i, _) in grp]})
    return out


# --------------------------------------------------------------------------------------
# Whole search
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class SearchResult:
    dk: np.ndarray
    dk_max: np.ndarray
    amp: np.ndarray          # [n_bl][n_dm][S_tot]
    amp2: np.ndarray
    m: np.ndarray
    q: np.ndarray
    P: np.ndarray
    S_tot: int
    events: dict
    pulses_dm: dict          # (bl, d) -> pulses before the DM merge
    pulses: dict             # bl -> DM-merged pulses
    groups: list
    combined: dict           # combo index -> DM-merged combined pulses
    combined_events: dict
    combo_amp: np.ndarray
    combo_P: np.ndarray


def search(st: Setup, vis: np.ndarray, dms, windows, threshold=3.0, nwin_min=3, combos=(),
           sbd_win_ns=None, mbd_win_ns=None, n_threads=0) -> SearchResult:
    """The whole hot path: Eq. 1-3, Eq. 5 on the Sec. 5.1 grid, Eq. 6, threshold,
    Sec. 2.4.1 steps b-d per (baseline, DM), Sec. 5.3 DM merge, cross matching, and the
    Sec. 2.4.2 power-summation scheme for each baseline combination (bit mask)."""
    vis = np.ascontiguousarray(vis, dtype=np.complex64)
    n_bl, T, C = vis.shape
    windows = [int(l) for l in windows]
    dk = shift_table(st, dms)
    dk_max = dk.max(axis=1)
    n_dm = dk.shape[0]
    seg, idx, S_tot = all_segments(T, n_bl, windows, dk_max)
    am, aq = window_masks(st, sbd_win_ns, mbd_win_ns)
    amp_f = np.full(n_bl * n_dm * S_tot, np.nan)
    amp2_f = np.full_like(amp_f, np.nan)
    m_f = np.full(amp_f.shape, -1, np.int32)
    q_f = np.full(amp_f.shape, -1, np.int32)
    if seg.shape[0]:
        a, mm, qq, a2 = fit_segments(st, vis, dk, seg, am, aq, n_threads=n_threads)[:4]
        amp_f[idx], m_f[idx], q_f[idx], amp2_f[idx] = a, mm, qq, a2
    shape = (n_bl, n_dm, S_tot)
    amp, amp2, m_idx, q_idx = amp_f.reshape(shape), amp2_f.reshape(shape), m_f.reshape(shape), q_f.reshape(shape)
    P = normalise(amp, T, windows, dk_max)
    ev = events(P, amp, m_idx, q_idx, T, windows, dk_max, threshold)
    pulses_dm, pulses = {}, {}
    for b in range(n_bl):
        by_d = {}
        for d in range(n_dm):
            by_d[d] = single_series_pulses(ev[(b, d)], windows, nwin_min, st.Lm, use_mbd=True)
            pulses_dm[(b, d)] = by_d[d]
        pulses[b] = dm_merge(by_d)
    groups = cross_match(pulses)
    combined, combined_ev = {}, {}
    combo_amp = np.zeros((len(combos), n_dm, S_tot))
    for ci, mask in enumerate(combos):
        members = [b for b in range(n_bl) if (int(mask) >> b) & 1]
        acc = np.zeros((n_dm, S_tot))
        for b in members:
            acc = acc + amp[b]
        combo_amp[ci] = acc
    combo_P = normalise(combo_amp, T, windows, dk_max) if len(combos) else np.zeros((0, n_dm, S_tot))
    if len(combos):
        cev = events(combo_P, combo_amp, None, None, T, windows, dk_max, threshold)
        for ci in range(len(combos)):
            by_d = {d: single_series_pulses(cev[(ci, d)], windows, nwin_min, st.Lm, use_mbd=False)
                    for d in range(n_dm)}
            combined[ci] = dm_merge(by_d)
            for d in range(n_dm):
                combined_ev[(ci, d)] = cev[(ci, d)]
    return SearchResult(dk=dk, dk_max=dk_max, amp=amp, amp2=amp2, m=m_idx, q=q_idx, P=P, S_tot=S_tot,
                        events=ev, pulses_dm=pulses_dm, pulses=pulses, groups=groups, combined=combined,
                        combined_events=combined_ev, combo_amp=combo_amp, combo_P=combo_P)


# --------------------------------------------------------------------------------------
# Closed forms the paper prints (used as pins)
# --------------------------------------------------------------------------------------
def radiometer_noise_jy(sefd1, sefd2, bw_hz, t_s):
    """Eq. 7: S_noise = sqrt(SEFD1 SEFD2 / (2 B T))."""
    return math.sqrt(sefd1 * sefd2 / (2.0 * bw_hz * t_s))


def dm_resolution(t_win_ms, f_low_mhz, f_high_mhz):
    """Eq. 11: DM_res = 2.41e-7 t_win / (f_low^-2 - f_high^-2)."""
    return 2.41e-7 * t_win_ms / (f_low_mhz ** -2 - f_high_mhz ** -2)


def coincidence_counts(groups, pulses_per_bl):
    """Counting of Tab. 3: the one-baseline column of baseline b is the number of its
    single pulses; a multi-baseline column "A & B (& C)" counts the cross-match groups
    whose baseline set contains all of them (a pulse seen on 3 baselines is also counted
    in every pair column, which is what makes the paper's 16 / 15 two-baseline totals)."""
    def count(bls):
        if len(bls) == 1:
            return pulses_per_bl.get(bls[0], 0)
        need = 0
        for b in bls:
            need |= 1 << b
        return sum(1 for g in groups if (g["mask"] & need) == need)
    return count
