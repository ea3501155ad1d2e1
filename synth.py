"""Seeded synthetic cross-spectrum cubes shaped like the paper's observing setups.

This module only makes *inputs*: circular complex Gaussian noise, dispersed
pulses and RFI, written into a complex64 cube ``vis[bl][k][n*J + j]`` (baseline,
AP, frequency point; point-fastest).  It holds no part of the search method:
the dispersion delay used for injection is the physical cold-plasma law with
the literature constant 4.148808e6 ms MHz^2 (the search itself uses the
paper's rounded 4.15e6, Eq. 1), pulses are boxcars on the AP grid, and random
draws come from numpy's PCG64 seeded per (workload, component, baseline).

Both the CUDA path and the oracle consume exactly the bytes made here.

Workloads (the paper measures on the psrf02 pulsar data, which is not
available; these stand in for it with the paper's shapes):

* ``small``  -- 3 baselines, 8 x 32 MHz subbands x 32 points at 1400-1656 MHz
  (the paper's S-band layout of Sec. 3.1 scaled to 8 subbands), 1 ms APs,
  T = 4096, DM 0..1000 step 10, one pulse (DM 557, 2 APs, SNR 20), two RFI
  points at 30x power.
* ``vgos``   -- 15 baselines, 4 bands x 8 subbands x 32 MHz x 64 points between
  3.0 and 10.7 GHz (the VGOS setup of Sec. 4), 0.5 ms APs, T = 20000,
  512 DM trials 0..2000, five pulses, 5 % of the points flagged and carrying
  RFI.
* ``batch``  -- many scans for the batched search: 16 scans of uneven length
  (1-30 s at 1 ms APs), 45 baselines (10 stations), each scan on one of three
  setups (256 points: the small layout; 1024 points: the two lower VGOS bands;
  2048 points: all four VGOS bands), 256 DM trials 0..1500, a pulse in a quarter
  of the scans.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1801_02391
K_DM_PHYS = 4.148808e6  # ms MHz^2 per (pc cm^-3); physical constant for injection only

_COMPONENTS = {"noise": 1, "pulse": 2, "rfi": 3, "flags": 4, "geometry": 5}


def seed_for(workload_id: int, component: str, index: int = 0) -> int:
    return SEED_BASE + 1000 * workload_id + 100 * _COMPONENTS[component] + index


@dataclasses.dataclass
class Pulse:
    dm: float          # pc cm^-3
    t0_bin: int        # arrival AP at the top frequency of the band
    width: int         # APs
    snr: float         # per-baseline coherent SNR (a * sqrt(width * n_used_points))


@dataclasses.dataclass
class Workload:
    name: str
    workload_id: int
    n_bl: int
    f0_mhz: np.ndarray          # [N] lower edge of each subband (USB)
    n_point: int                # J
    f_bw_mhz: float
    t_ap_ms: float
    T: int
    dms: np.ndarray             # [n_dm]
    windows: list
    sbd_pad: int = 2
    mbd_pad: int = 2
    flags: np.ndarray | None = None   # [N*J] uint8, 1 = flagged
    pulses: list = dataclasses.field(default_factory=list)
    rfi_points: list = dataclasses.field(default_factory=list)  # (n, j)
    rfi_power: float = 30.0
    tau_g_ns: np.ndarray | None = None     # [n_bl] geometric residual delay
    rate_mhz: np.ndarray | None = None     # [n_bl] fringe rate in mHz
    phase0: np.ndarray | None = None       # [n_bl] fringe phase

    @property
    def n_chan(self) -> int:
        return int(self.f0_mhz.shape[0])

    @property
    def C(self) -> int:
        return self.n_chan * self.n_point

    def point_freqs(self) -> np.ndarray:
        """Sky frequency of every point, [N*J], MHz (channel edge + j*f_bw/J)."""
        j = np.arange(self.n_point, dtype=np.float64)
        return (self.f0_mhz[:, None] + (j[None, :] * self.f_bw_mhz) / self.n_point).reshape(-1)


def _noise(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex Gaussian, E|z|^2 = 1 (re, im ~ N(0, 1/2))."""
    out = np.empty(shape + (2,), dtype=np.float32)
    rng.standard_normal(out.shape, dtype=np.float32, out=out)
    out *= np.float32(math.sqrt(0.5))
    return out.view(np.complex64)[..., 0]


def make_small(T: int = 4096, n_bl: int = 3, dms=None, seed_offset: int = 0) -> Workload:
    wid = 1 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed_for(wid, "geometry")))
    f0 = 1400.0 + 32.0 * np.arange(8)
    wl = Workload(
        name="small", workload_id=wid, n_bl=n_bl, f0_mhz=f0, n_point=32, f_bw_mhz=32.0,
        t_ap_ms=1.0, T=T, dms=np.arange(0, 1001, 10, dtype=np.float64) if dms is None else np.asarray(dms, np.float64),
        windows=[2, 4, 8, 16],
    )
    wl.tau_g_ns = rng.uniform(1.0, 50.0, n_bl)
    wl.rate_mhz = rng.uniform(-5.0, 5.0, n_bl)
    wl.phase0 = rng.uniform(0.0, 2 * math.pi, n_bl)
    t_lo, t_hi = 800, min(3000, T - 700)
    t0 = int(rng.integers(t_lo, t_hi)) if t_hi > t_lo else T // 8
    wl.pulses = [Pulse(dm=557.0, t0_bin=t0, width=2, snr=20.0)]
    rr = np.random.Generator(np.random.PCG64(seed_for(wid, "rfi")))
    wl.rfi_points = [(int(rr.integers(0, 8)), int(rr.integers(1, 32))) for _ in range(2)]
    return wl


def make_vgos(T: int = 20000, n_bl: int = 15, n_dm: int = 512, seed_offset: int = 0) -> Workload:
    wid = 2 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed_for(wid, "geometry")))
    bands = [3000.0, 5464.0, 7960.0, 10424.0]
    f0 = np.array([b + 32.0 * i for b in bands for i in range(8)])
    wl = Workload(
        name="vgos", workload_id=wid, n_bl=n_bl, f0_mhz=f0, n_point=64, f_bw_mhz=32.0,
        t_ap_ms=0.5, T=T, dms=np.linspace(0.0, 2000.0, n_dm), windows=[1, 2, 4, 8, 16, 32],
    )
    wl.tau_g_ns = rng.uniform(1.0, 50.0, n_bl)
    wl.rate_mhz = rng.uniform(-5.0, 5.0, n_bl)
    wl.phase0 = rng.uniform(0.0, 2 * math.pi, n_bl)
    pulses = []
    t_hi = max(2, T - 2200)
    for _ in range(5):
        pulses.append(Pulse(dm=float(rng.uniform(100.0, 1900.0)),
                            t0_bin=int(rng.integers(min(500, t_hi - 1), t_hi)),
                            width=int(rng.integers(1, 11)), snr=float(rng.uniform(8.0, 30.0))))
    wl.pulses = pulses
    fr = np.random.Generator(np.random.PCG64(seed_for(wid, "flags")))
    flags = (fr.random(wl.C) < 0.05).astype(np.uint8)
    wl.flags = flags
    wl.rfi_points = [(int(c // wl.n_point), int(c % wl.n_point)) for c in np.flatnonzero(flags)]
    return wl


def make_tiny(n_chan=3, n_point=8, T=64, n_bl=2, dms=(0.0, 150.0, 400.0), windows=(1, 2, 4),
              f0=None, f_bw=16.0, t_ap=1.0, seed_offset=0, pulse=True) -> Workload:
    """Small irregular setups for parity sweeps (ragged sizes, uneven channel grid)."""
    wid = 7 + seed_offset
    rng = np.random.Generator(np.random.PCG64(seed_for(wid, "geometry")))
    if f0 is None:
        f0 = 800.0 + f_bw * np.array(sorted(rng.choice(np.arange(12), n_chan, replace=False)), dtype=np.float64)
    wl = Workload(name="tiny", workload_id=wid, n_bl=n_bl, f0_mhz=np.asarray(f0, np.float64), n_point=n_point,
                  f_bw_mhz=f_bw, t_ap_ms=t_ap, T=T, dms=np.asarray(dms, np.float64), windows=list(windows))
    wl.tau_g_ns = rng.uniform(1.0, 50.0, n_bl)
    wl.rate_mhz = rng.uniform(-5.0, 5.0, n_bl)
    wl.phase0 = rng.uniform(0.0, 2 * math.pi, n_bl)
    if pulse:
        wl.pulses = [Pulse(dm=float(dms[-1]) * 0.9, t0_bin=int(T // 4), width=2, snr=25.0)]
    return wl


def used_points(wl: Workload) -> int:
    n = wl.n_chan * (wl.n_point - 1)
    if wl.flags is not None:
        fl = wl.flags.reshape(wl.n_chan, wl.n_point)[:, 1:]
        n -= int(fl.sum())
    return n


def generate_baseline(wl: Workload, b: int) -> np.ndarray:
    """Cube of one baseline, [T][N*J] complex64."""
    C = wl.C
    rng = np.random.Generator(np.random.PCG64(seed_for(wl.workload_id, "noise", b)))
    cube = _noise(rng, (wl.T, C))
    if wl.rfi_points:
        rr = np.random.Generator(np.random.PCG64(seed_for(wl.workload_id, "rfi", 10 + b)))
        cols = np.array(sorted({n * wl.n_point + j for (n, j) in wl.rfi_points}), dtype=np.int64)
        extra = _noise(rr, (wl.T, cols.size)) * np.float32(math.sqrt(wl.rfi_power))
        cube[:, cols] += extra
    if wl.pulses:
        f = wl.point_freqs()
        f_top = float(f.max())
        m_used = used_points(wl)
        t_k = np.arange(wl.T, dtype=np.float64) * wl.t_ap_ms * 1e-3
        for p in wl.pulses:
            a = p.snr / math.sqrt(p.width * m_used)
            delay_ms = K_DM_PHYS * p.dm * (f ** -2 - f_top ** -2)
            start = p.t0_bin + np.rint(delay_ms / wl.t_ap_ms).astype(np.int64)
            for c in range(C):
                k_lo = int(start[c])
                k_hi = min(wl.T, k_lo + p.width)
                if k_lo >= wl.T or k_hi <= 0:
                    continue
                k_lo = max(0, k_lo)
                ks = np.arange(k_lo, k_hi)
                phase = (2 * math.pi * (f[c] - wl.f0_mhz[0]) * wl.tau_g_ns[b] * 1e-3
                         + 2 * math.pi * wl.rate_mhz[b] * 1e-3 * (f[c] / wl.f0_mhz[0]) * t_k[ks]
                         + wl.phase0[b])
                cube[ks, c] += (a * np.exp(1j * phase)).astype(np.complex64)
    return cube


def generate(wl: Workload) -> np.ndarray:
    """Whole cube, [n_bl][T][N*J] complex64 (C-contiguous)."""
    out = np.empty((wl.n_bl, wl.T, wl.C), dtype=np.complex64)
    for b in range(wl.n_bl):
        out[b] = generate_baseline(wl, b)
    return out


def generate_device(wl: Workload, device="cuda"):
    """The same recipe as generate() made on the GPU with torch's seeded generator (a different
    random stream from numpy's PCG64, so the values differ from generate()'s): circular complex
    Gaussian noise with E|z|^2 = 1, extra noise at rfi_power on the RFI points, boxcar pulses with
    the physical dispersion delay and the baseline's geometric phase and fringe rate.  For
    workloads too large to make on the host in reasonable time (the batched workload at full
    size); returns a complex64 CUDA tensor [n_bl][T][N*J]."""
    import torch
    g = torch.Generator(device=device)
    out = torch.empty((wl.n_bl, wl.T, wl.C), dtype=torch.complex64, device=device)
    f = wl.point_freqs()
    cols = (np.array(sorted({n * wl.n_point + j for (n, j) in wl.rfi_points}), dtype=np.int64)
            if wl.rfi_points else np.zeros(0, np.int64))
    cols_t = torch.from_numpy(cols).to(device)
    for b in range(wl.n_bl):
        g.manual_seed(seed_for(wl.workload_id, "noise", b))
        torch.view_as_real(out[b]).normal_(0.0, math.sqrt(0.5), generator=g)
        if cols.size:
            g.manual_seed(seed_for(wl.workload_id, "rfi", 10 + b))
            extra = torch.empty((wl.T, cols.size, 2), dtype=torch.float32, device=device)
            extra.normal_(0.0, math.sqrt(0.5 * wl.rfi_power), generator=g)
            out[b][:, cols_t] += torch.view_as_complex(extra)
        if wl.pulses:
            f_top = float(f.max())
            m_used = used_points(wl)
            for p in wl.pulses:
                a = p.snr / math.sqrt(p.width * m_used)
                delay_ms = K_DM_PHYS * p.dm * (f ** -2 - f_top ** -2)
                start = p.t0_bin + np.rint(delay_ms / wl.t_ap_ms).astype(np.int64)
                ks = (start[:, None] + np.arange(p.width)[None, :]).reshape(-1)
                cs = np.repeat(np.arange(wl.C), p.width)
                ok = (ks >= 0) & (ks < wl.T)
                ks, cs = ks[ok], cs[ok]
                t_k = ks * wl.t_ap_ms * 1e-3
                phase = (2 * math.pi * (f[cs] - wl.f0_mhz[0]) * wl.tau_g_ns[b] * 1e-3
                         + 2 * math.pi * wl.rate_mhz[b] * 1e-3 * (f[cs] / wl.f0_mhz[0]) * t_k + wl.phase0[b])
                val = torch.from_numpy((a * np.exp(1j * phase)).astype(np.complex64)).to(device)
                out[b].index_put_((torch.from_numpy(ks).to(device), torch.from_numpy(cs).to(device)), val,
                                  accumulate=True)
    return out


def pure_tone_segment(wl: Workload, tau_ns: float, amp: float = 1.0) -> np.ndarray:
    """Noise-free [N*J] spectrum a*exp(2 pi i (f - f0[0]) tau) for transform pins."""
    f = wl.point_freqs()
    return (amp * np.exp(2j * math.pi * (f - wl.f0_mhz[0]) * tau_ns * 1e-3)).astype(np.complex128)


BATCH_SETUPS = ("c256", "c1024", "c2048")


def _batch_setup(kind: str, wid: int, T: int, n_bl: int, dms) -> Workload:
    if kind == "c256":
        f0, J = 1400.0 + 32.0 * np.arange(8), 32
    else:
        bands = [3000.0, 5464.0] if kind == "c1024" else [3000.0, 5464.0, 7960.0, 10424.0]
        f0, J = np.array([b + 32.0 * i for b in bands for i in range(8)]), 64
    wl = Workload(name=kind, workload_id=wid, n_bl=n_bl, f0_mhz=f0, n_point=J, f_bw_mhz=32.0, t_ap_ms=1.0, T=T,
                  dms=np.asarray(dms, np.float64), windows=[2, 4, 8, 16])
    if kind != "c256":  # the VGOS-like setups carry 5 % flagged points; one flag set per setup
        fr = np.random.Generator(np.random.PCG64(seed_for(30 + BATCH_SETUPS.index(kind), "flags")))
        wl.flags = (fr.random(wl.C) < 0.05).astype(np.uint8)
        wl.rfi_points = [(int(c // J), int(c % J)) for c in np.flatnonzero(wl.flags)]
    else:
        fr = np.random.Generator(np.random.PCG64(seed_for(30, "rfi")))
        wl.rfi_points = [(int(fr.integers(0, 8)), int(fr.integers(1, J))) for _ in range(2)]
    return wl


def make_batch(n_scans: int = 16, n_bl: int = 45, n_dm: int = 256, t_scale: float = 1.0,
               seed_offset: int = 0) -> list:
    """The batched-search workload: a list of Workloads, one per scan (``name`` is the
    scan's setup, so scans with equal names share one setup)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(20 + seed_offset, "geometry")))
    dms = np.linspace(0.0, 1500.0, n_dm)
    kinds = [BATCH_SETUPS[int(k)] for k in rng.integers(0, 3, n_scans)]
    lengths = [max(64, int(round(rng.uniform(1.0, 30.0) * 1000.0 * t_scale))) for _ in range(n_scans)]
    with_pulse = set(int(i) for i in rng.choice(n_scans, max(1, n_scans // 4), replace=False))
    out = []
    for s in range(n_scans):
        wl = _batch_setup(kinds[s], 100 + 20 * seed_offset + s, lengths[s], n_bl, dms)
        wl.tau_g_ns = rng.uniform(1.0, 50.0, n_bl)
        wl.rate_mhz = rng.uniform(-5.0, 5.0, n_bl)
        wl.phase0 = rng.uniform(0.0, 2 * math.pi, n_bl)
        if s in with_pulse:
            T = lengths[s]
            wl.pulses = [Pulse(dm=float(rng.uniform(100.0, 1400.0)), t0_bin=int(rng.integers(0, max(1, T // 2))),
                               width=int(rng.integers(1, 11)), snr=float(rng.uniform(8.0, 30.0)))]
        out.append(wl)
    return out
