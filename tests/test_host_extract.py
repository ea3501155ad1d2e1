"""The library's host extraction (steps b-d, DM merge, cross-matching; frbx_extract_events)
against the oracle's, on random and on oracle-produced event lists (no GPU)."""
import numpy as np
import pytest

import synth
from oracle import reference as R
from paper_1801_02391_gb300 import _build


@pytest.fixture(scope="module")
def frbx():
    _build.build()
    from paper_1801_02391_gb300 import frbx as f
    f.load()
    return f


def oracle_extract(ev, n_series, n_dm, windows, Lm, nwin_min, use_mbd, cross):
    by = {(s, d): [] for s in range(n_series) for d in range(n_dm)}
    for e in ev:
        w = int(e["win_idx"])
        by[(int(e["series"]), int(e["dm_idx"]))].append(
            R.Cand(series=int(e["series"]), d=int(e["dm_idx"]), w=w, l=windows[w], k0=int(e["k0"]),
                   amp=float(e["amp"]), p=float(e["pnorm"]), m=int(e["sbd_idx"]), q=int(e["mbd_idx"])))
    pre, merged = [], {}
    for s in range(n_series):
        per_d = {}
        for d in range(n_dm):
            per_d[d] = R.single_series_pulses(by[(s, d)], windows, nwin_min, Lm, use_mbd)
            pre.extend(per_d[d])
        merged[s] = R.dm_merge(per_d)
    groups = R.cross_match(merged) if cross else []
    return pre, merged, groups


def to_events(cands, frbx):
    ev = np.zeros(len(cands), frbx.EVENT_DTYPE)
    for i, c in enumerate(cands):
        ev[i] = (c["series"], c["d"], c["w"], c["k0"], c["amp"], c["p"], c["m"], c["q"])
    order = np.lexsort((ev["k0"], ev["win_idx"], ev["dm_idx"], ev["series"]))
    return ev[order]


def random_events(rng, n_series, n_dm, windows, T, Lm, density):
    cands = []
    for s in range(n_series):
        for d in range(n_dm):
            for w, l in enumerate(windows):
                step = R.window_step(l)
                for k0 in range(0, T - l + 1, step):
                    if rng.random() < density:
                        cands.append(dict(series=s, d=d, w=w, k0=k0, amp=float(rng.random() * 50),
                                          p=float(np.float32(3 + rng.exponential(2.0))), m=int(rng.integers(0, 64)),
                                          q=int(rng.integers(0, Lm))))
    return cands


def compare(frbx, ev, n_series, T, n_dm, windows, Lm, nwin_min, use_mbd, cross):
    pul, grp, pre = frbx.frbx_extract_events(ev, n_series, T, n_dm, windows, Lm if use_mbd else 0, nwin_min, cross)
    o_pre, o_merged, o_groups = oracle_extract(ev, n_series, n_dm, windows, Lm, nwin_min, use_mbd, cross)
    key = lambda p: (p.series, p.d, p.w, p.k0, p.m, p.q, p.n_win)
    assert [tuple(int(x) for x in (r["series"], r["dm_idx"], r["win_idx"], r["k0"], r["sbd_idx"], r["mbd_idx"], r["n_win"]))
            for r in pre] == [key(p) for p in o_pre]
    flat = [p for s in range(n_series) for p in o_merged[s]]
    assert [tuple(int(x) for x in (r["series"], r["dm_idx"], r["win_idx"], r["k0"], r["n_win"])) for r in pul] == \
        [(p.series, p.d, p.w, p.k0, p.n_win) for p in flat]
    np.testing.assert_array_equal(pul["pnorm"], np.array([p.p for p in flat], np.float32))
    if cross:
        assert [int(g) for g in pul["group"]] == [p.group for p in flat]
        assert [(int(g["bl_mask"]), int(g["n_baselines"]), int(g["n_pulses"])) for g in grp] == \
            [(g["mask"], g["n_baselines"], len(g["members"])) for g in o_groups]
    return len(pul)


@pytest.mark.parametrize("seed", range(6))
def test_random_event_lists(frbx, seed):
    rng = np.random.default_rng(100 + seed)
    windows = [[2, 4, 8, 16], [16, 4, 1, 8, 2], [4, 8, 16, 24, 32]][seed % 3]
    T, n_series, n_dm, Lm = 300, 3, 4, 16
    cands = random_events(rng, n_series, n_dm, windows, T, Lm, density=0.04)
    ev = to_events(cands, frbx)
    n = compare(frbx, ev, n_series, T, n_dm, windows, Lm, 2 + seed % 2, use_mbd=True, cross=True)
    n += compare(frbx, ev, n_series, T, n_dm, windows, Lm, 3, use_mbd=False, cross=False)
    assert n > 0


def test_empty_and_invalid(frbx):
    ev = np.zeros(0, frbx.EVENT_DTYPE)
    pul, grp, pre = frbx.frbx_extract_events(ev, 2, 100, 3, [2, 4], 16)
    assert pul.size == grp.size == pre.size == 0
    bad = np.zeros(2, frbx.EVENT_DTYPE)
    bad["k0"] = [5, 3]          # out of order
    with pytest.raises(frbx.FrbxError):
        frbx.frbx_extract_events(bad, 1, 100, 1, [2], 16)
    bad["k0"] = [3, 500]        # k0 >= T
    with pytest.raises(frbx.FrbxError):
        frbx.frbx_extract_events(bad, 1, 100, 1, [2], 16)


def test_oracle_event_lists_of_the_small_workload(frbx):
    """Events the oracle finds on a slice of the small workload (pulse, RFI, noise) give the
    same pulses, merged pulses and groups through the library's extraction."""
    dms = np.arange(530.0, 591.0, 10.0)
    wl = synth.make_small(T=3000, dms=dms)
    st = R.setup_from_workload(wl)
    vis = synth.generate(wl)
    res = R.search(st, vis, wl.dms, wl.windows)
    rows = []
    for (s, d), lst in sorted(res.events.items()):
        for c in lst:
            rows.append(dict(series=s, d=d, w=c.w, k0=c.k0, amp=c.amp, p=float(np.float32(c.p)), m=c.m, q=c.q))
    ev = to_events(rows, frbx)
    assert ev.size > 100
    compare(frbx, ev, wl.n_bl, wl.T, len(dms), wl.windows, st.Lm, 3, use_mbd=True, cross=True)


def test_large_event_list_split_across_threads(frbx):
    """More than 50,000 events: the library splits the series across host threads; pulses,
    merged pulses and groups must still equal the oracle's single pass."""
    rng = np.random.default_rng(7)
    windows = [2, 4, 8, 16]
    T, n_series, n_dm, Lm = 1200, 12, 3, 16
    cands = random_events(rng, n_series, n_dm, windows, T, Lm, density=0.65)
    ev = to_events(cands, frbx)
    assert ev.size > 50000
    n = compare(frbx, ev, n_series, T, n_dm, windows, Lm, 3, use_mbd=True, cross=True)
    # the combined-series form (no step c, no cross-matching) takes the same split
    n += compare(frbx, ev, n_series, T, n_dm, windows, Lm, 3, use_mbd=False, cross=False)
    assert n > 0
