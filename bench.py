#!/usr/bin/env python3
"""Throughput of the cross-spectrum FRB search: dedispersed fringe-search cells/s.

cells = baselines x DM trials x APs x frequency points (nominal, every AP counted).
One step = one frbx_search call: shift table, every half-overlapped segment of every
window / baseline / DM fitted on the SBD x MBD grid, Eq. 6 + threshold, single-pulse
extraction, DM merge, cross-matching and the all-baseline power sum.

Default workload ("vgos"): 15 baselines, 4 bands x 8 subbands x 32 MHz x 64 points
(2048 points), 0.5 ms APs, T = 20000, 512 DM trials 0..2000, windows 1..32 APs,
synthetic seeded data (synth.make_vgos).  The cube (4.9 GB) is larger than L2.

--gpus N > 1 (under torchrun): N independent replicas of the whole search, one per GPU
(the method has no exchange step between them); value = all ranks' cells / slowest time.
--impl reference: the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# DRAM bytes per fitted segment of the per-segment fit kernel (None: no capture of the
# current kernel).
FIT_DRAM_BYTES_PER_SEGMENT = None
# dram__bytes_read.sum + dram__bytes_write.sum of one k_tree_mbd launch per (series, AP) it
# covers, from an ncu capture of the vgos-profile workload; None: k_tree_mbd has changed since
# its last capture
TREE_MBD_DRAM_BYTES_PER_AP = None
# the same for k_tree_mma (the tensor-core MBD pass, 2048-AP time tiles): 2.701 + 0.009 GB over
# 4 x 20000 series-APs
TREE_MMA_DRAM_BYTES_PER_AP = (2.700700e9 + 0.009359e9) / (4 * 20000)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def measured_peaks():
    """HBM GB/s and BF16 TFLOP/s measured on this machine (MEASURED_PEAKS.json), else fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return {k: float(d[k]) for k in FALLBACK_PEAKS}, "measured"
    except (OSError, KeyError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


def measure_peaks(stream):
    """This GPU's own peak rates (libfrbx_peaks): the FP32 FMA pipe (scalar and packed f32x2)
    and the dense BF16 / E4M3 tcgen05 MMA, each as a burst (a few ms) and, for the MMAs, as a
    sustained run of about 1.5 s; TFLOP/s with 2 flop per multiply-add."""
    from paper_1801_02391_gb300 import peaks
    out = {}
    for k, it in (("fp32_fma", 20000), ("fp32_fma2", 20000)):
        out[k] = peaks.probe(k, it, stream)[0]
    for k, it in (("bf16_mma", 4000), ("fp8_mma", 4000)):
        tf, ms = peaks.probe(k, it, stream)
        out[k] = tf
        out[k + "_sustained"] = peaks.probe(k, max(1, int(it * 1500.0 / max(ms, 1e-3))), stream)[0]
    out["fp32"] = max(out["fp32_fma"], out["fp32_fma2"])
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="frbx", choices=["frbx", "reference"])
    ap.add_argument("--workload", default="vgos", choices=["vgos", "small", "vgos-slice", "vgos-profile", "vgos-dm8"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--e2e-warmup", type=int, default=1, help="untimed host-input steps before the e2e timing")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", type=int, default=0)
    ap.add_argument("--no-variants", action="store_true", help="skip the tensor-core and batched variants")
    ap.add_argument("--batch-bl", type=int, default=45, help="baselines per scan of the batched variant (config 3: 45)")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="scan-length factor of the batched variant (config 3: 1)")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--variant-steps", type=int, default=2, help="timed steps of each variant")
    return ap.parse_args()


def make_workload(name):
    if name == "vgos":
        wl = synth.make_vgos()
        combos = [(1 << wl.n_bl) - 1]
    elif name == "vgos-profile":  # one baseline of the VGOS cube (328 MB > L2), 4 DM trials
        wl = synth.make_vgos(n_bl=1, n_dm=4)
        combos = [1]
    elif name == "vgos-dm8":     # one baseline, 8 neighbouring DM trials of the 512-trial grid (as
        wl = synth.make_vgos(T=10000, n_bl=1, n_dm=512)  # within a chunk), cube 164 MB > L2
        wl.dms = wl.dms[256:264].copy()
        combos = [1]
    elif name == "vgos-slice":   # small case of the same kernel, for profiler captures
        wl = synth.make_vgos(T=2400, n_bl=1, n_dm=8)
        wl.dms = np.linspace(0.0, 200.0, 8)
        combos = [1]
    else:
        wl = synth.make_small()
        combos = [0b111, 0b011, 0b101, 0b110]
    return wl, combos


def workload_config(name, wl):
    return {"workload": f"{name}: {wl.n_bl} baselines x {len(wl.dms)} DM trials x {wl.T} APs x {wl.C} points "
                        f"({wl.n_chan} subbands x {wl.n_point}), windows {wl.windows}",
            "n_bl": wl.n_bl, "n_dm": int(len(wl.dms)), "T": wl.T, "n_point_total": wl.C,
            "windows": wl.windows, "l2_flush": "inputs larger than L2 (cube %.2f GB)" % (wl.n_bl * wl.T * wl.C * 8 / 1e9)}


def run_batch_variant(frbx, torch, stream, n_bl, t_scale, steps, barrier, cpu_seconds=0.0):
    """The batched search (config 3: many scans of uneven length on three setups) through
    frbx_search_batch.  At full size (n_bl 45, t_scale 1: 131 GB of cube, made on the GPU by
    synth.generate_device) one call is timed: it includes the time-tile tuning and the graph
    capture of the fit (well under 1 % of the call).  Scaled down, one untimed call tunes and
    captures, then `steps` timed calls replay the captured fit."""
    wls = synth.make_batch(n_bl=n_bl, t_scale=t_scale)
    full = n_bl == 45 and t_scale == 1.0
    handles, scans = {}, []
    for wl in wls:
        if wl.name not in handles:
            handles[wl.name] = frbx.Handle.from_workload(wl)
        vis = synth.generate_device(wl) if full else torch.from_numpy(synth.generate(wl)).cuda()
        scans.append((handles[wl.name], vis))
    torch.cuda.synchronize()
    dms, windows = wls[0].dms, wls[0].windows
    cells = sum(float(wl.n_bl) * len(wl.dms) * wl.T * wl.C for wl in wls)
    with frbx.Batch() as b:
        if not full:
            b.search(scans, dms, windows, stream=stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fit, launches = [], 0
        n_steps = 1 if full else steps
        e0.record(stream)
        for _ in range(n_steps):
            outs = b.search(scans, dms, windows, stream=stream)
            info = b.info()
            fit.append(info["fit_ms"])
            launches += info["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n_steps
    kinds = {}
    for wl in wls:
        kinds[wl.name] = kinds.get(wl.name, 0) + 1
    res = {"value": cells / (ms / 1e3), "unit": "cells/s", "ms_per_step": ms, "steps": n_steps,
           "warmup": 0 if full else 1, "fit_ms": statistics.mean(fit), "gpu_launches": launches,
           "workload": f"config 3{'' if full else ' scaled'}: {len(wls)} scans x {n_bl} baselines, "
                       f"T {min(w.T for w in wls)}..{max(w.T for w in wls)} APs (1-30 s x {t_scale} at 1 ms), "
                       f"setups {kinds}, {len(dms)} DM trials 0..1500, windows {windows}",
           "data": "synthetic, made on the GPU (synth.generate_device)" if full else "synthetic (synth.generate)",
           "cube_gb": sum(w.n_bl * w.T * w.C * 8 for w in wls) / 1e9, "cells": cells,
           "time_tile": info["time_tile"], "graph_captures": info["graph_captures"],
           "graph_replays": info["graph_replays"],
           "pulses": int(sum(o["counts"]["pulses"] for o in outs)), "dtype": "f32 (bf16x3 split tensor-core MBD "
                                                                              "transform on the 1024/2048-point setups)"}
    if cpu_seconds > 0:
        # the oracle on a bounded sample of the same data: baseline 0 of the first 2048-point scan
        i0 = next(i for i, w in enumerate(wls) if w.name == "c2048")
        wl0 = wls[i0]
        vis0 = scans[i0][1][0].cpu().numpy()
        v, cores, desc, _ = run_oracle_sample(wl0, vis0, cpu_seconds)
        res["cpu_baseline"] = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle",
                               "sample": f"scan {i0} (2048 points, T {wl0.T}): " + desc}
    del scans, outs
    torch.cuda.empty_cache()
    return res


def cells_of(wl):
    return float(wl.n_bl) * len(wl.dms) * wl.T * wl.C


def n_segments(wl, dk_max):
    tot = 0
    for d in range(len(wl.dms)):
        for l in wl.windows:
            r = wl.T - int(dk_max[d]) - l
            if r >= 0:
                tot += r // max(1, l // 2) + 1
    return tot * wl.n_bl


def fft_flops_per_segment(N, Ls, Lm):
    """Algorithmic work of the 2-D FFT form of Sec. 5.1: N FFTs of Ls, Ls FFTs of Lm
    (5 L log2 L each), plus |G|^2 and the compare (3 per cell)."""
    return N * 5 * Ls * math.log2(Ls) + Ls * 5 * Lm * math.log2(Lm) + 3 * Ls * Lm


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float) -> float:
    """Largest value of x over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample_rows(wl, dk_max, n_dm_s, ts):
    """Segments of baseline 0, n_dm_s DM trials spread over the grid, APs [0, ts)."""
    from oracle import reference as R
    ds = np.unique(np.linspace(0, len(wl.dms) - 1, n_dm_s).round().astype(int))
    rows = []
    for d in ds:
        for l in wl.windows:
            nv = R.n_valid(wl.T, l, int(dk_max[d]))
            step = R.window_step(l)
            for s in range(nv):
                if s * step >= ts:
                    break
                rows.append((0, int(d), l, s * step))
    return np.array(rows, np.int32), len(ds)


def run_oracle_sample(wl, vis0, target_s):
    """Time the oracle's fit on a bounded sample; returns cells/s, cores, description."""
    from oracle import reference as R
    from oracle import _clib
    st = R.setup_from_workload(wl)
    dk = R.shift_table(st, wl.dms)
    dk_max = dk.max(axis=1)
    cube = vis0[None]
    n_dm_s = 16
    ts = 16
    rows, nd = oracle_sample_rows(wl, dk_max, n_dm_s, ts)
    t0 = time.perf_counter()
    R.fit_segments(st, cube, dk, rows)
    pilot = time.perf_counter() - t0
    ts = int(max(16, min(wl.T, ts * target_s / max(pilot, 1e-3))))
    rows, nd = oracle_sample_rows(wl, dk_max, n_dm_s, ts)
    t0 = time.perf_counter()
    R.fit_segments(st, cube, dk, rows)
    dt = time.perf_counter() - t0
    cells = 1.0 * nd * ts * wl.C
    desc = (f"oracle FP64 fit of baseline 0, {nd} of {len(wl.dms)} DM trials, APs [0, {ts}) of {wl.T}, all "
            f"{len(wl.windows)} windows: {rows.shape[0]} segments in {dt:.1f} s "
            "(normalisation and extraction excluded: <1% of its time)")
    return cells / dt, _clib.num_threads(), desc, dt


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl, combos = make_workload(args.workload)
    cfg = workload_config(args.workload, wl)
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
    metric = "dedispersed fringe-search cells/s (bl x DM x bin x chan)"

    if args.impl == "reference":
        if rank != 0:
            return 0
        vis0 = synth.generate_baseline(wl, 0)
        per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
        vals = []
        for i in range(args.warmup + args.steps):
            v, cores, desc, dt = run_oracle_sample(wl, vis0, per_step)
            if i >= args.warmup:
                vals.append((v, dt))
        v = statistics.median(x for x, _ in vals)
        ms = statistics.mean(dt for _, dt in vals) * 1e3
        line = {"impl": "reference", "metric": metric, "value": v, "unit": "cells/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, synth.py)",
                "config": cfg, "cpu_baseline": {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle",
                                                "sample": desc},
                "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1801_02391_gb300 import _build
    _build.build()
    from paper_1801_02391_gb300 import frbx

    t_gen = time.perf_counter()
    vis_host = synth.generate(wl)
    t_gen = time.perf_counter() - t_gen
    vis_pinned = torch.from_numpy(vis_host).pin_memory()
    vis_dev = vis_pinned.to("cuda", non_blocking=False)
    stream = torch.cuda.current_stream()
    h = frbx.Handle.from_workload(wl)
    dk_max = h.shift_table(wl.dms).max(axis=1)
    n_seg = n_segments(wl, dk_max)
    cells = cells_of(wl)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def step(vis):
        return h.search(vis, wl.dms, wl.windows, combos=combos, kernel=args.kernel, stream=stream)

    line_peaks = measure_peaks(stream)
    for _ in range(args.warmup):
        out = step(vis_dev)
    barrier()
    clk = Clocks(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fit_ms, mbd_ms, launches = [], [], 0
    ev0.record(stream)
    for _ in range(args.steps):
        out = step(vis_dev)
        st_ = h.stage_times()
        fit_ms.append(st_["fit"])
        mbd_ms.append(st_["tree_mbd_kernels"])
        launches += out["launches"]
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    stages = h.stage_times()
    ms = max_over_ranks(ms)
    value = world * cells / (ms / 1e3)

    # end to end through the public API from pinned host memory (the warm-up sizes the handle's
    # device copy of the cube, as the device-input warm-up sized everything else)
    for _ in range(max(0, args.e2e_warmup)):
        step(vis_pinned)
    e2e_ms = []
    h2d = wl.n_bl * wl.T * wl.C * 8
    d2h = 0
    for _ in range(max(1, args.e2e_steps)):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        o = step(vis_pinned)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        d2h = 4 * len(wl.dms) + 16 + 28 * o["counts"]["events_baseline"] + \
            28 * (o["counts"]["events"] - o["counts"]["events_baseline"]) + 16 * (1 + len(combos))
    e2e = max_over_ranks(statistics.mean(e2e_ms))

    peaks, peaks_kind = measured_peaks()
    own = line_peaks  # this GPU's own probes, measured before the warm-up
    seg_flop = fft_flops_per_segment(wl.n_chan, h.Ls, h.Lm)
    flops = n_seg * seg_flop
    fit_mean = statistics.mean(fit_ms)
    tree = stages["tree_chunks"] > 0
    tc = tree and stages["tree_tensor"] > 0
    hbm_frac = (8.0 * cells / (ms / 1e3)) / (peaks["hbm_gbs"] * 1e9)
    bf16_peak = peaks["bf16_tflops_sustained"]
    if tree:
        # dominant kernel: the MBD pass of the window-tree fit (k_tree_mma on the tensor cores,
        # or k_tree_mbd on the CUDA cores), timed per chunk with CUDA events on the library's
        # stream it runs on; it emits every segment
        kms = statistics.mean(mbd_ms)
        achieved = flops / (kms / 1e3) / 1e12
        n_ap = wl.n_bl * sum(max(0, wl.T - int(x)) for x in dk_max)
        n_l1 = n_ap if 1 in wl.windows else 0
        epilogue = (n_seg - n_l1) * 2 * h.Ls * h.Lm + n_seg * 3 * h.Ls * h.Lm
        launches_ = max(1, int(stages["tree_chunks"]))
        per_ap = TREE_MMA_DRAM_BYTES_PER_AP if tc else TREE_MBD_DRAM_BYTES_PER_AP
        traffic = None if per_ap is None else per_ap * n_ap / launches_
        work = (f"{n_seg} segments x {seg_flop:.0f} flop (the method's 2-D FFT count per segment, Sec. 5.1) "
                f"over {launches_} launches")
        if tc:  # three BF16 GEMMs of Ls x 2N (padded to 64-wide K atoms) x 2 Lm per AP
            gemm = n_ap * 3 * 2 * h.Ls * (64 * ((2 * wl.n_chan + 63) // 64)) * 2 * h.Lm
            roof = {"bound": "tensor", "kernel": "k_tree_mma", "achieved": achieved, "peak": bf16_peak,
                    "unit": "TFLOP/s", "frac": achieved / bf16_peak, "traffic": traffic,
                    "peak_kind": f"{peaks_kind} sustained bf16 (MEASURED_PEAKS.json, cuBLAS)",
                    "work": work,
                    "executed_tensor": {
                        "achieved": gemm / (kms / 1e3) / 1e12, "peak": bf16_peak,
                        "frac": gemm / (kms / 1e3) / 1e12 / bf16_peak, "unit": "TFLOP/s",
                        "work": f"{n_ap} APs x 3 BF16 GEMMs (split operands) of the MBD transform, "
                                "Ls x 2N x 2Lm each"},
                    "executed_cuda_core": {
                        "achieved": epilogue / (kms / 1e3) / 1e12, "peak": own["fp32"],
                        "frac": epilogue / (kms / 1e3) / 1e12 / own["fp32"], "unit": "TFLOP/s",
                        "peak_kind": "this GPU's FP32 FMA pipe, measured by libfrbx_peaks",
                        "work": "2 Ls Lm per summed window + 3 Ls Lm per emitted segment"}}
        else:
            executed = n_ap * h.Ls * 5 * h.Lm * math.log2(h.Lm) + epilogue
            roof = {"bound": "alu", "kernel": "k_tree_mbd", "achieved": achieved, "peak": own["fp32"],
                    "unit": "TFLOP/s", "frac": achieved / own["fp32"], "traffic": traffic,
                    "peak_kind": "this GPU's FP32 FMA pipe, measured by libfrbx_peaks", "work": work,
                    "executed": {"achieved": executed / (kms / 1e3) / 1e12,
                                 "frac": executed / (kms / 1e3) / 1e12 / own["fp32"],
                                 "work": f"{n_ap} AP transforms x Ls 5 Lm log2 Lm + 2 Ls Lm per summed window "
                                         "+ 3 Ls Lm per emitted segment"}}
        roof.update({"traffic_note": "bytes per launch, scaled by series-APs from the vgos-profile ncu capture",
                     "kernel_ms": kms, "launches": launches_, "fit_ms": fit_mean})
    else:
        achieved = flops / (fit_mean / 1e3) / 1e12
        kname = ("k_fit_mma" if args.kernel in (3, 5) else
                 "k_fit_fft" if (h.Ls % 32 == 0 and h.Lm % 32 == 0 and args.kernel != 1) else "k_fit_direct")
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": own["fp32"], "unit": "TFLOP/s",
                "frac": achieved / own["fp32"],
                "traffic": None if FIT_DRAM_BYTES_PER_SEGMENT is None else FIT_DRAM_BYTES_PER_SEGMENT * n_seg,
                "peak_kind": "this GPU's FP32 FMA pipe, measured by libfrbx_peaks",
                "work": f"{n_seg} segments x {seg_flop:.0f} flop (2-D FFT count)", "fit_ms": fit_mean}
    roof.update({"hbm_frac_8B_per_cell": hbm_frac, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_kind": peaks_kind})
    dtype = ("bf16x3 split operands, f32 accumulate (MBD transform on tcgen05); f32 elsewhere" if tc else
             "f32")

    line = {"metric": metric, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded, synth.py)", "config": cfg,
            "dtype_note": ("three BF16 products of split operands (A_hi W_hi + A_hi W_lo + A_lo W_hi) with f32 "
                           "accumulation: about 2^-16 relative per product, measured <= 1e-5 relative on |G|; "
                           "the argmax key keeps |G|^2 to 2^-17") if tc else "f32 arithmetic",
            "e2e": {"value": world * cells / (e2e / 1e3), "unit": "cells/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
            "gpu_launches": launches, "roofline": roof, "clocks": clocks, "peaks_measured": own,
            "stages_ms": stages, "segments_per_step": n_seg,
            "pulses": int(out["counts"]["pulses"]), "groups": int(out["counts"]["groups"])}
    # variants on this GPU, each timed with CUDA events on the stream after one untimed call:
    #  * the window tree's lower-precision forms on the same workload (kernel 7: one BF16 product
    #    per AP, kernel 8: E4M3), pulses compared with the default path's;
    #  * the windowed regime: the same workload with a +-64 ns SBD search window (9 of 128 SBD
    #    rows) and the whole MBD range, where the metric's 8 B/cell HBM fraction applies;
    #  * config 1 (the small S-band cube, plain: the automatic choice, the FP32 window tree, and
    #    the per-segment direct fit) and config 4 (the same cube with the MBD transform as a
    #    BF16 / E4M3 DFT-GEMM per segment, kernels 3 and 5).
    line_variants = {}

    def timed(hh, vis, wll, cmb, kernel, steps, **kw):
        hh.search(vis, wll.dms, wll.windows, combos=cmb, kernel=kernel, stream=stream, **kw)
        barrier()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fits, mbds, o = [], [], None
        v0.record(stream)
        for _ in range(steps):
            o = hh.search(vis, wll.dms, wll.windows, combos=cmb, kernel=kernel, stream=stream, **kw)
            stg = hh.stage_times()
            fits.append(stg["fit"])
            mbds.append(stg["tree_mbd_kernels"])
        v1.record(stream)
        torch.cuda.synchronize()
        vms = max_over_ranks(v0.elapsed_time(v1) / steps)
        return vms, statistics.mean(fits), statistics.mean(mbds), o

    if not args.no_variants and args.kernel == 0 and args.workload == "vgos":
        for vname, vk, vdt, peak, pkind in (
                ("tree_bf16", 7, "bf16 operands (one product per AP), f32 accumulate (MBD transform on tcgen05); "
                                 "f32 elsewhere", peaks["bf16_tflops_sustained"], peaks_kind + " sustained bf16"),
                ("tree_fp8", 8, "e4m3 operands (A scaled per AP by a power of two), f32 accumulate (MBD transform "
                                "on tcgen05); f32 elsewhere", own["fp8_mma_sustained"],
                 "this GPU's sustained E4M3 tcgen05 rate (libfrbx_peaks)")):
            try:
                vms, vfit, vmbd, o3 = timed(h, vis_dev, wl, combos, vk, args.variant_steps)
                n_ap = wl.n_bl * sum(max(0, wl.T - int(x)) for x in dk_max)
                kdim = 64 * ((2 * wl.n_chan + 63) // 64) if vk == 7 else 32 * ((2 * wl.n_chan + 31) // 32)
                gemm = n_ap * 2.0 * h.Ls * kdim * 2 * h.Lm
                line_variants[vname] = {
                    "value": world * cells / (vms / 1e3), "unit": "cells/s", "ms_per_step": vms,
                    "steps": args.variant_steps, "dtype": vdt,
                    "roofline": {"bound": "tensor", "kernel": "k_tree_mma", "achieved": flops / (vmbd / 1e3) / 1e12,
                                 "peak": peak, "unit": "TFLOP/s", "frac": flops / (vmbd / 1e3) / 1e12 / peak,
                                 "traffic": None, "peak_kind": pkind, "work": roof["work"],
                                 "executed_tensor": {"achieved": gemm / (vmbd / 1e3) / 1e12,
                                                     "frac": gemm / (vmbd / 1e3) / 1e12 / peak,
                                                     "work": f"{n_ap} APs x one GEMM of Ls x 2N x 2Lm"},
                                 "kernel_ms": vmbd, "fit_ms": vfit},
                    "pulses": int(o3["counts"]["pulses"]), "pulses_default_path": int(out["counts"]["pulses"]),
                    "groups": int(o3["counts"]["groups"])}
            except Exception as exc:  # a variant that cannot run on this setup is reported, not fatal
                line_variants[vname] = {"unavailable": str(exc)}
        try:
            sbd_win = (-64.0, 64.0)
            vms, vfit, vmbd, o4 = timed(h, vis_dev, wl, combos, 0, args.variant_steps, sbd_win_ns=sbd_win)
            sbd_ax = (np.where(np.arange(h.Ls) < h.Ls // 2, np.arange(h.Ls), np.arange(h.Ls) - h.Ls) * wl.n_point
                      * 1000.0) / (h.Ls * wl.f_bw_mhz)
            rows = int(np.sum((sbd_ax >= sbd_win[0]) & (sbd_ax <= sbd_win[1])))
            wcells = cells  # the metric's cells count the search volume as it is defined (bl x DM x AP x point)
            hbm_w = 8.0 * wcells / (vms / 1e3) / (peaks["hbm_gbs"] * 1e9)
            line_variants["windowed"] = {
                "value": world * wcells / (vms / 1e3), "unit": "cells/s", "ms_per_step": vms,
                "steps": args.variant_steps, "dtype": dtype,
                "sbd_window_ns": list(sbd_win), "sbd_rows_searched": rows, "mbd": "whole grid",
                "roofline": {"bound": "hbm", "kernel": "search (8 B per cell)", "achieved": 8.0 * wcells / (vms / 1e3) / 1e9,
                             "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_w, "traffic": None,
                             "peak_kind": peaks_kind, "kernel_ms": vmbd, "fit_ms": vfit,
                             "note": "the metric's HBM fraction: 8 B per (bl, DM, AP, point) cell over the step time"},
                "pulses": int(o4["counts"]["pulses"])}
        except Exception as exc:
            line_variants["windowed"] = {"unavailable": str(exc)}
    if not args.no_variants and args.kernel == 0 and args.workload == "vgos":
        try:
            ws, wcombos = make_workload("small")
            svis = torch.from_numpy(synth.generate(ws)).cuda()
            hs = frbx.Handle.from_workload(ws)
            scells = cells_of(ws)
            base = None
            for vname, vk, vdt in (("config1_small", 0, "f32"),
                                   ("config1_small_direct", 1, "f32"),
                                   ("config4_bf16", 3, "bf16 operands, f32 accumulate (MBD DFT-GEMM per segment)"),
                                   ("config4_fp8", 5, "e4m3 operands (A scaled per segment), f32 accumulate "
                                                      "(MBD DFT-GEMM per segment)")):
                vms, vfit, _, o5 = timed(hs, svis, ws, wcombos, vk, max(3, args.variant_steps))
                ent = {"value": world * scells / (vms / 1e3), "unit": "cells/s", "ms_per_step": vms, "fit_ms": vfit,
                       "dtype": vdt, "workload": workload_config("small", ws)["workload"],
                       "pulses": int(o5["counts"]["pulses"]), "groups": int(o5["counts"]["groups"]),
                       "fit": ("FP32 window tree (kernel 4)" if hs.stage_times()["tree_chunks"] > 0 else
                               f"per-segment fit (kernel {vk})")}
                if base is None:
                    base = o5
                else:
                    a = {(int(p["series"]), int(p["dm_idx"]), int(p["k0"]), int(p["width"])) for p in base["pulses"]}
                    b2 = {(int(p["series"]), int(p["dm_idx"]), int(p["k0"]), int(p["width"])) for p in o5["pulses"]}
                    ent["pulses_same_as_f32"] = len(a & b2)
                    ent["pulses_f32"] = len(a)
                line_variants[vname] = ent
            del svis
        except Exception as exc:
            line_variants["config1_small"] = {"unavailable": str(exc)}
    if not args.no_variants and args.kernel == 0:
        # config 3 needs the device memory the main workload holds: release it first
        h.close()
        del vis_dev
        torch.cuda.empty_cache()
        try:
            line_variants["batch"] = run_batch_variant(frbx, torch, stream, args.batch_bl, args.batch_scale,
                                                       max(1, args.batch_steps), barrier,
                                                       cpu_seconds=0.0 if (args.no_cpu_baseline or world > 1) else
                                                       args.cpu_seconds)
        except Exception as exc:
            line_variants["batch"] = {"unavailable": str(exc)}
    if line_variants:
        line["variants"] = line_variants
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, dt = run_oracle_sample(wl, vis_host[0], args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
