#!/usr/bin/env python
"""Benchmark: convolution gridding (Winkel, Lenz & Floeer 2016) on GB300.

Workload: the spectral cube -- 1e6 samples on a basket-weave raster over
10 x 10 deg, 256 channels per sample, gridded onto 512 x 512 plate-carree
targets with a Gaussian kernel of sigma = 3', support 9', HEALPix nside 4096
(hpx_maxres = sigma / 2).  Inputs are synthetic and seeded (workloads.cube).

One step = one full pass of the hot path over the batch, through the C ABI
(cg_grid_oneshot): sample HEALPix keys, radix sort, sample gather / ring
offsets / tile ranges, tile gridder, normalisation into the [P][C] cube.
Inputs are resident in HBM at the start of the timed region and are larger
than L2 (1 GB of FP32 data / 512 MB of BF16), so no flush is needed.

Metric: sample-channel kernel updates per second = C x #{(p, n): d_pn <= r}
per step / step time; the pair count comes from the library's own count of
the cut decisions and is checked against the FP64 oracle's count stored in
tests/golden/pair_counts.json.

`--impl reference` times the FP64 CPU oracle (the HEALPix-lookup gridder of
oracle/) on bounded samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sample·channel kernel updates/s and % HBM roofline, mixed vs FP32 form"
UNIT = "updates/s"
GOLDEN_PAIRS = os.path.join(ROOT, "tests", "golden", "pair_counts.json")
FFMA_LANES_PER_SM = 128
N_SMS = 152


def progress(msg):
    """Progress marker on stderr (flushed), so a crash can be located."""
    sys.stderr.write("[bench] %s\n" % msg)
    sys.stderr.flush()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["auto", "fp32", "bf16", "bf16s"], default="auto",
                    help="bf16: BF16 data, hi + lo BF16 weights; bf16s: single BF16 weights")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = full)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the differentiable-workload timings")
    ap.add_argument("--cpu-samples", type=int, default=12000)
    ap.add_argument("--only", choices=["plain2d", "allsky", "example1"], default=None,
                    help="time one other workload alone (at --scale; --form picks the form) "
                         "and print its record instead of the benchmark line")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def golden_pairs(name):
    if not os.path.exists(GOLDEN_PAIRS):
        return None
    with open(GOLDEN_PAIRS) as f:
        return json.load(f).get(name)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """Largest x over the ranks (the slowest rank's time); device "cpu" for
    a gloo process group."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_max):
    """Whole-job throughput of N replicas: every rank processes the same
    units per step (weak scaling); the job takes as long as its slowest
    rank."""
    return units_per_rank * world / (ms_max / 1e3)


def is_bf16(form):
    return form.startswith("bf16")


def form_path(form):
    """The accumulation form of a bench form name: bf16 = BF16 data with hi +
    lo BF16 weights on the tensor cores, bf16s = single BF16 weights, fp32 =
    FP32 CUDA cores."""
    from paper_1604_06667_gb300 import _capi
    return {"bf16": _capi.CG_PATH_TC, "bf16s": _capi.CG_PATH_TC_FAST,
            "fp32": _capi.CG_PATH_FP32}[form]


def sample_targets(n_targets, n, seed):
    """n distinct target indices drawn with a seeded generator (sorted)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n_targets, min(n, n_targets), replace=False))


def keep_rows(out, out_w, tsel):
    """Host copies of the map rows and weights of the targets tsel (taken
    after a timed region, for the comparison with the FP64 oracle)."""
    import torch
    idx = torch.from_numpy(tsel).to(out.device)
    return out.index_select(0, idx).cpu().numpy(), out_w.index_select(0, idx).cpu().numpy()


def sig(x, n=4):
    """x rounded to n significant digits (floats in nested containers)."""
    if isinstance(x, float):
        return float("%.*g" % (n, x)) if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: sig(v, n) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, n) for v in x]
    return x


def strip_private(x):
    """Drop the '_'-prefixed working entries (host arrays) before JSON."""
    if isinstance(x, dict):
        return {k: strip_private(v) for k, v in x.items() if not str(k).startswith("_")}
    if isinstance(x, list):
        return [strip_private(v) for v in x]
    return x


def workload_desc(wl, form):
    what = {"bf16s": "BF16 data, BF16 weights", "bf16": "BF16 data, hi+lo BF16 weights",
            "fp32": "FP32 data"}[form]
    return ("spectral cube: %d raster samples x %d ch -> %dx%d CAR targets, gauss1d sigma 3', "
            "r 9', nside 4096, %s"
            % (wl.n_samples, wl.n_channels, wl.grid_shape[1], wl.grid_shape[0], what))


def algorithmic_bytes(wl, data_bytes):
    """Bytes the method must move once per step: sample coordinates (FP64 lon,
    lat) and data rows read once; the map and weight map written once."""
    N, C, P = wl.n_samples, wl.n_channels, wl.n_targets
    return N * (16 + C * data_bytes) + P * (C * 4 + 4)


def cpu_oracle_rate(wl, n_sub, seed=12345):
    """Time the FP64 lookup oracle as it stands on a random subset of the
    workload's samples (all targets).  Returns (updates/s, seconds, sample)."""
    import numpy as np
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.sort(rng.choice(wl.n_samples, size=min(n_sub, wl.n_samples), replace=False))
    ns = oracle.nside_for_resolution(wl.hpx_maxres)
    k = oracle_kernel(wl)
    d64 = wl.data[idx].astype(np.float64)
    t0 = time.perf_counter()
    res = oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s[idx], wl.lat_s[idx], d64, k)
    dt = time.perf_counter() - t0
    upd = res.npairs * wl.n_channels
    return upd / dt, dt, idx.size, res.npairs


def cpu_baseline_entry(wl, n_sub, seed):
    rate, dt, n, npairs = cpu_oracle_rate(wl, n_sub, seed)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d random samples x all %d targets (%d pairs), %.1f s"
                      % (n, wl.n_targets, npairs, dt)}


def oracle_candidates(wl, tsel):
    """Samples that can reach the targets tsel: a latitude band from one sort,
    then the great-circle distance against the support widened by 1e-6 (a
    superset, so the brute-force sum over them is exact for those targets)."""
    import numpy as np
    order = np.argsort(wl.lat_s, kind="stable")
    ls = wl.lat_s[order]
    rad = wl.support * (1.0 + 1e-6) + 1e-9
    keep = []
    for lc, bc in zip(wl.lon_t[tsel], wl.lat_t[tsel]):
        lo = np.searchsorted(ls, bc - rad, "left")
        hi = np.searchsorted(ls, bc + rad, "right")
        idx = order[lo:hi]
        b1, b2 = np.radians(bc), np.radians(wl.lat_s[idx])
        dl = np.radians(wl.lon_s[idx] - lc)
        h = np.sin(0.5 * (b2 - b1)) ** 2 + np.cos(b1) * np.cos(b2) * np.sin(0.5 * dl) ** 2
        d = 2.0 * np.arcsin(np.sqrt(np.minimum(h, 1.0)))
        keep.append(idx[d <= np.radians(rad)])
    return np.unique(np.concatenate(keep)) if keep else np.zeros(0, dtype=np.int64)


def oracle_kernel(wl):
    import oracle
    k = wl.kernel
    if k["type"] == "gauss1d":
        return oracle.gauss1d(k["sigma"], wl.support)
    return oracle.gauss2d(k["smaj"], k["smin"], k["pa"], wl.support)


def oracle_errors(wl, tsel, rows):
    """Error of GPU rows (map, weights at the targets tsel) against the FP64
    brute-force oracle on the caller's FP32 data: max and 99th percentile of
    |R - R_oracle| / S (S = sum |omega w D| / W, the oracle's scale) over
    W > 0 targets and channels, the largest relative weight-map error, and
    support mismatches.  Returns (error dict, oracle seconds, oracle pairs)."""
    import numpy as np
    import oracle
    cand = oracle_candidates(wl, tsel)
    t0 = time.perf_counter()
    ref = oracle.grid_bruteforce(wl.lon_t[tsel], wl.lat_t[tsel], wl.lon_s[cand], wl.lat_s[cand],
                                 np.asarray(wl.data, dtype=np.float64)[cand], oracle_kernel(wl),
                                 None if wl.omega is None else np.asarray(wl.omega)[cand])
    dt = time.perf_counter() - t0
    res = {}
    for form, (got, got_w) in rows.items():
        got = np.asarray(got, dtype=np.float64)
        got_w = np.asarray(got_w, dtype=np.float64)
        on = ref.wsum > 0
        mism = int((on != (got_w > 0)).sum())
        both = on & (got_w > 0)
        scale = np.where(ref.sabs[both] > 0, ref.sabs[both], 1.0)
        e = np.abs(got[both] - ref.out[both]) / scale
        e = np.where(np.isnan(e), np.inf, e).ravel()
        we = np.abs(got_w[both] - ref.wsum[both]) / ref.wsum[both]
        res[form] = {"max": float(e.max()) if e.size else 0.0,
                     "p99": float(np.percentile(e, 99)) if e.size else 0.0,
                     "w_max": float(we.max()) if we.size else 0.0,
                     "support_mismatch": mism, "targets": int(len(tsel)),
                     "values": int(e.size)}
    return res, dt, ref.npairs


def run_reference(args):
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    import workloads
    wl = workloads.cube(scale=args.scale)
    form = "fp32" if args.form == "auto" else args.form
    n_sub = max(200, args.cpu_samples // 4)
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, max(50, n_sub // 10), seed=7)
    tot_upd, tot_t = 0.0, 0.0
    for s in range(args.steps):
        rate, dt, n, pairs = cpu_oracle_rate(wl, n_sub, seed=1000 + s)
        tot_upd += pairs * wl.n_channels
        tot_t += dt
    value = tot_upd / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(wl, form), "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d random samples of the workload per step, all %d targets"
                                   % (n_sub, wl.n_targets)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def time_form(g, wl, form, lon, lat, data, out, out_w, args, world, local, peaks, peaks_src,
              tsel):
    """Warm up, then time K one-shot steps of one accumulation form."""
    import torch
    from paper_1604_06667_gb300 import _capi
    dev = out.device
    g.set_path(form_path(form))
    stream = torch.cuda.current_stream(dev)

    def step():
        g.grid_oneshot(lon, lat, data, out=out, out_weights=out_w)

    for i in range(args.warmup):
        step()
        g.sync()
        progress("  warm-up step %d ok" % i)
    info0 = g.info()
    g.set_timing(True)
    g.read_timing()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    stages = g.read_timing()
    g.set_timing(False)
    info1 = g.info()
    sel = keep_rows(out, out_w, tsel)
    ms_max = max_over_ranks(ms, world)
    pairs = info1["n_pairs"]
    C = wl.n_channels
    upd = float(pairs) * C
    dbytes = 2 if is_bf16(form) else 4
    t_grid = stages["grid"] / max(1, stages["grid_launches"])
    if form == "fp32":
        peak_tf = N_SMS * FFMA_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = 2.0 * upd / (t_grid / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": None,
                "kernel": "k_grid_f32 (tile gridder, FP32 CUDA cores)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    else:
        hbm = peaks["hbm_gbs"]
        # the method's bytes (sample lon/lat and data rows read once, map
        # and weight map written once), charged to the dominant kernel
        kbytes = algorithmic_bytes(wl, dbytes)
        ach = kbytes / (t_grid / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm,
                "traffic": captured_traffic() if args.scale == 1.0 else None,
                "kernel": "k_grid_tc (tile gridder, BF16 tcgen05 + TMEM)",
                "bytes_per_launch": kbytes, "peak_source": peaks_src,
                "tensor_useful_tflops": 2.0 * upd / (t_grid / 1e3) / 1e12,
                # MMA work as executed: every evaluated (target, candidate)
                # weight times C channels, hi + lo BF16 halves
                "tensor_executed_tflops": (2.0 if form == "bf16" else 1.0) * 2.0 * C *
                float(info1["n_candidates"]) *
                float(info1["tile_size"]) / (t_grid / 1e3) / 1e12,
                "tensor_peak_tflops": peaks.get("bf16_tflops")}
    step_bytes = algorithmic_bytes(wl, dbytes)
    return {
        "form": form, "value": job_value(upd, world, ms_max), "ms_per_step": ms_max,
        "pairs": pairs, "updates_per_step": upd,
        "weights_evaluated": int(info1["n_candidates"]) * int(info1["tile_size"]),
        "hbm_roofline": {"bytes_per_step": step_bytes,
                         "achieved_gbs": step_bytes / (ms_max / 1e3) / 1e9,
                         "peak_gbs": peaks["hbm_gbs"],
                         "frac": step_bytes / (ms_max / 1e3) / 1e9 / peaks["hbm_gbs"],
                         "peak_source": peaks_src},
        "roofline": roof,
        "stages_ms_per_step": {k: v / args.steps for k, v in stages.items()
                               if k != "grid_launches"},
        "gpu_launches": info1["n_launches"] - info0["n_launches"],
        "clocks": clocks,
        "_sel": sel,
    }


def time_differentiable(args, dev):
    """The differentiable workload (2e5 samples x 16 channels -> 256 x 256,
    sigma = 4', r = 12'): one forward + backward step (one-shot gridding, the
    adjoint of dL/dR and dL/dsigma) and the 50-step map-making loop, each
    timed with CUDA events after warm-up."""
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder, mapmaking
    wl = workloads.diff(scale=1.0)
    P, C = wl.n_targets, wl.n_channels
    lon = torch.from_numpy(wl.lon_s).to(dev)
    lat = torch.from_numpy(wl.lat_s).to(dev)
    data = torch.from_numpy(wl.data).to(dev)
    gR = torch.randn((P, C), device=dev, generator=torch.Generator(dev).manual_seed(5))
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=C, device=dev)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    R = torch.empty((P, C), device=dev)
    W = torch.empty(P, device=dev)
    gx = torch.empty((wl.n_samples, C), device=dev)

    def step():
        g.grid_oneshot(lon, lat, data, out=R, out_weights=W)
        g.degrid(gR, map_weights=W, out=gx)
        g.dsigma(data, grad_out=gR, want_dR=False)

    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(5, args.steps)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    mapmaking.gd(g, lon, lat, data, steps=50)         # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    _, losses, _ = mapmaking.gd(g, lon, lat, data, steps=50)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    g.close()
    return {"workload": "differentiable: %d samples x %d channels -> %dx%d targets at 2', "
                        "gauss1d sigma=4', r=12' (fixed in d/dsigma)"
                        % (wl.n_samples, C, wl.grid_shape[1], wl.grid_shape[0]),
            "ms_forward_backward": ms_step,
            "ms_mapmaking_50_steps": ms_loop,
            "mapmaking_loss_first_last": [float(losses[0]), float(losses[-1])]}


# DRAM bytes (read + write) of one k_grid_tc launch on the full cube, from an
# ncu capture of `dram__bytes_read.sum,dram__bytes_write.sum` (summary under
# profiles/); valid only for the kernel source it was taken with.
TRAFFIC_CAPTURE = {"source": "paper_1604_06667_gb300/csrc/k_grid_tc.cu",
                   "sha256": "3e561e8b1826564df4792670765e39acc7f8e740c023143b66a485656258c3d7",
                   "bytes_per_launch": 961199616 + 263374592}


def captured_traffic():
    import hashlib
    if not TRAFFIC_CAPTURE["sha256"]:
        return None
    try:
        with open(os.path.join(ROOT, TRAFFIC_CAPTURE["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return TRAFFIC_CAPTURE["bytes_per_launch"] if sha == TRAFFIC_CAPTURE["sha256"] else None


def time_batched(args, dev, n_jobs=64):
    """64 independent jobs (sample count log-uniform in [1e4, 1e6], channels
    in {1, 16, 64, 512}, grids 64^2 .. 1024^2, sigma U[1', 8']) replayed as one
    CUDA graph; mixed form = BF16 data for the jobs with C >= 16 and the
    autotuner free to pick the tensor-core form, plain form = FP32 data on
    the FP32 CUDA-core path (autotuned shapes).  Each form is timed twice on
    the same jobs and choices: the per-job graph (one pipeline per job on 16
    branches) and the fused graph (one sample index and one persistent FP32
    gridder launch per register shape).  Inputs resident in HBM."""
    import torch
    import workloads
    from paper_1604_06667_gb300 import Batch, Gridder
    specs = workloads.batch_specs(n_jobs)
    forms = {"mixed": [], "fp32": []}
    keep = []
    for sp in specs:
        lon, lat, d32, lon_t, lat_t = workloads.batch_job_device(sp, dev)
        for form in forms:
            g = Gridder(lon_t, lat_t, n_channels=sp["C"], device=dev)
            g.set_kernel("gauss1d", (sp["sigma"],), 3.0 * sp["sigma"], sp["sigma"] / 2.0)
            d = d32.to(torch.bfloat16) if (form == "mixed" and sp["C"] >= 16) else d32
            out = torch.empty((g.n_targets, sp["C"]), device=dev)
            forms[form].append((g, lon, lat, d, out))
        keep.append(d32)
    res = {}
    peaks, _ = load_peaks()
    stream = torch.cuda.current_stream(dev)
    for form, jobs in forms.items():
        b = Batch(jobs, n_streams=16).autotune(reps=2, allow_tc=(form == "mixed")).capture()
        for _ in range(max(3, args.warmup)):
            b.run()
        torch.cuda.synchronize()
        pairs = [j[0].info()["n_pairs"] for j in jobs]
        upd = float(sum(p * sp["C"] for p, sp in zip(pairs, specs)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(3, args.steps)
        e0.record(stream)
        for _ in range(steps):
            b.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ch = b.choices()
        res[form] = {"ms_per_batch": ms, "updates_per_s": upd / (ms / 1e3),
                     "updates_per_batch": upd, "pairs_per_batch": int(sum(pairs)),
                     "graph_kernels": b.info()["graph_kernels"],
                     "tc_jobs": sum(1 for c in ch if c["path"] == 2)}
        # the fused pipeline on the same jobs and choices: one sample index,
        # one persistent FP32 gridder launch, tensor-core jobs on their own
        b.set_fused(True).capture()
        for _ in range(max(3, args.warmup)):
            b.run()
        b.sync()
        e0.record(stream)
        for _ in range(steps):
            b.run()
        e1.record(stream)
        b.sync()
        torch.cuda.synchronize()
        msf = e0.elapsed_time(e1) / steps
        res[form]["fused"] = {"ms_per_batch": msf, "updates_per_s": upd / (msf / 1e3),
                              "graph_kernels": b.info()["graph_kernels"]}
        # the method's bytes of the batch (every job's samples and data read
        # once, its map and weight map written once) against the HBM peak
        nbytes = sum(sp["n"] * (16 + sp["C"] * j[3].element_size()) +
                     sp["side"] ** 2 * (4 * sp["C"] + 4) for sp, j in zip(specs, jobs))
        best = min(ms, msf)
        res[form]["bytes_per_batch"] = nbytes
        res[form]["hbm_frac"] = nbytes / (best / 1e3) / 1e9 / peaks["hbm_gbs"]
        b.close()
    for jobs in forms.values():
        for j in jobs:
            j[0].close()
    res["mixed_over_fp32"] = res["mixed"]["updates_per_s"] / res["fp32"]["updates_per_s"]
    res["workload"] = ("%d jobs: %d samples, %.2e channel values, %d targets in total"
                       % (n_jobs, sum(s["n"] for s in specs), sum(s["n"] * s["C"] for s in specs),
                          sum(s["side"] ** 2 for s in specs)))
    return res


def time_config(args, dev, name):
    """Plain 2-D (2e4 samples -> 100^2, sigma 2.5') and all-sky elliptical
    (1e7 samples x 32 channels -> 4096 x 2048, 10'/6'/PA 30, r = 30')
    one-shot calls, each form timed with CUDA events after warm-up."""
    import numpy as np
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder, _capi
    wl = workloads.plain2d(args.scale) if name == "plain2d" else workloads.allsky(args.scale)
    lon = torch.from_numpy(wl.lon_s).to(dev)
    lat = torch.from_numpy(wl.lat_s).to(dev)
    d32 = torch.from_numpy(wl.data).to(dev)
    k = wl.kernel
    kt, kp = ("gauss1d", (k["sigma"],)) if k["type"] == "gauss1d" else \
        ("gauss2d", (k["smaj"], k["smin"], k["pa"]))
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels, device=dev)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    out = torch.empty((wl.n_targets, wl.n_channels), device=dev)
    w = torch.empty(wl.n_targets, device=dev)
    # targets checked against the FP64 oracle afterwards: the whole plain 2-D
    # map; for the all-sky map random targets plus the rows next to the poles
    if name == "plain2d":
        tsel = np.arange(wl.n_targets)
    else:
        nx = wl.grid_shape[1]
        tsel = np.unique(np.concatenate([sample_targets(wl.n_targets, 160, 612),
                                         np.arange(0, 32), np.arange(wl.n_targets - 32, wl.n_targets),
                                         nx * (wl.grid_shape[0] // 2) + np.arange(0, nx, nx // 16)]))
    forms = [("fp32", _capi.CG_PATH_FP32, d32)]
    if wl.n_channels % 8 == 0:
        d16 = d32.to(torch.bfloat16)
        forms.append(("bf16", _capi.CG_PATH_TC, d16))
        forms.append(("bf16s", _capi.CG_PATH_TC_FAST, d16))
    if args.form != "auto":
        forms = [f for f in forms if f[0] == args.form]
    res = {"workload": "%s: %d samples x %d channels -> %d targets" % (
        name, wl.n_samples, wl.n_channels, wl.n_targets)}
    stream = torch.cuda.current_stream(dev)
    for form, path, d in forms:
        g.set_path(path)
        for _ in range(3):
            g.grid_oneshot(lon, lat, d, out=out, out_weights=w)
        g.sync()
        pairs = g.info()["n_pairs"]
        steps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.grid_oneshot(lon, lat, d, out=out, out_weights=w)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        db = 2 if is_bf16(form) else 4
        nbytes = wl.n_samples * (16 + wl.n_channels * db) + wl.n_targets * (4 * wl.n_channels + 4)
        res[form] = {"ms_per_call": ms, "pairs": pairs,
                     "updates_per_s": pairs * wl.n_channels / (ms / 1e3),
                     "hbm_frac": nbytes / (ms / 1e3) / (load_peaks()[0]["hbm_gbs"] * 1e9),
                     "_sel": keep_rows(out, w, tsel)}
    g.close()
    res["_wl"] = wl
    res["_tsel"] = tsel
    return res


def time_example1(args, dev):
    """The paper's Example 1 (Sect. 4) at 1e8 samples: 5 x 5 deg field, 200"
    pixels, FWHM 300" Gaussian, one channel of noise -- the paper quotes about
    67 s on 16 cores for this size.  One-shot calls timed with CUDA events."""
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder
    lon, lat, data, lon_t, lat_t, kern, support, maxres = workloads.example1_device(
        dev, n=max(1, int(round(100_000_000 * args.scale))))
    g = Gridder(lon_t, lat_t, n_channels=1, device=dev)
    g.set_kernel("gauss1d", (kern["sigma"],), support, maxres)
    out = torch.empty((g.n_targets, 1), device=dev)
    w = torch.empty(g.n_targets, device=dev)
    for _ in range(2):
        g.grid_oneshot(lon, lat, data, out=out, out_weights=w)
    g.sync()
    g.set_timing(True)
    g.read_timing()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 3
    e0.record(stream)
    for _ in range(steps):
        g.grid_oneshot(lon, lat, data, out=out, out_weights=w)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stages = g.read_timing()
    info = g.info()
    g.close()
    # a bounded random subset (host copy) for the CPU leg's oracle timing
    import numpy as np
    import workloads as wlmod
    rng = np.random.Generator(np.random.PCG64(77))
    sub = torch.from_numpy(np.sort(rng.choice(lon.numel(), 200000, replace=False))).to(dev)
    wl_sub = wlmod.Workload("example1-subset", lon[sub].cpu().numpy(), lat[sub].cpu().numpy(),
                            data[sub].float().cpu().numpy().reshape(-1, 1), None,
                            np.asarray(lon_t), np.asarray(lat_t), dict(kern), support, maxres,
                            (90, 90), {})
    return {"_wl": wl_sub,
            "workload": "paper Example 1: %d samples uniform in 5x5 deg, 90x90 targets at 200\", "
                        "FWHM 300\" Gaussian, support 3 sigma, one channel" % lon.numel(),
            "ms_per_call": ms, "pairs_per_call": info["n_pairs"],
            "stages_ms": {k: v / steps for k, v in stages.items() if k != "grid_launches"},
            "paper_16_cores_s": 67.0, "speedup_vs_paper_16_cores": 67.0e3 / ms}


def time_sightline(args, dev):
    """Appendix A.1 of the paper: ~4.7e7 samples uniform on the sphere (1024
    PSF-convolved point sources + noise) gridded onto the 3,145,728 pixel
    centres of an nside-512 HEALPix grid (sight-line targets), kernel FWHM
    13.7'.  One-shot calls timed with CUDA events."""
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder
    lon, lat, data, lon_t, lat_t, kern, support, maxres, meta = workloads.sightline_device(dev)
    g = Gridder(lon_t, lat_t, n_channels=1, device=dev)
    g.set_kernel("gauss1d", (kern["sigma"],), support, maxres)
    out = torch.empty((g.n_targets, 1), device=dev)
    w = torch.empty(g.n_targets, device=dev)
    for _ in range(2):
        g.grid_oneshot(lon, lat, data, out=out, out_weights=w)
    g.sync()
    g.set_timing(True)
    g.read_timing()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = 3
    e0.record(stream)
    for _ in range(steps):
        g.grid_oneshot(lon, lat, data, out=out, out_weights=w)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stages = g.read_timing()
    info = g.info()
    g.close()
    return {"workload": "paper App. A.1: %d samples uniform on the sphere -> %d HEALPix nside-%d "
                        "pixel centres, kernel FWHM %.2f', support 3 sigma, one channel"
                        % (lon.numel(), lon_t.size, meta["nside_targets"],
                           meta["fwhm_kernel_deg"] * 60.0),
            "ms_per_call": ms, "pairs_per_call": info["n_pairs"],
            "updates_per_s": info["n_pairs"] / (ms / 1e3),
            "stages_ms": {k: v / steps for k, v in stages.items() if k != "grid_launches"}}


def study_aliasing(args, dev):
    """Appendix A.2 of the paper: scan lines 0.2-0.5 PSF apart gridded with
    kernels of 0.3-0.7 PSF (FWHM), support 5 and 3 sigma, over a 1.5 x 1.5
    deg field with PSF / 20 pixels; max |R - T| / T against the field
    convolved with the kernel (T).  The paper prints these only as figures."""
    import numpy as np
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder
    table, t_gpu = {}, 0.0
    truths = {}
    for fs in (0.2, 0.3, 0.4, 0.5):
        row = {}
        for fk in (0.3, 0.4, 0.5, 0.6, 0.7):
            cell = {}
            for ssig in (5.0, 3.0):
                wl = workloads.aliasing(fs, fk, support_sigmas=ssig)
                if fk not in truths:
                    truths[fk] = workloads.aliasing_truth(wl)
                g = Gridder(wl.lon_t, wl.lat_t, n_channels=1, device=dev)
                g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
                d = torch.from_numpy(wl.data).to(dev)
                lon = torch.from_numpy(wl.lon_s).to(dev)
                lat = torch.from_numpy(wl.lat_s).to(dev)
                out = torch.empty((wl.n_targets, 1), device=dev)
                g.grid_oneshot(lon, lat, d, out=out)
                g.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.grid_oneshot(lon, lat, d, out=out)
                e1.record()
                torch.cuda.synchronize()
                t_gpu += e0.elapsed_time(e1)
                r = out[:, 0].cpu().numpy().astype(np.float64)
                g.close()
                cell["support_%dsigma" % int(ssig)] = float(np.max(np.abs(r - truths[fk]) / truths[fk]))
            row["kernel_%.1f" % fk] = cell
        table["spacing_%.1f" % fs] = row
    return {"workload": "paper App. A.2: scan lines, 1.5 x 1.5 deg, PSF 0.1 deg, pixel PSF/20, "
                        "no noise; max relative deviation from the kernel-convolved field",
            "max_rel_deviation": table, "gpu_ms_total": t_gpu}


def detail_path():
    """Where the full result record goes: BENCH_DETAIL if set, else
    bench_detail.json in the working directory."""
    return os.environ.get("BENCH_DETAIL") or "bench_detail.json"


def compact_line(line, detail_file):
    """The one JSON line: the contract's keys plus short summaries (forms,
    mixed / FP32 ratio, oracle errors, batched); everything else stays in the
    detail file, so the line fits a short log tail."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "gpu_launches", "clocks", "roofline", "e2e", "cpu_baseline")
    out = {k: line[k] for k in keep if k in line}
    out["clocks"] = {k: v for k, v in line["clocks"].items() if k != "samples"}
    out["roofline"] = {k: v for k, v in line["roofline"].items()
                       if k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    out["roofline"]["kernel"] = line["roofline"]["kernel"].split(" ")[0]
    if "e2e" in line:
        out["e2e"] = {k: line["e2e"][k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                  "d2h_bytes_per_step")}
    out["forms"] = {f: {"ms": r["ms_per_step"], "value": r["value"], "frac": r["roofline"]["frac"]}
                    for f, r in line["forms"].items()}
    if "mixed_over_fp32" in line:
        out["mixed_over_fp32"] = line["mixed_over_fp32"]
    if "error_vs_oracle" in line:
        # largest error of each form and config in units of S (p99 and the
        # weight-map error are in the detail file)
        out["err_max"] = {k: sig(v.get("max"), 2)
                          for k, v in line["error_vs_oracle"].items() if isinstance(v, dict)}
    if "batched" in line:
        b = line["batched"]
        out["batched"] = {"mixed_ms": b["mixed"]["ms_per_batch"],
                          "fp32_ms": b["fp32"]["ms_per_batch"],
                          "ratio": b["mixed_over_fp32"],
                          "kernels": b["mixed"]["graph_kernels"],
                          "fused_ms": [b["mixed"]["fused"]["ms_per_batch"],
                                       b["fp32"]["fused"]["ms_per_batch"]],
                          "fused_kernels": [b["mixed"]["fused"]["graph_kernels"],
                                            b["fp32"]["fused"]["graph_kernels"]],
                          "hbm_frac": [b["mixed"]["hbm_frac"], b["fp32"]["hbm_frac"]]}
    if "allsky" in line:
        out["allsky_ms"] = {f: line["allsky"][f]["ms_per_call"] for f in ("bf16", "bf16s", "fp32")
                            if f in line["allsky"]}
    if "paper_example1" in line:
        out["example1_ms"] = line["paper_example1"]["ms_per_call"]
    out["detail"] = detail_file
    return sig(out, 3)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import workloads
    from paper_1604_06667_gb300 import Gridder

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peaks_src = load_peaks()
    if args.only:
        progress("workload %s alone" % args.only)
        r = time_example1(args, dev) if args.only == "example1" else \
            time_config(args, dev, args.only)
        print(json.dumps(strip_private(r), default=float))
        return
    progress("generating workload")
    wl = workloads.cube(scale=args.scale)
    # headline: BF16 data with hi + lo BF16 weights; then single BF16
    # weights, then the FP32 form (each with its error against the oracle)
    forms = ["bf16", "bf16s", "fp32"] if args.form == "auto" else [args.form]
    N, C, P = wl.n_samples, wl.n_channels, wl.n_targets
    lon = torch.from_numpy(wl.lon_s).to(dev)
    lat = torch.from_numpy(wl.lat_s).to(dev)
    data32 = torch.from_numpy(wl.data).to(dev)
    data16 = data32.to(torch.bfloat16)
    progress("create")
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=C, device=dev)
    progress("set_kernel")
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    out = torch.empty((P, C), device=dev, dtype=torch.float32)
    out_w = torch.empty(P, device=dev, dtype=torch.float32)
    tsel_cube = sample_targets(P, 200, 613)
    results = {}
    for form in forms:
        progress("timing form %s" % form)
        data = data16 if is_bf16(form) else data32
        results[form] = time_form(g, wl, form, lon, lat, data, out, out_w, args, world, local,
                                  peaks, peaks_src, tsel_cube)
    prim = results[forms[0]]
    form = prim["form"]
    gold = golden_pairs("cube_scale%g" % args.scale)
    line = {
        "metric": METRIC, "value": prim["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": prim["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if is_bf16(form) else "f32",
        "data": "synthetic (seeded raster cube, no dataset)",
        "config": {"workload": workload_desc(wl, form),
                   "l2": "inputs > L2 (%d MB data), no flush"
                         % (N * C * (2 if is_bf16(form) else 4) // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "pairs_per_step": prim["pairs"],
        "pairs_oracle": (gold or {}).get("pairs"),
        "weights_evaluated_per_step": prim["weights_evaluated"],
        "tile_fill": (prim["pairs"] / prim["weights_evaluated"]
                      if prim["weights_evaluated"] else None),
        "hbm_roofline": prim["hbm_roofline"],
        "roofline": prim["roofline"],
        "stages_ms_per_step": prim["stages_ms_per_step"],
        "gpu_launches": prim["gpu_launches"],
        "clocks": prim["clocks"],
        "forms": {f: {k: r[k] for k in ("value", "ms_per_step", "hbm_roofline", "roofline",
                                        "stages_ms_per_step", "clocks")}
                  for f, r in results.items()},
    }
    if "fp32" in results and prim["form"] != "fp32":
        line["mixed_over_fp32"] = prim["value"] / results["fp32"]["value"]
    configs = {}
    if not args.no_extra and args.scale == 1.0:
        progress("differentiable workload")
        line["differentiable"] = time_differentiable(args, dev)
        progress("batched workload")
        line["batched"] = time_batched(args, dev)
        progress("paper example 1")
        line["paper_example1"] = time_example1(args, dev)
        progress("paper appendix A.1 (HEALPix sight lines)")
        line["paper_sightline_a1"] = time_sightline(args, dev)
        progress("paper appendix A.2 (scan-line aliasing study)")
        line["paper_aliasing_a2"] = study_aliasing(args, dev)
        progress("plain 2-D and all-sky")
        for name in ("plain2d", "allsky"):
            configs[name] = time_config(args, dev, name)
            line[name] = configs[name]

    # ---- end to end: pinned host inputs, copies inside the timed region ----
    # cg_grid_oneshot_host: every step copies its samples and channel data in
    # and its map out; consecutive steps overlap (copy-in of step k + 1, the
    # compute of step k, copy-out of step k - 1).  Host wall clock from the
    # first call to the return of cg_sync after the last.
    if not args.no_e2e:
        progress("e2e")
        from paper_1604_06667_gb300 import _capi
        g.set_path(form_path(form))
        data = data16 if is_bf16(form) else data32
        dbytes = 2 if is_bf16(form) else 4
        h_lon = torch.from_numpy(wl.lon_s).pin_memory()
        h_lat = torch.from_numpy(wl.lat_s).pin_memory()
        h_data = data.cpu().pin_memory()
        h_out = [torch.empty((P, C), dtype=torch.float32).pin_memory() for _ in range(2)]

        def e2e_step(k):
            g.grid_oneshot_host(h_lon, h_lat, h_data, h_out[k & 1])

        for k in range(max(1, args.warmup)):
            e2e_step(k)
        g.sync()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_step(k)
        g.sync()
        ms_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world)
        upd = prim["updates_per_step"]
        line["e2e"] = {"value": job_value(upd, world, ms_e2e), "unit": UNIT,
                       "h2d_bytes_per_step": N * 16 + N * C * dbytes,
                       "d2h_bytes_per_step": P * C * 4, "ms_per_step": ms_e2e,
                       "api": "cg_grid_oneshot_host (pipelined over consecutive calls)",
                       "timer": "host wall clock"}
    g.close()

    # ---- CPU leg (rank 0 only): the FP64 oracle as it stands ----
    # (1) the CPU baseline: the HEALPix-lookup oracle timed on a bounded
    # random subset of the cube's samples onto all targets, one host thread;
    # (2) the error of every timed GPU form against the brute-force oracle on
    # the caller's FP32 data at sampled targets (after all GPU timing).
    if rank == 0 and world == 1 and not args.no_cpu:
        progress("cpu baseline")
        rate, dt, n, npairs = cpu_oracle_rate(wl, args.cpu_samples)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "%d random samples x all %d targets, %.1f s"
                                          % (n, P, dt)}
        # the same oracle beside the other timed workloads (detail record)
        if "allsky" in configs:
            configs["allsky"]["cpu_baseline"] = cpu_baseline_entry(configs["allsky"]["_wl"],
                                                                   12000, 5)
        if "paper_example1" in line:
            line["paper_example1"]["cpu_baseline"] = cpu_baseline_entry(
                line["paper_example1"]["_wl"], 200000, 6)
        progress("errors against the FP64 oracle")
        errs = {}
        e, _, _ = oracle_errors(wl, tsel_cube, {f: r["_sel"] for f, r in results.items()})
        for f, v in e.items():
            errs["cube_" + f] = v
        for name, res in configs.items():
            rows = {f: res[f]["_sel"] for f in ("bf16", "bf16s", "fp32") if f in res}
            e, _, _ = oracle_errors(res["_wl"], res["_tsel"], rows)
            for f, v in e.items():
                errs[name + "_" + f] = v
        line["error_vs_oracle"] = errs
        line["error_vs_oracle_note"] = (
            "max and 99th percentile of |R - R_oracle| / S over W > 0 targets x channels, "
            "largest relative W error; FP64 brute-force oracle on the caller's FP32 data at "
            "sampled targets (cube 200, all-sky 226, plain 2-D the whole map)")
    if rank == 0:
        dpath = detail_path()
        detail = strip_private(line)
        try:
            with open(dpath, "w") as f:
                json.dump(detail, f, indent=1, default=float)
        except OSError as ex:
            progress("could not write %s: %s" % (dpath, ex))
        s = json.dumps(compact_line(detail, dpath), separators=(",", ":"))
        # large whole floats in exponent form (5.09e+13, not 50900000000000.0)
        s = re.sub(r"(?<=[:,\[])(\d{8,})\.0(?=[,}\]])", lambda m: "%.3g" % float(m.group(1)), s)
        print(s)
        sys.stdout.flush()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
