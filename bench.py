#!/usr/bin/env python
"""Benchmark of the TACAW hot path (multislice + time transform) on one node.

One step = the whole hot path for one synthetic trajectory: slice binning, projected
potential, transmission, multislice for every (probe, frame), FP64-class mean/residual, time
transform and |.|^2, through tacaw_run on device-resident inputs.  The default workload is
the largest single-GPU configuration, the probe scan: a 30 mrad probe on a 16 x 16 grid of
positions over 576 diamond-cubic atoms, 256 frames at 5 fs, 256^2, 20 slices (65,536 waves);
probe scans return the detector-summed spectrum image, plane waves the full S(q, w).
With N ranks (torchrun) every rank runs its own independently seeded trajectory (weak
scaling, no collective on the data path); value = all ranks' wave-slice steps / max time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c2]

--impl reference times the FP64 CPU oracle (the only reference this method has) on a bounded
sample of the same workload, on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wave-slice steps/s & S(q,ω) spectra/s vs plain path; p50/p99 latency @tol"
UNIT = "wave-slice steps/s"
PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 2, "bf16": 3, "tf32": 4}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_workload(name, seed_offset=0, frames=None, probes=None):
    """The named configuration; frames and probes (for small profiling cases) truncate the
    trajectory and the probe scan."""
    import workloads
    if name == "c1":
        w = workloads.diamond_si(n_frames=frames or 64, seed=1 + seed_offset, name="c1-diamond-si-64x128sq")
    elif name == "c2":
        w = workloads.config2(n_frames=frames or 1024, seed=2 + seed_offset)
    elif name == "c3":
        w = workloads.config3(n_frames=frames or 256, seed=3 + seed_offset)
    elif name == "c4":
        w = workloads.config4(n_frames=frames or 2048, seed=4 + seed_offset)
    elif name == "m1":
        w = workloads.minimal_example_si(n_frames=frames or 200, seed=6 + seed_offset)
    elif name == "m1s":  # the minimal example's 32 x 32 scan at 30 mrad
        w = workloads.minimal_example_si(n_frames=frames or 200, seed=6 + seed_offset, n_scan=32)
    else:
        raise SystemExit(f"unknown workload {name}")
    if probes and w.alpha_mrad > 0 and probes < w.n_probes:
        w.probes = w.probes[:probes]
    return w


def reduce_of(w):
    """Probe scans return the spectrum image (detector sum), plane waves the full S."""
    return "detector" if w.alpha_mrad > 0 else "none"


def workload_config(w, name, precision):
    return {"workload": w.name, "config": name, "atoms": int(w.n_atoms), "frames": int(w.n_frames),
            "grid": [int(w.ny), int(w.nx)], "slices": int(w.n_slices), "probes": int(w.n_probes),
            "alpha_mrad": float(w.alpha_mrad), "dt_fs": float(w.dt_fs), "voltage_kev": w.voltage_ev / 1e3,
            "bandlimit": "2/3", "time_transform": precision, "output": reduce_of(w),
            "l2": "256 MiB buffer written between timed steps (and each step streams > 3 GB)"}


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# roofline helpers
# ------------------------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "of fallback"


# the sources each profiled kernel class is compiled from (device code, launch configuration
# constants and tuning table); a class not listed hashes every CUDA source
KERNEL_SOURCES = {k: ("k_slices.cu", "fft.cuh", "tacaw_internal.cuh", "tuning_table.h")
                  for k in ("slice_row", "slice_col", "splat_row", "col_pot", "row_pot_t", "row_vt", "col_t",
                            "row_tout", "sort_rows", "bin")}


def src_hash(kernel=None):
    """Hash of the CUDA sources the kernel class is built from (all of them if unlisted)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_10064_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or [f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    for f in sorted(files):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, config, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.md): the captured
    ratio of DRAM to algorithmic bytes times this run's algorithmic bytes per launch, if the
    row matches the config, the kernel class and the current sources of that kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) == 5 and cells[0] == config and cells[1] == kernel and cells[4] == src_hash(kernel):
            try:
                return float(cells[2]) * alg_bytes_per_launch
            except ValueError:
                return None
    return None


# FP32 lanes per SM (4 SMSPs x 32), SMs: the ALU roofline of the FFT kernels
FP32_LANES, N_SM = 128, 152


def roofline(prof, steps, config, sm_mhz):
    name = max(prof, key=lambda k: prof[k][0])
    ms, nl, by, fl = prof[name]
    per_launch_s = ms / 1e3 / nl
    peaks, tag = measured_peaks()
    gbs = by / nl / per_launch_s / 1e9
    tfl = fl / nl / per_launch_s / 1e12
    if name.startswith("dft_") and "fp32" not in name:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        r = {"bound": "tensor", "achieved": tfl, "peak": peak, "unit": "TFLOP/s", "frac": tfl / peak}
    else:
        alu_peak = 2.0 * FP32_LANES * N_SM * (peaks.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
        hbm = peaks["hbm_gbs"]
        if gbs / hbm >= tfl / alu_peak:
            r = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
        else:
            r = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfl / alu_peak,
                 "peak_basis": "FP32 FMA: 2 x 128 lanes x 152 SMs x 2.07 GHz"}
        r["hbm_gbs_achieved"] = gbs
        r["fp32_tflops_achieved"] = tfl
    r.update({"kernel": name, "launches_per_step": nl / steps, "ms_per_launch": per_launch_s * 1e3,
              "algorithmic_bytes_per_launch": by / nl, "algorithmic_flops_per_launch": fl / nl,
              "traffic": ncu_traffic(name, config, by / nl), "peak_source": tag})
    return r


# ------------------------------------------------------------------------------------------
# weak scaling across ranks
# ------------------------------------------------------------------------------------------
def rank_seed_offset(rank):
    """Every rank simulates its own independently seeded trajectory."""
    return 1000 * rank


def aggregate_ranks(local_seconds, local_units, dist=None):
    """(value, max_seconds): all ranks' units over the slowest rank's time (no data exchange
    besides this one scalar reduction)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_units / local_seconds, local_seconds
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_seconds, float(local_units)], dtype=torch.float64, device=dev)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    units = t[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return float(units.item()) / float(tmax.item()), float(tmax.item())


# ------------------------------------------------------------------------------------------
# CPU baseline (the FP64 oracle as it stands) on a bounded sample
# ------------------------------------------------------------------------------------------
def cpu_baseline(w, budget_s=20.0):
    """The oracle on a bounded sample of the workload: frames in parallel (one per thread) and,
    for a probe scan, the first probes of the scan; rate = wave-slice steps of the sample / time."""
    import numpy as np

    import oracle
    oracle.build()
    p = oracle.params_of(w)
    threads = oracle.num_threads()
    scan = w.alpha_mrad > 0
    t0 = time.perf_counter()
    oracle.multislice(p, w.pos[:1], w.Z, w.form_Z, w.form_coef, w.alpha_mrad, w.probes[:1] if scan else None)
    t1 = time.perf_counter() - t0
    # frames run in parallel (one per thread): n frames take about ceil(n / threads) frame times
    if scan:
        # a frame's time is its potential plus k probe propagations: calibrate both parts
        t0 = time.perf_counter()
        oracle.multislice(p, w.pos[:1], w.Z, w.form_Z, w.form_coef, w.alpha_mrad, w.probes[:3])
        per_probe = max((time.perf_counter() - t0 - t1) / 2, 1e-3)
        fixed = max(t1 - per_probe, 0.0)
        n = min(w.n_frames, threads)
        k = max(1, min(w.n_probes, int((budget_s - fixed) / per_probe)))
    else:
        n, k = max(1, min(w.n_frames, threads * max(1, int(budget_s / max(t1, 1e-3))))), 1
    probes = w.probes[:k] if scan else None
    t0 = time.perf_counter()
    psi = oracle.multislice(p, w.pos[:n], w.Z, w.form_Z, w.form_coef, w.alpha_mrad, probes)
    oracle.spectrum(psi)
    dt = time.perf_counter() - t0
    units = n * w.n_slices * k
    what = (f"{n} of {w.n_frames} frames x {k} of {w.n_probes} probe(s) x {w.n_slices} slices, multislice + "
            f"time transform of that sample, {dt:.1f} s; the rate is extrapolated to the whole workload")
    return {"value": units / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": what,
            "extrapolated": True}, psi, n, probes


# ------------------------------------------------------------------------------------------
# the reference arm: the oracle on the host cores
# ------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload, frames=args.frames)
    import oracle
    oracle.build()
    p = oracle.params_of(w)
    probes = w.probes if w.alpha_mrad > 0 else None
    # one frame per oracle thread (the oracle parallelises over frames), unless set
    per_step = max(1, int(args.ref_frames)) if args.ref_frames else max(1, oracle.num_threads())
    for _ in range(args.warmup):
        oracle.multislice(p, w.pos[:1], w.Z, w.form_Z, w.form_coef, w.alpha_mrad, probes)
    times = []
    # a probe scan times the first ref_probes probes of the scan per step (the rate is per wave)
    if probes is not None:
        probes = probes[:max(1, int(args.ref_probes))]
    n_pr = 1 if probes is None else len(probes)
    for k in range(args.steps):
        fr = w.pos[(k * per_step) % w.n_frames:][:per_step]
        t0 = time.perf_counter()
        psi = oracle.multislice(p, fr, w.Z, w.form_Z, w.form_coef, w.alpha_mrad, probes)
        oracle.spectrum(psi)
        times.append(time.perf_counter() - t0)
    units = per_step * w.n_slices * n_pr * args.steps
    tot = sum(times)
    v = units / tot
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, args.workload, "fp64 oracle"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{per_step} frame(s) x {n_pr} probe(s) per step of {w.n_frames} frames x "
                                   f"{w.n_probes} probe(s), multislice + time transform"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------------------------------
# serving: Poisson-arriving requests, continuous batching vs the plain path
# ------------------------------------------------------------------------------------------
# the small mix of the default bench line; the serving configuration itself (--workload c5)
# draws from its full stated ranges (workloads.request_stream defaults: grids 128^2-1024^2,
# 64-1024 frames, 8-40 slices, 2-13 cubic cells per edge, plane waves or 4x4-16x16 scans)
SERVING_MIX = dict(grids=(128, 256, 512), frames=(64, 128, 256), slices=(8, 20), reps=(2, 5), scans=(2, 4),
                   p_plane=0.5)
FULL_MIX = dict(grids=(128, 256, 512, 1024), frames=(64, 128, 256, 512, 1024), slices=(8, 40), reps=(2, 13),
                scans=(4, 16), p_plane=0.5)


def run_serving(T, n_requests, seed=5, rate_factor=0.8, device=0, mix=None, warm=True, plain_sample=None,
                n_geometries=None, streams=None):
    """Serve n_requests seeded requests arriving as a Poisson stream at rate_factor x the
    measured batched capacity; compare with the plain path (requests one by one).  Plane-wave
    requests return the full S, probe scans the detector-summed spectrum image.
    mix: request ranges (SERVING_MIX or FULL_MIX); warm: run every request once first (tables,
    operands, pools); plain_sample: time the plain path on a seeded sample of that many requests
    and extrapolate it to the whole stream by pixel-slice work (None: every request);
    n_geometries: draw the requests from that many geometries (repeated screening), and also
    time the batched capacity without coalescing same-geometry requests."""
    import numpy as np
    import torch

    import workloads
    mix = SERVING_MIX if mix is None else mix
    specs = workloads.request_stream(n_requests, seed=seed, rate_hz=1.0, n_geometries=n_geometries, **mix)
    ws = [workloads.request_workload(sp) for sp in specs]
    fz, fc = workloads.placeholder_form_factors(sorted(set(int(z) for w in ws for z in w.Z)))
    reqs = []
    for w in ws:
        red = T.REDUCE_NONE if w.alpha_mrad <= 0 else T.REDUCE_DETECTOR
        shape = (w.n_probes, w.n_frames, w.ny, w.nx) if red == T.REDUCE_NONE else (w.n_probes, w.n_frames)
        reqs.append(dict(w=w, red=red, pos=torch.from_numpy(w.pos).cuda(), Z=np.ascontiguousarray(w.Z),
                         out=torch.empty(shape, dtype=torch.float32, device="cuda"), pr=T.probe_of(w)))
    # the context after the request buffers: its serving budget is 90% of the memory left
    ctx = T.Context(device)
    ctx.load_form_factors(fz, fc)
    if streams:
        ctx.set_option("serving_streams", streams)
    work = lambda r: r["w"].n_probes * r["w"].n_frames * r["w"].n_slices
    pxwork = lambda r: work(r) * r["w"].nx * r["w"].ny
    units = sum(work(r) for r in reqs)
    spectra = sum(r["w"].n_probes for r in reqs)

    def one(r, prec):
        w = r["w"]
        T.tacaw_run(ctx.h, T.params_of(w), r["pos"], r["Z"], w.n_atoms, w.n_frames, r["pr"], prec, r["red"], r["out"])

    batch = []  # requests in the run each request was part of (coalescing), last serve() call

    def serve(prec, arrivals):
        tickets = []
        t0 = time.perf_counter()
        for r, a in zip(reqs, arrivals):
            dt = t0 + a - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            w = r["w"]
            req = T.make_request(T.params_of(w), r["pos"], r["Z"], w.n_atoms, w.n_frames, r["pr"], prec, r["red"],
                                 r["out"])
            tickets.append(T.tacaw_submit(ctx.h, req))
        lat, first, last = [], None, None
        batch.clear()
        for t in tickets:
            rc, res = T.tacaw_wait(ctx.h, t, 3600.0)
            if rc != T.TACAW_OK:
                raise RuntimeError(f"serving request failed: {rc}")
            lat.append(res.t_done - res.t_submit)
            batch.append(res.batched)
            first = res.t_submit if first is None else min(first, res.t_submit)
            last = res.t_done if last is None else max(last, res.t_done)
        return lat, last - first

    if warm:
        for r in reqs:
            one(r, T.DFT_BF16X3)
            one(r, T.DFT_FP32)
        torch.cuda.synchronize()
    # plain path: one frame per launch batch, FP32 SIMT transform, one request at a time
    if plain_sample is None or plain_sample >= len(reqs):
        sample = list(range(len(reqs)))
    else:
        sample = sorted(np.random.default_rng(seed).choice(len(reqs), plain_sample, replace=False).tolist())
    ctx.set_option("max_chunk_frames", 1)
    plain_lat = []
    t0 = time.perf_counter()
    for i in sample:
        a = time.perf_counter()
        one(reqs[i], T.DFT_FP32)
        torch.cuda.synchronize()
        plain_lat.append(time.perf_counter() - a)
    plain_sample_s = time.perf_counter() - t0
    ctx.set_option("max_chunk_frames", 0)
    extrap = len(sample) < len(reqs)
    plain_s = plain_sample_s * (sum(pxwork(r) for r in reqs) / sum(pxwork(reqs[i]) for i in sample))
    # batched capacity: everything submitted at once
    cap_nocoal_s = None
    if n_geometries:
        ctx.set_option("max_coalesce", 1)
        _, cap_nocoal_s = serve(T.DFT_BF16X3, [0.0] * len(reqs))
        ctx.set_option("max_coalesce", 16)
    _, cap_s = serve(T.DFT_BF16X3, [0.0] * len(reqs))
    rate = rate_factor * len(reqs) / cap_s
    arrivals = [sp.arrival_s / rate for sp in specs]
    lat, span = serve(T.DFT_BF16X3, arrivals)
    coalesced = sum(1 for b in batch if b > 1)
    ctx.check()
    ctx.close()
    pct = lambda x, q: float(np.percentile(np.asarray(x), q))
    plain_what = "requests one by one: one frame per launch batch, FP32 SIMT time transform"
    if extrap:
        plain_what += (f"; timed on a seeded sample of {len(sample)} of {len(reqs)} requests "
                       f"({plain_sample_s:.1f} s) and extrapolated by pixel-slice work")
    return {
        "requests": len(reqs), "spectra": spectra, "wave_slice_steps": units,
        "mix": {k: list(v) if isinstance(v, tuple) else v for k, v in mix.items()},
        "arrival_rate_hz": rate, "offered_load": rate_factor,
        "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
        "spectra_per_s": spectra / span, "wave_slice_steps_per_s": units / span,
        "batched_capacity_spectra_per_s": spectra / cap_s,
        "plain_path": {"spectra_per_s": spectra / plain_s, "wave_slice_steps_per_s": units / plain_s,
                       "p50_latency_s": pct(plain_lat, 50), "p99_latency_s": pct(plain_lat, 99),
                       "latencies_from": f"{len(sample)} requests", "extrapolated": extrap, "what": plain_what},
        "capacity_speedup_vs_plain": (spectra / cap_s) / (spectra / plain_s),
        "served_rate_vs_plain": (spectra / span) / (spectra / plain_s),
        "precision": "bf16x3 served, fp32 plain (both within 1e-4 of the oracle in the tests)",
        "warmed": warm,
        "coalesced_requests": coalesced, "mean_run_size": float(np.mean(batch)) if batch else 1.0,
        "serving_streams": streams or 4,
        **({"geometries": n_geometries,
            "capacity_without_coalescing_spectra_per_s": spectra / cap_nocoal_s,
            "coalescing_speedup": cap_nocoal_s / cap_s} if n_geometries else {}),
    }


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5", "m1", "m1s"])
    ap.add_argument("--precision", default="bf16x3", choices=sorted(PRECISIONS))
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-frames", type=int, default=0, help="frames per reference step (0: one per host thread)")
    ap.add_argument("--ref-probes", type=int, default=2, help="probes of a scan per reference step")
    ap.add_argument("--frames", type=int, default=None, help="truncate the trajectory (profiling cases)")
    ap.add_argument("--probes", type=int, default=None, help="truncate the probe scan (profiling cases)")
    ap.add_argument("--option", action="append", default=[], metavar="NAME=VALUE",
                    help="context option (tacaw_set_option) for the timed runs, e.g. max_chunk_frames=2")
    ap.add_argument("--serving-requests", type=int, default=24, help="requests in the serving run (0: skip)")
    ap.add_argument("--serving-streams", type=int, default=0, help="c5: serving streams (0: the library default)")
    ap.add_argument("--serving-mix", default="full", choices=["full", "small"],
                    help="c5: the configuration's full request ranges, or the small mix of the default line")
    ap.add_argument("--serving-geometries", type=int, default=0,
                    help="c5: draw the requests from this many geometries (repeated screening; 0: all distinct)")
    ap.add_argument("--plain-sample", type=int, default=16,
                    help="c5: requests of the stream the plain path is timed on (0: all)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if args.workload == "c5":
        return main_serving(args, rank, world, local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_2602_10064_gb300 as T

    w = make_workload(args.workload, seed_offset=rank_seed_offset(rank), frames=args.frames, probes=args.probes)
    prec = PRECISIONS[args.precision]
    ctx = T.Context(local)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    for opt in args.option:
        name, value = opt.split("=")
        ctx.set_option(name.strip(), int(value))
    params, probe = T.params_of(w), T.probe_of(w)
    pos = torch.from_numpy(w.pos).cuda()
    Z = torch.from_numpy(w.Z).cuda()
    P, F = w.n_probes, w.n_frames
    red = T.REDUCE_DETECTOR if reduce_of(w) == "detector" else T.REDUCE_NONE
    out_shape = (P, F) if red == T.REDUCE_DETECTOR else (P, F, w.ny, w.nx)
    S = torch.empty(out_shape, dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def step():
        T.tacaw_run(ctx.h, params, pos, Z, w.n_atoms, F, probe, prec, red, S, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # one more untimed step with an event pair around every kernel: the per-kernel breakdown,
    # and the dominant kernel, the only one the timed steps put events around
    T.tacaw_profile_select(ctx.h, "")
    T.tacaw_profile_begin(ctx.h)
    step()
    torch.cuda.synchronize()
    prof_all = T.tacaw_profile_end(ctx.h)
    dominant = max(prof_all, key=lambda k: prof_all[k][0])
    T.tacaw_profile_select(ctx.h, dominant)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    T.tacaw_profile_begin(ctx.h)
    for k in range(args.steps):
        flush.fill_(float(k))  # evict L2 between timed steps (not timed)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    prof = T.tacaw_profile_end(ctx.h)  # the dominant kernel timed; every launch counted
    T.tacaw_profile_select(ctx.h, "")
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    units_rank = P * F * w.n_slices * args.steps
    value, tot_s = aggregate_ranks(sum(step_ms) / 1e3, units_rank, dist)
    spectra = P * args.steps * world / tot_s

    # end to end through the C ABI with host buffers: H2D of the positions and species,
    # D2H of S, inside the timed region
    if args.e2e_steps < 1:
        args.e2e_steps = 0
    pos_h = torch.from_numpy(w.pos).pin_memory()
    Z_h = torch.from_numpy(w.Z)
    S_h = torch.empty(out_shape, dtype=torch.float32).pin_memory()
    T.tacaw_run(ctx.h, params, pos_h, Z_h, w.n_atoms, F, probe, prec, red, S_h, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    call_ms = []
    t0 = time.perf_counter()
    for _ in range(max(args.e2e_steps, 1)):
        t1 = time.perf_counter()
        T.tacaw_run(ctx.h, params, pos_h, Z_h, w.n_atoms, F, probe, prec, red, S_h, stream)
        call_ms.append((time.perf_counter() - t1) * 1e3)  # the call returns once S is on the host
    torch.cuda.synchronize()
    e2e_value, _ = aggregate_ranks(time.perf_counter() - t0, units_rank // args.steps * max(args.e2e_steps, 1), dist)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(w.pos.nbytes + w.Z.nbytes), "d2h_bytes_per_step": int(S_h.numel() * 4),
           "steps": args.e2e_steps, "call_ms": [round(x, 2) for x in call_ms],
           "api": "tacaw_run with pinned host pos/Z/S"}

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return
    launches = sum(v[1] for v in prof.values())  # all kernel launches of the timed region
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded harmonic-mode trajectory; placeholder Kirkland-form table)",
        "config": dict(workload_config(w, args.workload, args.precision),
                       **({"options": args.option} if args.option else {})),
        "spectra_per_s": spectra, "px_slices_per_s": value * w.nx * w.ny,
        "step_ms": step_ms,
        "roofline": roofline(prof, args.steps, args.workload, clk.get("sm_mhz")),
        "kernels": {k: {"ms_per_step": v[0], "launches_per_step": v[1],
                        "gbs": v[2] / max(v[0], 1e-9) / 1e6, "tflops": v[3] / max(v[0], 1e-9) / 1e9}
                    for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1][0])},
        "kernels_from": "one untimed step after the warm-up, an event pair around every kernel; "
                        "the timed steps put events around the dominant kernel only",
        "gpu_launches": int(round(launches)),
        "clocks": clk, "e2e": e2e,
    }
    if world == 1 and args.serving_requests > 0:
        out["serving"] = run_serving(T, args.serving_requests, device=local)
    if world == 1 and not args.no_cpu_baseline:
        cb, psi_ref, n, probes_s = cpu_baseline(w, args.cpu_seconds)
        out["cpu_baseline"] = cb
        # the same frames (and probes) on the GPU: exit-wave agreement at full size
        V = ctx.build_potential(params, pos[:n].contiguous(), Z)
        pr_s = probe if probes_s is None else T.ProbeSpec(w.alpha_mrad, probes_s)
        psi = ctx.propagate(params, V, pr_s).cpu().numpy()
        err = float(np.linalg.norm(psi - psi_ref) / np.linalg.norm(psi_ref))
        out["tol"] = {"psi_rel_l2_vs_oracle": err, "frames": n, "probes": 1 if probes_s is None else len(probes_s),
                      "S_rel_l2_bound": "1e-4 (tests/test_gpu_parity.py at oracle sizes)"}
    ctx.close()
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def main_serving(args, rank, world, local):
    """--workload c5: the 200-request serving stream is the step; value = served wave-slice steps/s."""
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    n = args.serving_requests if args.serving_requests > 24 else 200
    clocks = ClockSampler(local)
    clocks.start()
    mix = FULL_MIX if args.serving_mix == "full" else SERVING_MIX
    r = run_serving(T, n, seed=5 + 1000 * rank, device=local, mix=mix, warm=False,
                    plain_sample=args.plain_sample or None, n_geometries=args.serving_geometries or None,
                    streams=args.serving_streams or None)
    clk = clocks.stop()
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": r["wave_slice_steps_per_s"] * world, "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": r["wave_slice_steps"] / r["wave_slice_steps_per_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic request stream (seeded cubic/rocksalt cells, Poisson arrivals)",
        "config": {"workload": f"c5-serving-{n}-requests" + (f"-{args.serving_geometries}-geometries"
                                                              if args.serving_geometries else ""),
                   "mix": r["mix"]}, "serving": r, "clocks": clk,
        "spectra_per_s": r["spectra_per_s"], "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"]}))


if __name__ == "__main__":
    main()
