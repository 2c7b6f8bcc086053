#!/usr/bin/env python3
"""Benchmark: visibilities/sec for degrid and grid at eps = 1e-5 (FP32) and 1e-12 (FP64).

Workload (default ``wide_2k``): 2048^2 image at 20 arcsec, 999,936 visibilities from a
64-antenna earth-rotation synthesis (2016 baselines x 62 time steps x 8 channels in
0.9-1.7 GHz), point-source image (1% of pixels, log-normal flux), complex N(0, 1) data.

One step = the four operator applications on that input: degrid + grid at eps = 1e-5 in
FP32 and degrid + grid at eps = 1e-12 in FP64, each on a resident plan (index built once,
outside the timed region).  ``value`` = 4 * nvis / step time.  The L2 cache is flushed
between steps (256 MiB write), steps are timed with CUDA events on the launching stream,
nvidia-smi clocks are sampled during the timed region.

``--impl reference`` times the FP64 direct-sum oracle on the host cores on a bounded sample
of the same workload (the reference arm); without it the oracle is timed once as the
``cpu_baseline`` (rank 0, N = 1 only).  Under torchrun (N > 1) every rank runs an
independent replica (the path is "replicas only"), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "visibilities/sec for degrid and grid on 1 GB300 at eps=1e-5 (FP32) and 1e-12 (FP64)"
MODES = (("f32", 1e-5), ("f64", 1e-12))
FFT_NAMES = {1: "cuFFT 2-D", 2: "double-float (pruned rows)", 3: "cuFFT Z2Z (pruned rows)",
             4: "library FP32 (pruned rows)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wgrid", choices=["wgrid", "reference"])
    ap.add_argument("--workload", default="wide_2k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-seconds", type=float, default=12.0)
    ap.add_argument("--modes", default="f32,f64",
                    help="precision modes in a step (f32 = eps 1e-5, f64 = eps 1e-12)")
    ap.add_argument("--fft-impl", type=int, default=0,
                    help="plane FFT (0 automatic, 1 cuFFT, 4 the library's FP32 FFT for the FP32 mode)")
    ap.add_argument("--grid-variant", type=int, default=0,
                    help="gridding accumulation (0 automatic, 1 shared atomics, 2 plane-owner warps)")
    ap.add_argument("--sweep", action="store_true",
                    help="precision sweep on the workload: vis/s and sampled error per epsilon")
    ap.add_argument("--serve", action="store_true",
                    help="continuous-batching serving benchmark (p50/p99 latency, vis/s)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-obs", type=int, default=32)
    ap.add_argument("--serve-sizes", default="512,1024,2048,4096,8192")
    ap.add_argument("--serve-vis", default="1e5,5e7")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-loads", default="0.5,0.9",
                    help="Poisson arrival rates as multiples of the one-at-a-time capacity")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave out the bounded serving sub-mix of the default run")
    ap.add_argument("--modes-1e8", default="f32,f64",
                    help="modes of the 1e8-visibility block (\"none\": skip it)")
    ap.add_argument("--steps-1e8", type=int, default=2)
    ap.add_argument("--only", default=None,
                    help="profiling aid: run only one call per step, e.g. f64:grid or f32:degrid")
    return ap.parse_args()


def dist_env():
    from paper_2010_10122_gb300 import replicas
    return replicas.world()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
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
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax = float(parts[2]); power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------------------
# oracle (CPU) timing on a bounded sample
# ------------------------------------------------------------------------------------------
def oracle_rate(obs, I, d, seconds):
    """Direct-sum terms per second of the oracle on this host, measured on a bounded sample:
    degrid of a few visibilities (each a sum over all pixels) and grid of a few pixels (each
    a sum over all visibilities), on all host cores and on one core.  Returns (vis_per_s,
    cores, sample description, step seconds, vis_per_s on one core)."""
    from oracle import direct
    direct.build()
    rng = np.random.default_rng(0)
    npix = obs.npix_x * obs.npix_y
    nnz = int(np.count_nonzero(I))     # the oracle skips zero pixels in degrid
    # one core: a few visibilities and pixels on one thread (also the calibration)
    v1 = rng.choice(obs.nvis, size=8, replace=False)
    t0 = time.perf_counter()
    direct.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y, vis_index=v1, nthreads=1)
    t1v = (time.perf_counter() - t0) / len(v1)
    p1 = rng.choice(npix, size=2, replace=False)
    t0 = time.perf_counter()
    direct.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                pixel_index=p1, nthreads=1)
    t1p = (time.perf_counter() - t0) / len(p1)
    step1 = 2 * (obs.nvis * t1v + npix * t1p)
    cores = direct.threads_used(0)
    nv = int(max(cores, min(200000, 0.5 * seconds / max(t1v, 1e-9) * cores)))
    vsel = rng.choice(obs.nvis, size=min(nv, obs.nvis), replace=False)
    t0 = time.perf_counter()
    direct.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y, vis_index=vsel)
    td = time.perf_counter() - t0
    degrid_vps = len(vsel) / td                      # visibilities degridded per second
    # grid: one pixel costs nvis terms
    npx = int(max(cores, min(npix, 0.5 * seconds / max(t1p, 1e-9) * cores)))
    psel = rng.choice(npix, size=npx, replace=False)
    t0 = time.perf_counter()
    direct.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y, pixel_index=psel)
    tg = time.perf_counter() - t0
    grid_vps = obs.nvis / (tg * npix / len(psel))    # full image takes npix/len(psel) x longer
    # one step = degrid + grid in each of the two modes (the oracle is FP64 in both)
    step_s = 2 * (obs.nvis / degrid_vps + obs.nvis / grid_vps)
    sample = (f"degrid of {len(vsel)} sampled visibilities against all {nnz} nonzero pixels "
              f"({td:.1f} s) and grid of {len(psel)} sampled pixels over all {obs.nvis} "
              f"visibilities ({tg:.1f} s) on {cores} threads, extrapolated to the full workload; "
              f"one core: {len(v1)} visibilities and {len(p1)} pixels, extrapolated")
    return 4 * obs.nvis / step_s, cores, sample, step_s, 4 * obs.nvis / step1


def make_inputs(workload):
    from paper_2010_10122_gb300 import synthetic as S
    obs = S.WORKLOADS[workload]()
    I = S.point_source_image(obs.npix_x, obs.npix_y, seed=0)
    d = S.complex_normal((obs.nrows, obs.nchan), seed=1)
    return obs, I, d


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    obs, I, d = make_inputs(args.workload)
    per_step = max(2.0, args.oracle_seconds / max(1, args.steps + args.warmup))
    rates = []
    cores = sample = None
    for i in range(args.warmup + args.steps):
        vps, cores, sample, _, _ = oracle_rate(obs, I, d, per_step)
        if i >= args.warmup:
            rates.append(vps)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "vis/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 4 * obs.nvis / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nvis": obs.nvis,
                       "npix": [obs.npix_x, obs.npix_y], "modes": ["f32 eps=1e-5", "f64 eps=1e-12"]},
            "cpu_baseline": {"value": value, "unit": "vis/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "vis/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def algorithmic_flops_per_vis(alpha):
    """FLOPs a (de)gridding kernel must do per visibility: alpha^3 complex-by-real
    multiply-adds over the alpha planes x alpha x alpha cells (4 flops each), plus 3 alpha
    kernel values by Horner of degree alpha + 3 (2 flops per step)."""
    return 4 * alpha ** 3 + 3 * alpha * 2 * (alpha + 3)


# FP32 arithmetic instructions of the double-float FFT (paper_2010_10122_gb300/csrc/fft_df64.cu),
# counted from its operations: double-float add 11 (two-sum 6, two adds, renormalisation 3),
# product 7, complex add 22, scale by a constant 14, twiddle product 38 (two fused two-product
# sums of 19), fused multiply-add 15; butterflies: radix 2 44, 3 160, 4 176, 5 464, 8 600, and
# the symmetric odd radices R = 7, 11 (P = (R - 1) / 2: (R - 1) + P complex adds, then per output
# pair 4 P fused multiply-adds and 2 complex adds) 870 and 2050.
DF64_BUTTERFLY = {2: 44, 3: 160, 4: 176, 5: 464, 7: 870, 8: 600, 11: 2050}


def df64_radices(n):
    """Radix plan of a double-float line transform (8s and 4s for the power of two, a single 2
    only for n = 2 x odd, then 5, 3, 7, 11) -- the plan the library uses."""
    m, p2 = n, 0
    while m % 2 == 0:
        m //= 2
        p2 += 1
    r = []
    if p2 == 1:
        r.append(2)
    else:
        e8, rem = p2 // 3, p2 % 3
        if rem == 1:
            e8 -= 1
        r += [8] * e8 + ([4, 4] if rem == 1 else [4] if rem == 2 else [])
    for p in (5, 3, 7, 11):
        while m % p == 0:
            r.append(p)
            m //= p
    return r


def df64_part_ops(n):
    """FP32 instructions of one length-n double-float transform held by one CTA (butterflies and
    the twiddle products of every stage after the first)."""
    ops, ns = 0, 1
    for r in df64_radices(n):
        bf = DF64_BUTTERFLY[r]
        ops += (n // r) * (bf + (38 * (r - 1) if ns > 1 else 0))
        ns *= r
    return ops


def df64_line_split(n):
    """CTAs per double-float line, the library's rule: up to 6400 points one CTA, except that
    above 2048 a line whose half needs only the radices 8, 4, 5, 3 runs as two halves; longer
    lines on 2 or 4 CTAs of at most 6400 points (each split line on a thread-block cluster)."""
    def plan_ok(m):
        k = m
        for p in (2, 3, 5, 7, 11):
            while k % p == 0:
                k //= p
        return m >= 2 and k == 1
    if n <= 6400:
        if n > 2048 and n % 2 == 0 and plan_ok(n // 2) and \
                not set(df64_radices(n // 2)) & {2, 7, 11}:
            return 2
        return 1
    for s in (2, 4):
        if n % s == 0 and n // s <= 6400:
            return s
    return 0


def df64_line_ops(n):
    """FP32 instructions of one length-n double-float line: one CTA's transform, or for a line
    on S CTAs the radix-S decimation step (butterfly and S - 1 twiddle products per group of S)
    and S transforms of n / S points."""
    S = df64_line_split(n)
    if S <= 1:
        return df64_part_ops(n)
    return (n // S) * (DF64_BUTTERFLY[S] + 38 * (S - 1)) + S * df64_part_ops(n // S)


# DRAM bytes the double-float FFT moved per algorithmic byte (one 16-byte read and one 16-byte
# write per cell and pass), measured by ncu on full 3456^2 transforms (lines as two halves on
# clusters of 2 CTAs): 30.86 of 32 B per cell and pass (profiles/k_fft_lines_cluster_df64_3456.md);
# the rest stays in L2 when the kernel ends
DF64_DRAM_PER_ALGORITHMIC_BYTE = 30.86 / 32.0


def df64_fft_bytes(nx, ny, nu, nv, direction):
    """Algorithmic bytes of one plane's double-float FFT in the library's pruned form (16 B per
    cell read or written): degrid (forward) -- column pass over the ny image columns loading
    their nx image rows and storing nu, row pass over all nu rows loading their ny image cells
    and storing nv; grid (inverse) -- row pass over all nu x nv cells storing the ny image
    columns, column pass over those loading nu and storing the nx image rows."""
    if direction == "degrid":
        return 16 * (nx * ny + nu * ny) + 16 * (nu * ny + nu * nv)
    return 16 * (nu * nv + nu * ny) + 16 * (nu * ny + nx * ny)


def run_sweep(args):
    """Precision sweep (eps in {1e-3, 1e-5 FP32; 1e-7, 1e-10, 1e-12 FP64}): per epsilon the
    degrid and grid vis/s (CUDA events, resident plan) and the relative L2 error against the
    oracle on sampled visibilities / pixels.  One JSON line per epsilon."""
    import torch
    import paper_2010_10122_gb300 as wg
    from oracle import direct
    direct.build()
    obs, I, d = make_inputs(args.workload)
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(0)
    vsel = rng.choice(obs.nvis, 256, replace=False)
    psel, nb, share = stratified_pixels(obs.npix_x, obs.npix_y, seed=1)
    rv = direct.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y, vis_index=vsel)
    ri = direct.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                     pixel_index=psel)
    for prec, eps in (("f32", 1e-3), ("f32", 1e-5), ("f64", 1e-7), ("f64", 1e-10), ("f64", 1e-12)):
        rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
        plan = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                       eps, prec, device=dev)
        dimg = torch.from_numpy(I).to(dev, rdt)
        dvis = torch.from_numpy(d).to(dev, cdt)
        res = {}
        for direction in ("degrid", "grid"):
            fn = (lambda: plan.degrid(dimg)) if direction == "degrid" else (lambda: plan.grid(dvis))
            out = fn()
            torch.cuda.synchronize()
            times = []
            for _ in range(max(1, args.steps)):
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(); out = fn(); e1.record(); e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            o = out.cpu().numpy()
            err = (direct.rel_l2(o.reshape(-1)[vsel], rv) if direction == "degrid"
                   else stratified_rel_l2(o.reshape(-1)[psel], ri, nb, share))
            res[direction] = {"ms": ms, "vis_per_s": obs.nvis / (ms * 1e-3), "rel_l2_err": err}
            del out
        info = plan.info
        print(json.dumps({"sweep": args.workload, "precision": prec, "eps": eps,
                          "alpha": info["alpha"], "sigma": info["sigma"],
                          "uv_grid": [info["nu"], info["nv"]], "nw": info["nw"],
                          "fft": FFT_NAMES[info["fft_impl"]], "err_model": info["err_model"],
                          **res, "error_sample": f"256 visibilities; {len(psel)} pixels stratified "
                                                 f"({nb} within {EDGE_BAND} of the image edge, "
                                                 f"weighted by area) vs the FP64 oracle"}),
              flush=True)
        plan.close()
        del dimg, dvis
        torch.cuda.empty_cache()
    return 0


def serve_benchmark(n_requests, n_obs, sizes, vis_range, slots, budget_gb, loads, seed=5,
                    workspace_cap_gb=8.0, serial_sample=200):
    """Continuous-batching serving benchmark: resident observations of mixed image sizes and
    visibility counts (64-antenna array, 16 channels, time steps chosen to hit the count),
    Poisson arrivals of mixed degrid / grid requests at eps in {1e-4, 1e-5 (FP32), 1e-12
    (FP64)}, admission by stream slots and a device-memory budget (plans, workspaces and
    outputs), plans built off the scheduler thread.  The one-at-a-time capacity is measured on
    `serial_sample` distinct requests; the served lists repeat that mix up to `n_requests` and
    arrive at each load (arrival rate as a multiple of that capacity).  Returns a dict of p50 /
    p99 latency and served vis/s per load beside the one-at-a-time vis/s."""
    import torch
    from paper_2010_10122_gb300 import synthetic as S
    from paper_2010_10122_gb300.server import CudaExecutor, Request, Server, run_serial
    rng = np.random.default_rng(seed)
    vlo, vhi = vis_range
    obs = {}
    for i in range(n_obs):
        n = sizes[rng.integers(len(sizes))]
        nvis = int(np.exp(rng.uniform(np.log(vlo), np.log(vhi))))
        nt = max(1, nvis // (2016 * 16))
        pix = 20 * S.ARCSEC * 2048 / n      # same field of view (11.4 deg) for every size
        obs[f"obs{i}"] = S.array_observation(64, nt, 16, n, pix, seed=100 + i)
    keys = sorted(obs)
    epss = [(1e-4, "f32"), (1e-5, "f32"), (1e-12, "f64")]
    # one device input per (observation, direction, precision), shared by the requests that use
    # it (the mix would otherwise hold every request's input on the device at once)
    inputs = {}

    def data_for(k, direction, prec):
        key = (k, direction, prec)
        if key not in inputs:
            o = obs[k]
            seed_ = 1000 + keys.index(k)
            if direction == "degrid":
                inputs[key] = torch.from_numpy(S.point_source_image(o.npix_x, o.npix_y, seed=seed_)).to(
                    "cuda", torch.float32 if prec == "f32" else torch.float64)
            else:
                inputs[key] = torch.from_numpy(S.complex_normal((o.nrows, o.nchan), seed=seed_)).to(
                    "cuda", torch.complex64 if prec == "f32" else torch.complex128)
        return inputs[key]

    # the request mix: `serial_sample` distinct (observation, direction, epsilon) draws; the
    # served lists repeat that mix (each draw n_requests / serial_sample times, in a random
    # order), so that served and one-at-a-time throughput are taken on the same composition
    r = np.random.default_rng(2)
    specs = []
    for _ in range(min(serial_sample, n_requests)):
        k = keys[r.integers(len(keys))]
        eps, prec = epss[r.integers(len(epss))]
        specs.append((k, "degrid" if r.uniform() < 0.5 else "grid", eps, prec))

    def make(nreq, s_):
        order = np.random.default_rng(s_).permutation(nreq) % len(specs)
        return [Request(k, d, data_for(k, d, prec), eps, prec)
                for k, d, eps, prec in (specs[i] for i in order)]

    budget = int(budget_gb * (1 << 30))
    ex = CudaExecutor(obs, slots=slots, workspace_cap=int(workspace_cap_gb * (1 << 30)),
                      keep_results=False)
    sample = make(len(specs), 2)
    t0 = time.perf_counter()
    for r in sample:                    # the sample's plans (built here, not timed)
        ex.plan_bytes(r.obs, r.epsilon, r.precision)
    plan_s = time.perf_counter() - t0
    plan_gb = sum(ex.resident_plans().values()) / (1 << 30)
    run_serial(ex, sample[: min(8, len(sample))])          # warm-up
    torch.cuda.synchronize()
    t_serial = run_serial(ex, sample)
    serial_vis = sum(ex.plans[(r.obs, r.epsilon, r.precision)].info["nvis"] for r in sample)
    rate_req = len(sample) / t_serial
    del sample
    out = {"serve": "continuous batching", "requests": n_requests, "observations": n_obs,
           "image_sizes": sizes, "vis_range": [vlo, vhi], "eps_mix": [e for e, _ in epss],
           "slots": slots, "budget_gb": budget_gb, "workspace_cap_gb": workspace_cap_gb,
           "plans_built_s": round(plan_s, 1), "plans_resident_gb": round(plan_gb, 2),
           "one_at_a_time": {"requests": len(specs), "s": t_serial,
                             "vis_per_s": serial_vis / t_serial, "requests_per_s": rate_req},
           "loads": [], "inputs_gb": round(sum(t.numel() * t.element_size() for t in inputs.values()) / (1 << 30), 2),
           "warm_up": "one unreported pass at twice the capacity grows the stream-ordered pools",
           "mix": f"the served lists repeat the {len(specs)} one-at-a-time requests"}
    for load in [None] + list(loads):
        reqs = make(n_requests, 3)
        t = 0.0
        arr = np.random.default_rng(11)
        for r in reqs:
            t += arr.exponential(1.0 / ((load or 2.0) * rate_req))
            r.arrival = t
        srv = Server(ex, slots=slots, memory_budget=budget)
        srv.adopt(ex.resident_plans())     # plans already built count against the budget
        srv.run(reqs if load is not None else reqs[: max(slots * 4, n_requests // 10)])
        torch.cuda.synchronize()
        rep = srv.report()
        if load is None:
            continue
        out["loads"].append({"load": load, "arrival_rate_per_s": load * rate_req,
                             "p50_latency_s": rep.get("p50_s"), "p99_latency_s": rep.get("p99_s"),
                             "mean_latency_s": rep.get("mean_s"), "vis_per_s": rep.get("vis_per_s"),
                             "served_span_s": rep.get("span_s"), "failed": rep.get("failed"),
                             "errors": rep.get("errors"),
                             "max_inflight": rep.get("max_inflight"),
                             "plan_waits": rep.get("plan_waits"),
                             "peak_memory_gb": rep.get("peak_memory", 0) / (1 << 30)})
        out["inputs_gb"] = round(sum(t.numel() * t.element_size() for t in inputs.values()) / (1 << 30), 2)
        del reqs
        torch.cuda.empty_cache()
    ex.close()
    return out


def run_serve(args):
    """The serving benchmark at the flags' sizes (default: the full mix of 2000 requests over 32
    observations, images 512^2 - 8192^2, 1e5 - 5e7 visibilities, 150 GB budget)."""
    from paper_2010_10122_gb300 import _build
    _build.build()
    import torch
    torch.cuda.set_device(0)
    line = serve_benchmark(args.serve_requests, args.serve_obs,
                           [int(x) for x in args.serve_sizes.split(",")],
                           tuple(float(x) for x in args.serve_vis.split(",")),
                           args.serve_slots, args.serve_budget_gb,
                           [float(x) for x in args.serve_loads.split(",")])
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# algorithmic bytes (scope-table accounting) and per-stage roofline fractions
# ------------------------------------------------------------------------------------------
STAGE_KEYS = {"screen": "ms_screen", "fft": "ms_fft", "gridding": "ms_grid", "accumulate": "ms_accum"}


def bytes_8d(info, obs, prec, direction):
    """Algorithmic HBM bytes of one operator call, per stage: every w-plane cell (b = 8 bytes in
    FP32, 16 in FP64) is written once by the screen, read and written once by the plane FFT,
    read once by the degridding, read and written once by the gridding, and read once by the
    accumulation (k_plane = 4 for degrid, 5 for grid); the (de)gridding also moves the
    visibilities (b each), a 4-byte index entry per visibility and the 24-byte uvw rows."""
    b = 8 if prec == "f32" else 16
    cells = info["nu"] * info["nv"] * info["nw"]
    vis_b = obs.nvis * (b + 4) + obs.nrows * 24
    if direction == "degrid":
        return {"screen": cells * b, "fft": 2 * cells * b, "gridding": cells * b + vis_b}
    return {"gridding": 2 * cells * b + vis_b, "fft": 2 * cells * b, "accumulate": cells * b}


def stage_fractions(stats, info, obs, prec, direction, hbm_gbs):
    """Per stage and for the whole call: algorithmic bytes / HBM peak / measured time."""
    by = bytes_8d(info, obs, prec, direction)
    out = {}
    for st, nb in by.items():
        ms = stats[STAGE_KEYS[st]]
        out[st] = {"bytes": nb, "ms": round(ms, 4),
                   "frac": (nb / (hbm_gbs * 1e9)) / (ms * 1e-3) if ms > 0 else None}
    tot = sum(by.values())
    out["call"] = {"bytes": tot, "ms": round(stats["ms_total"], 4),
                   "frac": (tot / (hbm_gbs * 1e9)) / (stats["ms_total"] * 1e-3)}
    return out


def median_stats(sts):
    return {k: statistics.median(s[k] for s in sts) for k in
            ("ms_total", "ms_prep", "ms_screen", "ms_fft", "ms_grid", "ms_accum")}


def make_plans(wg, obs, modes, dev, grid_variant=0, fft_impl=0):
    """Resident plans per precision mode, with their creation time (the index build, the
    per-pixel tables, the FFT set-up; wg_plan_create synchronises)."""
    import torch
    plans, plan_ms = {}, {}
    for prec, eps in modes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plans[prec] = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x,
                              obs.pixsize_y, eps, prec, device=dev, grid_variant=grid_variant,
                              fft_impl=fft_impl if (fft_impl != 4 or prec == "f32") else 0)
        plan_ms[prec] = (time.perf_counter() - t0) * 1e3
    return plans, plan_ms


# The gridded image's error is largest in a thin band at the image edge, where the 1 / psi
# correction amplifies the kernel and rounding errors (on the 1e8-visibility workload at eps =
# 1e-12: 1.8e-12 rms within 64 pixels of the edge, 3.6e-13 inside), so a uniform pixel sample
# estimates the image's relative L2 error (Sec. 5.2) with a large variance.  The pixel samples
# are therefore stratified: EDGE_SAMPLES pixels within EDGE_BAND of the edge and INTERIOR_SAMPLES
# inside, each stratum's mean squares weighted by its share of the image.
EDGE_BAND, EDGE_SAMPLES, INTERIOR_SAMPLES = 64, 192, 64


def stratified_pixels(nx, ny, seed=0, band=EDGE_BAND, nb=EDGE_SAMPLES, ni=INTERIOR_SAMPLES):
    """Flat pixel indices: nb within `band` pixels of the image edge, then ni inside (each sorted),
    with the edge band's share of the image."""
    rng = np.random.default_rng(seed)
    jx = np.arange(nx)[:, None]
    jy = np.arange(ny)[None, :]
    edge = np.minimum(np.minimum(jx, nx - 1 - jx), np.minimum(jy, ny - 1 - jy)).reshape(-1)
    bidx, iidx = np.flatnonzero(edge < band), np.flatnonzero(edge >= band)
    sb = np.sort(rng.choice(bidx, min(nb, len(bidx)), replace=False))
    si = np.sort(rng.choice(iidx, min(ni, len(iidx)), replace=False)) if len(iidx) else iidx
    return np.concatenate([sb, si]), len(sb), len(bidx) / edge.size


def stratified_rel_l2(x, ref, nb, band_share):
    """Relative L2 error of an image from a stratified pixel sample (edge stratum first): the
    squared error and the squared reference are each averaged per stratum and weighted by the
    strata's shares of the image."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    def mean_sq(a, lo, hi):
        return float(np.mean(a[lo:hi] ** 2)) if hi > lo else 0.0
    e2 = band_share * mean_sq(x - ref, 0, nb) + (1 - band_share) * mean_sq(x - ref, nb, len(x))
    r2 = band_share * mean_sq(ref, 0, nb) + (1 - band_share) * mean_sq(ref, nb, len(x))
    return float(np.sqrt(e2 / r2))


def error_sample(obs, nv, seed=0):
    """Uniform visibility sample and stratified pixel sample (indices, edge count, edge share)."""
    rng = np.random.default_rng(seed)
    vsel = np.sort(rng.choice(obs.nvis, nv, replace=False))
    return vsel, stratified_pixels(obs.npix_x, obs.npix_y, seed=seed + 1)


def gpu_samples(vout, gout, vsel, psel):
    """The GPU outputs at the sampled visibilities / pixels (host numpy, complex128 / float64)."""
    import torch
    vi = torch.from_numpy(vsel).to(vout.device)
    pi = torch.from_numpy(psel).to(gout.device)
    return (vout.reshape(-1).index_select(0, vi).cpu().numpy().astype(np.complex128),
            gout.reshape(-1).index_select(0, pi).cpu().numpy().astype(np.float64))


def oracle_errors(obs, I, d, vsel, pix, samples):
    """Relative L2 error (Sec. 5.2) of each mode's sampled GPU outputs against the FP64 oracle
    evaluated at the same visibilities and pixels (part of the CPU-baseline leg); the image's
    error from the stratified pixel sample `pix` (indices, edge count, edge share)."""
    from oracle import direct
    direct.build()
    psel, nb, share = pix
    t0 = time.perf_counter()
    rv = direct.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y, vis_index=vsel)
    ri = direct.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x,
                     obs.pixsize_y, pixel_index=psel)
    t = time.perf_counter() - t0
    errs = {m: {"degrid": direct.rel_l2(v, rv), "grid": stratified_rel_l2(g, ri, nb, share)}
            for m, (v, g) in samples.items()}
    return errs, (f"{len(vsel)} sampled visibilities; {len(psel)} pixels stratified ({nb} within "
                  f"{EDGE_BAND} of the image edge, {share:.1%} of the image, {len(psel) - nb} "
                  f"inside, weighted by area) against the FP64 direct-sum oracle "
                  f"({t:.1f} s on the host)")


def run_config_1e8(args, wg, dev, hbm_gbs):
    """The 1e8-visibility workload (8192^2 at 4 arcsec, 128 antennas x 193 times x 64 channels
    truncated to 1e8 visibilities) at eps = 1e-5 FP32 and eps = 1e-12 FP64: plan creation time,
    one warm-up and `steps` timed calls per direction with per-stage CUDA-event times, the
    per-stage fractions of the HBM roofline by algorithmic bytes, and sampled GPU outputs for
    the error against the oracle."""
    import torch
    from paper_2010_10122_gb300 import synthetic as S
    modes8 = tuple(m for m in (("f32", 1e-5), ("f64", 1e-12)) if m[0] in args.modes_1e8.split(","))
    t0 = time.perf_counter()
    obs = S.wide_8k()
    I = S.point_source_image(obs.npix_x, obs.npix_y, seed=0)
    d = S.complex_normal((obs.nrows, obs.nchan), seed=1)
    gen_s = time.perf_counter() - t0
    vsel, pix = error_sample(obs, 128, seed=2)
    out = {"workload": "wide_8k", "nvis": obs.nvis, "npix": [obs.npix_x, obs.npix_y],
           "pixsize_arcsec": obs.pixsize_x / S.ARCSEC, "uv_scale": obs.uv_scale,
           "steps": args.steps_1e8, "warmup": 1, "input_generation_s": round(gen_s, 1),
           "modes": {}}
    samples = {}
    for prec, eps in modes8:
        rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
        plans, plan_ms = make_plans(wg, obs, ((prec, eps),), dev)
        p = plans[prec]
        din = torch.from_numpy(I).to(dev, rdt)
        vin = torch.from_numpy(d).to(dev, cdt)
        vout = torch.empty((obs.nrows, obs.nchan), dtype=cdt, device=dev)
        gout = torch.empty((obs.npix_x, obs.npix_y), dtype=rdt, device=dev)
        p.degrid(din, out=vout)
        p.grid(vin, out=gout)
        torch.cuda.synchronize()
        sts = {"degrid": [], "grid": []}
        for _ in range(args.steps_1e8):
            sts["degrid"].append(p.degrid(din, out=vout, stats=True)[1])
            sts["grid"].append(p.grid(vin, out=gout, stats=True)[1])
        torch.cuda.synchronize()
        info = p.info
        m = {"eps": eps, "alpha": info["alpha"], "sigma": info["sigma"],
             "uv_grid": [info["nu"], info["nv"]], "nw": info["nw"], "batch": info["batch"],
             "fft": FFT_NAMES[info["fft_impl"]], "err_model": info["err_model"],
             "plan_ms": round(plan_ms[prec], 1),
             "index_bytes_per_vis": info["index_bytes"] / max(1, obs.nvis)}
        for direction in ("degrid", "grid"):
            med = median_stats(sts[direction])
            m[direction] = {"vis_per_s": obs.nvis / (med["ms_total"] * 1e-3),
                            **{k: round(v, 3) for k, v in med.items()},
                            "hbm_roofline": stage_fractions(med, info, obs, prec, direction, hbm_gbs)}
        out["modes"][f"{prec}_eps{eps:g}"] = m
        samples[f"{prec}_eps{eps:g}"] = gpu_samples(vout, gout, vsel, pix[0])
        p.close()
        # the same calls on a compact index (4 bytes per visibility and the uvw rows resident,
        # the records recomputed per call)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pc = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                     eps, prec, device=dev, compact_index=True)
        cplan_ms = (time.perf_counter() - t0) * 1e3
        pc.degrid(din, out=vout)
        pc.grid(vin, out=gout)
        sd = pc.degrid(din, out=vout, stats=True)[1]
        sg = pc.grid(vin, out=gout, stats=True)[1]
        m["compact_index"] = {"plan_ms": round(cplan_ms, 1),
                              "index_bytes_per_vis": pc.info["index_bytes"] / max(1, obs.nvis),
                              "degrid_ms": round(sd["ms_total"], 3), "grid_ms": round(sg["ms_total"], 3),
                              "records_ms_per_call": round(sd["ms_prep"], 3)}
        pc.close()
        del din, vin, vout, gout
        torch.cuda.empty_cache()
    tm = {k: mm["degrid"]["ms_total"] + mm["grid"]["ms_total"] for k, mm in out["modes"].items()}
    if "f64_eps1e-12" in tm and "f32_eps1e-05" in tm:
        out["fp32_vs_fp64_speedup"] = tm["f64_eps1e-12"] / tm["f32_eps1e-05"]
    return out, (obs, I, d, vsel, pix, samples)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.serve:
        return run_serve(args)
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2010_10122_gb300 import _build
    if rank == 0 or ws == 1:
        _build.build()
    if ws > 1:
        dist.barrier()
    import paper_2010_10122_gb300 as wg

    global MODES
    MODES = tuple(m for m in MODES if m[0] in args.modes.split(","))
    obs, I, d = make_inputs(args.workload)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    plans, plan_ms = make_plans(wg, obs, MODES, dev, args.grid_variant, args.fft_impl)
    dins, vins, vouts, gouts = {}, {}, {}, {}
    for prec, eps in MODES:
        rdt, cdt = (torch.float32, torch.complex64) if prec == "f32" else (torch.float64, torch.complex128)
        dins[prec] = torch.from_numpy(I).to(dev, rdt)
        vins[prec] = torch.from_numpy(d).to(dev, cdt)
        vouts[prec] = torch.empty((obs.nrows, obs.nchan), dtype=cdt, device=dev)
        gouts[prec] = torch.empty((obs.npix_x, obs.npix_y), dtype=rdt, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    per_call = {}

    only = tuple(args.only.split(":")) if args.only else None

    def step(with_stats=False):
        for prec, _ in MODES:
            p = plans[prec]
            if only is None or only == (prec, "degrid"):
                r1 = p.degrid(dins[prec], out=vouts[prec], stats=with_stats)
                if with_stats:
                    per_call.setdefault((prec, "degrid"), []).append(r1[1])
            if only is None or only == (prec, "grid"):
                r2 = p.grid(vins[prec], out=gouts[prec], stats=with_stats)
                if with_stats:
                    per_call.setdefault((prec, "grid"), []).append(r2[1])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: per-step events, L2 flush between steps -----------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    clk = clocks.stop()
    from paper_2010_10122_gb300 import replicas
    total_ms = replicas.max_over_ranks(sum(step_ms), device=dev)
    ms_per_step = total_ms / args.steps
    ncalls = 2 * len(MODES)
    value = ws * ncalls * obs.nvis / (ms_per_step * 1e-3)

    # ---- per-call / per-stage breakdown (events inside the library, stage by stage) --------
    for _ in range(max(2, args.steps // 2)):
        flush.fill_(1)
        step(with_stats=True)
    torch.cuda.synchronize()
    if only is not None:
        st = per_call[only]
        if rank == 0:
            print(json.dumps({"only": args.only, "workload": args.workload,
                              "ms_per_call": ms_per_step, "stats": st[-1],
                              "plan": plans[only[0]].info}), flush=True)
        for p in plans.values():
            p.close()
        return 0

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp32_meas = wg.fma_peak("f32")     # flop/s, an FMA = 2 (measured now, on this GPU)
    fp64_meas = wg.fma_peak("f64")

    modes = {}
    launches = 0
    step_bytes = 0
    for prec, eps in MODES:
        info = plans[prec].info
        m = {"eps": eps, "alpha": info["alpha"], "sigma": info["sigma"],
             "uv_grid": [info["nu"], info["nv"]], "nw": info["nw"], "batch": info["batch"],
             "fft": FFT_NAMES[info["fft_impl"]], "err_model": info["err_model"],
             "plan_ms": round(plan_ms[prec], 2),
             "index_bytes_per_vis": info["index_bytes"] / max(1, obs.nvis)}
        for direction in ("degrid", "grid"):
            med = median_stats(per_call[(prec, direction)])
            hr = stage_fractions(med, info, obs, prec, direction, hbm_peak)
            step_bytes += hr["call"]["bytes"]
            m[direction] = {"vis_per_s": obs.nvis / (med["ms_total"] * 1e-3),
                            **{k: round(v, 4) for k, v in med.items()}, "hbm_roofline": hr}
            launches += per_call[(prec, direction)][-1]["n_kernels"]
        modes[f"{prec}_eps{eps:g}"] = m
    tm = {k: m["degrid"]["ms_total"] + m["grid"]["ms_total"] for k, m in modes.items()}
    speedup = (tm["f64_eps1e-12"] / tm["f32_eps1e-05"]
               if "f64_eps1e-12" in tm and "f32_eps1e-05" in tm else None)

    # ---- roofline of the dominant library kernel ----------------------------------------------
    stage_ms = {}
    for prec, _ in MODES:
        k = f"{prec}_eps{dict(MODES)[prec]:g}"
        for direction in ("degrid", "grid"):
            s = modes[k][direction]
            stage_ms[(prec, direction, "gridding")] = s["ms_grid"]
            stage_ms[(prec, direction, "screen" if direction == "degrid" else "accumulate")] = (
                s["ms_screen"] if direction == "degrid" else s["ms_accum"])
            if plans[prec].info["fft_impl"] == 2:   # the library's own FFT kernel
                stage_ms[(prec, direction, "fft")] = s["ms_fft"]
    dom = max(stage_ms, key=stage_ms.get)
    prec_d, dir_d, stage_d = dom
    info_d = plans[prec_d].info
    hbm_d = modes[f"{prec_d}_eps{dict(MODES)[prec_d]:g}"][dir_d]["hbm_roofline"][stage_d]
    hbm_8d = {"bytes": hbm_d["bytes"], "achieved_gbs": hbm_d["bytes"] / (stage_ms[dom] * 1e-3) / 1e9,
              "peak_gbs": hbm_peak, "frac": hbm_d["frac"],
              "accounting": "w-plane cells x bytes per cell x passes (screen 1, FFT 2, degrid 1, "
                            "grid 2, accumulate 1) + visibility data"}
    roof = None
    if stage_d == "fft":
        # double-float plane FFT: FP32-ALU (issue) bound; work = its FP32 arithmetic
        # instructions; one pass over the ny image columns (length nu), one over all nu rows
        nu, nv, nw = info_d["nu"], info_d["nv"], info_d["nw"]
        ops = nw * (obs.npix_y * df64_line_ops(nu) + nu * df64_line_ops(nv))
        peak = 152 * 128 * 2.07e9   # SMs x FP32 lanes x max SM clock, one instruction per lane
        ach = ops / (stage_ms[dom] * 1e-3)
        abytes = nw * df64_fft_bytes(obs.npix_x, obs.npix_y, nu, nv, dir_d)
        kname = "k_fft_lines_cluster" if df64_line_split(nu) > 1 else "k_fft_lines"
        roof = {"bound": "alu", "kernel": f"{kname} (double-float plane FFT, row + column pass)",
                "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": DF64_DRAM_PER_ALGORITHMIC_BYTE * abytes,
                "algorithmic_bytes": abytes,
                "peak_source": "FP32 arithmetic instructions/s: 152 SMs x 128 lanes x 2.07 GHz "
                               "(an FMA counts once)",
                "peak_measured": fp32_meas / 2 / 1e12, "frac_measured": ach / (fp32_meas / 2),
                "peak_measured_source": "wg_fma_peak(WG_F32) on this GPU now: FMA instructions/s",
                "stage": f"{prec_d} {dir_d}", "hbm_8d": hbm_8d}
    elif stage_d == "gridding" and prec_d == "f64":
        flops = algorithmic_flops_per_vis(info_d["alpha"]) * plans[prec_d].info["nvis"]
        peak = 1.25e12   # FP64 FMA pipe: nominal GB300 rate (152 SMs x 2 FMA/clk x 2 x 2.07 GHz)
        ach = flops / (stage_ms[dom] * 1e-3)
        roof = {"bound": "alu", "kernel": f"k_{dir_d}<double,16>", "achieved": ach / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_measured": fp64_meas / 1e12, "frac_measured": ach / fp64_meas,
                "stage": f"{prec_d} {dir_d}", "hbm_8d": hbm_8d}
    else:
        roof = {"bound": "hbm", "kernel": f"{stage_d} ({prec_d}, {dir_d})",
                "achieved": hbm_8d["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_d["frac"], "traffic": None, "stage": f"{prec_d} {dir_d}",
                "hbm_8d": hbm_8d}
    step_roof = {"bytes": step_bytes, "achieved_gbs": step_bytes / (ms_per_step * 1e-3) / 1e9,
                 "peak_gbs": hbm_peak, "frac": step_bytes / (hbm_peak * 1e9) / (ms_per_step * 1e-3)}

    # sampled outputs of the headline workload for the error against the oracle (CPU leg), and
    # the whole outputs for the adjointness test of Sec. 5.1
    vsel2, pix2 = error_sample(obs, 256, seed=0)
    samples2 = {f"{prec}_eps{eps:g}": gpu_samples(vouts[prec], gouts[prec], vsel2, pix2[0])
                for prec, eps in MODES}
    adj = {}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import direct
        for prec, eps in MODES:
            adj[f"{prec}_eps{eps:g}"] = direct.adjointness_error(
                I, vouts[prec].cpu().numpy(), d, gouts[prec].cpu().numpy())

    # ---- end to end: host buffers, copies inside the timed region ------------------------------
    e2e = e2e_one = None
    if not args.no_e2e:
        h_in = {}
        for prec, _ in MODES:
            h_in[prec] = (dins[prec].cpu().pin_memory(), vins[prec].cpu().pin_memory())
        h_out = {prec: (torch.empty(vouts[prec].shape, dtype=vouts[prec].dtype).pin_memory(),
                        torch.empty(gouts[prec].shape, dtype=gouts[prec].dtype).pin_memory())
                 for prec, _ in MODES}
        bi = sum(a.numel() * a.element_size() + b_.numel() * b_.element_size() for a, b_ in h_in.values())
        bo = sum(a.numel() * a.element_size() + b_.numel() * b_.element_size() for a, b_ in h_out.values())

        def e2e_step():
            for prec, _ in MODES:
                di = h_in[prec][0].to(dev, non_blocking=True)
                vi = h_in[prec][1].to(dev, non_blocking=True)
                vo = plans[prec].degrid(di)
                go = plans[prec].grid(vi)
                h_out[prec][0].copy_(vo, non_blocking=True)
                h_out[prec][1].copy_(go, non_blocking=True)
        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            e0.record(stream)
            e2e_step()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        e2e = {"value": ws * ncalls * obs.nvis / (tot / args.steps * 1e-3), "unit": "vis/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}

        # one-shot calls (the paper's dirty2ms / ms2dirty, App. B): plan creation -- index
        # build, tables, FFT set-up -- inside every call, from host buffers
        uvw_h = torch.from_numpy(obs.uvw).pin_memory()
        freq_h = torch.from_numpy(obs.freq)

        def oneshot_step():
            for prec, eps in MODES:
                vo = wg.dirty2ms(uvw_h, freq_h, h_in[prec][0], pixsize_x=obs.pixsize_x,
                                 pixsize_y=obs.pixsize_y, epsilon=eps, device=dev)
                go = wg.ms2dirty(uvw_h, freq_h, h_in[prec][1], npix_x=obs.npix_x,
                                 npix_y=obs.npix_y, pixsize_x=obs.pixsize_x,
                                 pixsize_y=obs.pixsize_y, epsilon=eps, device=dev)
                h_out[prec][0].copy_(vo, non_blocking=True)
                h_out[prec][1].copy_(go, non_blocking=True)
        oneshot_step()
        torch.cuda.synchronize()
        n1 = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(n1):
            oneshot_step()
        torch.cuda.synchronize()
        t1 = (time.perf_counter() - t0) / n1
        e2e_one = {"value": ncalls * obs.nvis / t1, "unit": "vis/s", "steps": n1,
                   "timing": "host wall clock (plan creation synchronises the stream)",
                   "h2d_bytes_per_step": bi + len(MODES) * 2 * uvw_h.numel() * 8,
                   "d2h_bytes_per_step": bo}

    # ---- the 1e8-visibility workload ---------------------------------------------------------
    cfg8 = ctx8 = None
    if args.modes_1e8 not in ("", "none") and ws == 1 and args.workload != "wide_8k":
        cfg8, ctx8 = run_config_1e8(args, wg, dev, hbm_peak)

    # ---- serving: a bounded sub-mix of the serving workload ----------------------------------
    serve = None
    if ws == 1 and not args.no_serve:
        for p in plans.values():
            p.close()
        plans = {}
        torch.cuda.empty_cache()
        serve = serve_benchmark(60, 6, [512, 1024, 2048], (1e5, 2e6), 8, 150.0, [0.5, 0.9, 2.0],
                                serial_sample=60)
        serve["sub_mix"] = ("60 requests over 6 observations (512^2 - 2048^2, 1e5 - 2e6 "
                            "visibilities); the full mix runs with bench.py --serve")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        vps, cores, sample, _, vps1 = oracle_rate(obs, I, d, args.oracle_seconds)
        cpu = {"value": vps, "unit": "vis/s", "cores": cores, "kind": "oracle", "sample": sample,
               "value_1core": vps1}
        errs, how = oracle_errors(obs, I, d, vsel2, pix2, samples2)
        for k, e in errs.items():
            modes[k]["rel_l2_err"] = {**e, "sample": how}
        for k, e in adj.items():
            modes[k]["eps_adj"] = e
        if cfg8 is not None:
            o8, I8, d8, vs8, ps8, smp8 = ctx8
            errs8, how8 = oracle_errors(o8, I8, d8, vs8, ps8, smp8)
            for k, e in errs8.items():
                cfg8["modes"][k]["rel_l2_err"] = {**e, "sample": how8}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "vis/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": args.workload, "nvis": obs.nvis,
                           "npix": [obs.npix_x, obs.npix_y], "pixsize_arcsec": obs.pixsize_x / S_ARCSEC(),
                           "uv_scale": obs.uv_scale,
                           "step": "degrid+grid at " + " and ".join(
                               f"eps={e:g} {p}" for p, e in MODES) + ", resident plans",
                           "parallelism": f"replicas{ws}" if ws > 1 else "single",
                           "l2": "flushed between steps (256 MiB write)"},
                "modes": modes, "fp32_vs_fp64_speedup": speedup,
                "roofline": roof, "step_hbm_roofline": step_roof,
                "peaks": {"hbm_gbs": hbm_peak, "hbm_source": "MEASURED_PEAKS.json",
                          "fp32_fma_tflops_measured": fp32_meas / 1e12,
                          "fp64_fma_tflops_measured": fp64_meas / 1e12},
                "cpu_baseline": cpu, "e2e": e2e, "e2e_oneshot": e2e_one,
                "config_1e8": cfg8, "serve": serve,
                "gpu_launches": launches * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    for p in plans.values():
        p.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def S_ARCSEC():
    from paper_2010_10122_gb300 import synthetic as S
    return S.ARCSEC


if __name__ == "__main__":
    sys.exit(main())
