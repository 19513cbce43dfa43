#!/usr/bin/env python3
"""Benchmark of the slice projection operator on the microscopy-shaped fit step.

Workload (one step = the whole hot path): 500k Gaussians in a 1024 x 1024 x 256
light-sheet-shaped volume (z-scale 3x the xy-scale, log-normal intensities),
sigma_z = 3; each step renders a random batch of 16 of the 256 slices
(K-pre, pair binning, radix sort, K-range, K-fwd), takes the MSE against the
same slices of a seeded 256-slice target stack (K-loss), runs the backward
(K-bwd on the forward's bins, K-bwd-pre) to gradients of all 11 parameters per
Gaussian, and applies the Adam update with the paper's learning rates.
Inputs are synthetic (seeded); the target stack is rendered once, untimed,
from a second seeded set of the same distribution.

Metric: Gaussian-pixel evaluations per second, forward + backward, counting
ALGORITHMIC evaluations (pixels inside each pair's culling ellipse,
d^T Sigma_2d^-1 d <= 2 ln(1/eps), on slices with opacity_r >= eps), twice per
step (forward and backward).  Also reported: slices/s, per-phase times, the
roofline of the dominant kernel, an end-to-end figure through host buffers,
and the FP64 oracle timed on host cores on a bounded sample.  At N = 1 the
line also carries the batched form ("batched": 64 uneven sets in one autotuned
graph launch against 64 plain render + backward calls) and the served form
("serving": a seeded Poisson request stream at two offered rates, served with
continuous batching and replayed through sequential plain calls), each with
its own clocks, after the fit step's timed region.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--fit-only]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Gaussian-pixel evals/s"
UNIT = "evals/s"
WORKLOAD = {"workload": "microscopy fit step: 500k Gaussians, 1024x1024x256 volume, sigma_z=3, "
                        "random batch of 16 slices per step, fwd + MSE + bwd + Adam update",
            "n_gaussians": 500_000, "slice_hw": [1024, 1024], "n_planes": 256, "slices_per_step": 16,
            "sigma_z": 3.0, "eps": 1e-6, "l2": "flushed between steps (256 MiB write)"}
N, H, W, DEPTH, S, SIGMA = 500_000, 1024, 1024, 256, 16, 3.0
# A quarter-size case with the same Gaussian density and list lengths (125k
# Gaussians, 512 x 512 x 256), used for profiler captures.
SMALL = dict(N=125_000, H=512, W=512, extent=(512, 512, 256))


def use_small_case():
    global N, H, W, WORKLOAD
    N, H, W = SMALL["N"], SMALL["H"], SMALL["W"]
    WORKLOAD = dict(WORKLOAD, workload="microscopy fit step, quarter size for profiling: 125k Gaussians, "
                                       "512x512x256 volume, sigma_z=3, 16 slices per step",
                    n_gaussians=N, slice_hw=[H, W])


def microscopy_set(synth, seed):
    if N == SMALL["N"]:
        return synth.microscopy(seed=seed, n=N, extent=SMALL["extent"])
    return synth.microscopy(seed=seed)

# Lane instructions of the FP32/INT pipes per ALGORITHMIC evaluation, counted from
# the method's arithmetic with the project-written exp2 (range reduction 3 FADD,
# Horner 6 FFMA for the forward's degree-6 polynomial and 4 for the backward's
# degree-4 one, exponent insert 2 INT): forward = offset 1 + quadratic form 2 +
# clamp 1 + exp2 11 + accumulate 1; backward = offset 1 + quadratic form 2 +
# clamp 1 + exp2 9 + 5 moment updates (g = G E, 2 sums, 1 product, 1 FMA).
OPS_PER_EVAL = {"fwd": 16, "bwd": 18}
# The row-factored form (GP_EXP_POLY_ROW) does its exponentials per row of 8
# pixels: per row 2 exp2 (22) + 2 clamps + the larger end's exponent 1 + powers
# r^2..r^7 6 + row coefficients 4, then forward 7 scalings by L + 8 accumulates
# (50 per row), backward 7 products r^j 2^(C q^2) + 8 products with dL/dI +
# 24 moment updates + 3 pair sums + 3 products with L + 6 row-moment updates
# (84 per row), i.e. 50/8 and 84/8 lane instructions per evaluation.
OPS_PER_EVAL_ROW = {"fwd": 6.25, "bwd": 10.5}
EXP_MODES = {"poly": 0, "hw": 1, "row": 3}
# What each --exp choice computes, for the JSON line's config.
EXP_NOTE = {"poly": "project-written exp2, no ex2.approx: degree-6 polynomial (about 2 ulp) in the forward, "
                    "degree-4 (3.6e-6 relative) for the exponentials the backward recomputes",
            "hw": "the SFU ex2.approx instruction in both passes",
            "row": "row-factored exponentials (two exp2 per row of 8 pixels), per-pixel exp2 for narrow Gaussians"}
RASTER_FORMS = {"auto": 0, "block": 1, "rows": 2}


def raster_kernel(pass_, raster, exp, vox=False):
    """Name of the kernel a rasteriser pass runs on this configuration."""
    if exp == "row" or raster == "block":
        return f"k_raster_{pass_}_blk"
    if raster == "rows" or pass_ == "fwd" or vox:
        return f"k_raster_{pass_}_rows"
    return f"k_raster_{pass_}_blk"


def pass_roofline(evals, evaluated, ops, launch_s, peak, kernel):
    """Roofline figures of one rasteriser pass: algorithmic lane instructions per
    second against the measured FP32 peak, and the evaluated pixels per
    algorithmic evaluation."""
    achieved = evals * ops / launch_s / 1e12
    return {"kernel": kernel, "achieved": achieved, "peak": peak / 1e12, "frac": achieved / (peak / 1e12),
            "ops_per_eval": ops, "launch_ms": launch_s * 1e3,
            "evaluated_per_algorithmic": (evaluated / evals) if evals else None}


def fp32_probe_peak(ctx, stream, reps=5, iters=20000, mode=0):
    """Lane instructions per second of the throughput probe (mode 0: FP32 FMA,
    3: SFU ex2): best of reps launches."""
    import torch
    ctx.fma_probe(2000, mode=mode)
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, lanes = ctx.fma_probe(iters, mode=mode)
        e1.record(stream)
        e1.synchronize()
        best = max(best, lanes / (e0.elapsed_time(e1) * 1e-3))
    return best


def sfu_roofline(sfu_peak, evals_per_launch, launch_s):
    """The SFU side of the GP_EXP_HW variant's roofline: one ex2.approx per
    algorithmic evaluation against the measured ex2 rate (probe mode 3)."""
    if not sfu_peak:
        return {}
    achieved = evals_per_launch / launch_s / 1e12
    return {"sfu": {"achieved": achieved, "peak": sfu_peak / 1e12, "unit": "T ex2/s",
                    "frac": achieved * 1e12 / sfu_peak, "peak_kind": "measured ex2.approx probe, best of 5"}}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms; only the
    samples whose timestamps fall inside the timed window are summarised."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.p = None
        self.window = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)  # let the first samples arrive before the timed region

    def mark(self, t0, t1):
        """Wall-clock (time.time()) bounds of the timed region."""
        self.window = (t0, t1)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.15)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        return summarise_clocks(out, self.window)


def _num(x):
    try:
        return float(x)
    except ValueError:
        return None


def summarise_clocks(text, window=None):
    """Median SM clock, max clock, active slowdown reasons and sample count of
    nvidia-smi CSV rows; rows outside the (t0, t1) window are dropped unless
    none fall inside it (then all are kept and 'in_window' says so)."""
    import datetime
    rows = [[c.strip() for c in r.split(",")] for r in text.strip().splitlines() if r.count(",") >= 9]
    if not rows:
        return None
    inside = rows
    if window is not None:
        def ts(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None
        inside = [r for r in rows if ts(r) is not None and window[0] - 0.05 <= ts(r) <= window[1] + 0.05]
    in_window = bool(inside) and window is not None
    use = inside if inside else rows
    sm = [v for v in (_num(r[2]) for r in use) if v is not None]
    mx = [v for v in (_num(r[3]) for r in rows) if v is not None]
    pw = [v for v in (_num(r[4]) for r in use) if v is not None]
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({nm for r in use for nm, v in zip(names, r[6:10]) if v == "Active"})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(use), "in_window": in_window,
            "power_w_max": max(pw) if pw else None}


# Per-launch DRAM traffic of the rasterisers on this workload, from an ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), kept as data in
# profiles/raster_traffic.json with a hash of the kernels' sources, so that a
# changed kernel reports null.  A capture beyond gpu__time_duration is taken on
# one kernel and one or two launches of the quarter-size case (--case small,
# -k regex:k_raster_bwd_blk -s <warm-up launches> -c 2, --clock-control none)
# and scaled to a full launch by the binned pairs ("scale").
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "raster_traffic.json")
KERNEL_SOURCES = ("paper_2603_20611_b300/csrc/raster.cu", "paper_2603_20611_b300/csrc/gp_common.cuh",
                  "paper_2603_20611_b300/csrc/slice.cuh", "paper_2603_20611_b300/csrc/raster_rows.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """(bytes per launch, note) for `kernel` (e.g. 'k_raster_fwd_rows', 'k_raster_bwd_blk')."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no capture recorded"
    with open(TRAFFIC_FILE) as f:
        rec = json.load(f).get("kernels", {}).get(kernel)
    if rec is None:
        return None, "kernel not in the capture"
    if rec["source_hash"] != kernel_source_hash():
        return None, "stale: the kernel sources changed since the capture"
    return (rec["dram_read_bytes"] + rec["dram_write_bytes"]) * rec.get("scale", 1.0), \
        "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch: " + rec["note"]


def oblique_view(Wd, Hd, Dd, seed=8080):
    """Seeded rotation R and translation t putting the volume centre at the image
    centre on plane z_c = 0 (camera x_c = R x + t)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    c = np.array([Wd / 2.0, Hd / 2.0, Dd / 2.0])
    t = np.array([Wd / 2.0, Hd / 2.0, 0.0]) - R @ c
    return R.astype(np.float32), t.astype(np.float32)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def make_workload(B, synth, torch, dev, ctx):
    g = microscopy_set(synth, 1002)
    gs = B.GaussianSet.from_numpy(g, dev)
    tgt = B.GaussianSet.from_numpy(microscopy_set(synth, 2002), dev)
    target = torch.empty(DEPTH, H, W, device=dev)
    for s0 in range(0, DEPTH, 32):
        B.gp_render_slices(ctx, tgt, synth.slice_positions(range(s0, s0 + 32)), H, W, SIGMA,
                           out=target[s0:s0 + 32])
    torch.cuda.synchronize()
    del tgt
    return g, gs, target


def step_batches(synth, rank, count):
    from paper_2603_20611_b300.replicas import batch_seed
    return [synth.slice_batch(batch_seed(rank, k), DEPTH, DEPTH, S) for k in range(count)]


# ------------------------------------------------------------------ oracle arm

def oracle_step_seconds(oracle, synth, g, idx, n_px, n_gauss, seed):
    """Seconds the FP64 oracle would take for one full step, extrapolated from a
    bounded sample: the forward at n_px sampled pixels of the step's slices (its
    per-slice projection of every Gaussian timed separately with one pixel per
    slice), and the backward of n_gauss sampled Gaussians against a seeded
    dL/dI (its brute force costs the same for every Gaussian).  Returns
    (step seconds, sample seconds)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = synth.slice_positions(idx)
    G = synth.random_field(seed + 1, (S, H, W))
    one = np.arange(S, dtype=np.int32)
    ps = rng.integers(0, S, n_px).astype(np.int32)
    px = rng.integers(0, W, n_px) + 0.5
    py = rng.integers(0, H, n_px) + 0.5
    pick = np.sort(rng.choice(g.n, n_gauss, replace=False))
    t0 = time.perf_counter()
    oracle.render_points(g.mu, g.scale, g.quat, g.alpha, z, SIGMA, one, np.full(S, 0.5), np.full(S, 0.5))
    t1 = time.perf_counter()
    oracle.render_points(g.mu, g.scale, g.quat, g.alpha, z, SIGMA, ps, px, py)
    t2 = time.perf_counter()
    oracle.render_backward(g.mu[pick], g.scale[pick], g.quat[pick], g.alpha[pick], z, H, W, SIGMA, G)
    t3 = time.perf_counter()
    # the step's parameter update (FP64 Adam over the whole set, timed in full)
    from oracle import optim
    st = optim.FitState(g.mu, g.scale, g.quat, g.alpha)
    gz = [np.zeros_like(x, dtype=np.float64) for x in (g.mu, g.scale, g.quat, g.alpha)]
    t4 = time.perf_counter()
    st.step(gz, 1)
    t5 = time.perf_counter()
    t_fixed = t1 - t0
    per_px = max(t2 - t1 - t_fixed, 0.0) / max(n_px - S, 1)
    step = t_fixed + per_px * S * H * W + (t3 - t2) / n_gauss * g.n + (t5 - t4)
    return step, (t3 - t0) + (t5 - t4)


def oracle_evals(oracle, synth, g, idx):
    """Forward algorithmic evaluations of one step, counted by the oracle."""
    return oracle.count_evals(g.mu, g.scale, g.quat, g.alpha, synth.slice_positions(idx), H, W, SIGMA,
                              eps=WORKLOAD["eps"])


def oracle_baseline(oracle, synth, g, idx, n_px, n_gauss, seed, evals_fwd):
    step_s, sample_s = oracle_step_seconds(oracle, synth, g, idx, n_px, n_gauss, seed)
    return {"value": 2.0 * evals_fwd / step_s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one step's forward at {n_px} sampled pixels (+1 pixel per slice to separate the "
                      f"per-slice projection cost), backward of {n_gauss} sampled Gaussians and the Adam update of "
                      f"the whole set, FP64, "
                      f"{sample_s:.1f}s of CPU work, extrapolated to the full step "
                      f"({2.0 * evals_fwd:.3e} algorithmic evaluations)"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle, timed on host cores, on bounded samples."""
    if rank != 0:
        return 0
    import oracle
    from paper_2603_20611_b300 import synth
    g = microscopy_set(synth, 1002)
    batches = step_batches(synth, 0, args.warmup + args.steps)
    step_s, evals, sample_s = [], [], 0.0
    n_gauss = args.ref_gauss or 2 * oracle.num_threads()
    for k, idx in enumerate(batches):
        ev = oracle_evals(oracle, synth, g, idx)
        st, ss = oracle_step_seconds(oracle, synth, g, idx, args.ref_px, n_gauss, 5000 + k)
        if k >= args.warmup:
            step_s.append(st)
            evals.append(2.0 * ev)
            sample_s += ss
    value = sum(evals) / sum(step_s)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(step_s)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": WORKLOAD, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"per step: forward at {args.ref_px} sampled pixels, backward of "
                                       f"{n_gauss} sampled Gaussians (FP64 brute force) and the Adam update "
                                       f"of the whole set, extrapolated to the full step; {sample_s:.1f}s of "
                                       f"CPU work in the timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ native arm

def run_native(args, rank, world):
    import torch
    from paper_2603_20611_b300 import binding as B
    from paper_2603_20611_b300 import synth
    from paper_2603_20611_b300.replicas import reduce_timing
    dev_index = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev_index)
    dev = f"cuda:{dev_index}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ctx = B.Context(dev_index, exp_mode=EXP_MODES[args.exp],
                    deterministic=args.det, tile=args.tile, fwd_px=args.fwd_px, bwd_px=args.bwd_px,
                    reuse_bins=not args.rebin, raster=RASTER_FORMS[args.raster])
    stream = torch.cuda.current_stream()
    t_setup = time.perf_counter()
    g, gs, target = make_workload(B, synth, torch, dev, ctx)
    batches = step_batches(synth, rank, args.warmup + args.steps)
    zs = [synth.slice_positions(b) for b in batches]
    view = None
    if args.view == "oblique":
        # a seeded rotation through the volume's centre; plane s sits at
        # (s + 1/2) - DEPTH/2 along the rotated normal
        view = oblique_view(W, H, DEPTH)
        zs = [z - DEPTH / 2.0 for z in zs]
    # a second context counts the algorithmic evaluations of every step on the
    # parameters that step renders (the Adam update moves them between steps)
    cctx = B.Context(dev_index, deterministic=args.det, tile=args.tile, exp_mode=EXP_MODES[args.exp],
                     raster=RASTER_FORMS[args.raster])
    evals0 = [B.gp_count_evals(cctx, gs, z, H, W, SIGMA, view=view) for z in zs]  # initial parameters (e2e loop)
    # pixels the rasterisers evaluate on the first timed step (initial parameters)
    evaluated = B.gp_count_evaluated(cctx, gs, zs[args.warmup], H, W, SIGMA, view=view)
    evaluated_ratio = [e / max(evals0[args.warmup], 1) for e in evaluated]
    log(f"setup {time.perf_counter() - t_setup:.1f}s; evals/step (fwd) ~{np.mean(evals0):.3e}")
    host_params = [t.cpu().pin_memory() for t in (gs.mu, gs.scale, gs.quat, gs.alpha)]
    opt = B.Adam(ctx, gs, total_steps=30000, mu_extent=float(max(H, W)))
    I = torch.empty(S, H, W, device=dev)
    G = torch.empty(S, H, W, device=dev)
    loss = torch.zeros(1, device=dev)
    grads = (torch.empty(N, 3, device=dev), torch.empty(N, 3, device=dev), torch.empty(N, 4, device=dev),
             torch.empty(N, device=dev))
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MiB > 126 MB L2

    loss3 = torch.zeros(3, device=dev)

    def loss_grad(T, t_index):
        if args.loss == "l1dssim":
            B.gp_l1_dssim_grad(ctx, I, T, t_index=t_index, lam=0.2, dL_dI=G, loss=loss3)
        else:
            B.gp_mse_grad(ctx, I, T, t_index=t_index, dL_dI=G, loss=loss)

    def step(k):
        B.gp_render_slices(ctx, gs, zs[k], H, W, SIGMA, out=I, view=view)
        loss_grad(target, batches[k])
        B.gp_render_backward(ctx, gs, zs[k], H, W, SIGMA, G, grads=grads, view=view)
        opt.step(gs, grads)

    for k in range(args.warmup):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    # FP32-pipe peak at the clocks in force (burst, just before the timed region):
    # the best of five probe launches, so that one launch slowed by the host or a
    # clock transition does not lower the denominator
    fp32_peak = fp32_probe_peak(ctx, stream)
    sfu_peak = fp32_probe_peak(ctx, stream, mode=3) if args.exp == "hw" else None

    clocks = ClockSampler(dev_index)
    # Inside the timed steps only the two rasterisers' phases record events (the
    # roofline's launch times): every timed phase adds an event pair to the
    # step.  Each step's algorithmic evaluations are counted after the timed
    # region on a snapshot of the parameters that step renders (a stream-ordered
    # device copy before the step's first event), so the count's host
    # synchronisation does not leave the device idle at the start of the next step.
    pnames = ("mu", "scale", "quat", "alpha")
    snaps = [[torch.empty_like(getattr(gs, nm)) for nm in pnames] for _ in range(args.steps)]
    ctx.timing(True, phases=("fwd", "bwd"))
    ctx.timing_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = int(B.lib.gp_launch_count())
    clocks.start()
    evs = []
    wall0 = time.perf_counter()
    tw0 = time.time()
    for j, k in enumerate(range(args.warmup, args.warmup + args.steps)):
        for d, nm in zip(snaps[j], pnames):
            d.copy_(getattr(gs, nm))
        flush.zero_()  # after the snapshot, so the step starts with nothing of it in L2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(k)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.mark(tw0, time.time())
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = int(B.lib.gp_launch_count()) - launches0
    phases = ctx.timing_read()
    ctx.timing(False)
    ev_steps = [B.gp_count_evals(cctx, B.GaussianSet(*snaps[j], gs.scale_mod), zs[k], H, W, SIGMA, view=view)
                for j, k in enumerate(range(args.warmup, args.warmup + args.steps))]
    del snaps
    # the whole phase breakdown, reported beside the line: a separate pass of a
    # few steps with every phase timed
    n_ph = min(args.steps, 10)
    ctx.timing(True)
    ctx.timing_read()
    for k in range(args.warmup, args.warmup + n_ph):
        flush.zero_()
        step(k)
    torch.cuda.synchronize()
    phases_all = ctx.timing_read()
    ctx.timing(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(step_ms) * 1e-3
    my_evals = 2.0 * sum(ev_steps)
    t_total, tot_evals = reduce_timing(t_total, my_evals, device=dev if dist else None)
    value = tot_evals / t_total
    pairs, issued = ctx.last_counts()

    # roofline of the dominant kernel (the larger of the two rasterisers), and of both passes
    dom = "bwd" if phases["bwd"][0] >= phases["fwd"][0] else "fwd"
    ops_t = OPS_PER_EVAL_ROW if args.exp == "row" else OPS_PER_EVAL
    passes = {p: pass_roofline(float(np.mean(ev_steps)), float(np.mean(ev_steps)) * evaluated_ratio[i], ops_t[p],
                               phases[p][0] * 1e-3 / max(phases[p][2], 1), fp32_peak,
                               raster_kernel(p, args.raster, args.exp))
              for i, p in enumerate(("fwd", "bwd"))}
    ms_dom, _, calls_dom = phases[dom]
    avg_launch_s = ms_dom * 1e-3 / max(calls_dom, 1)
    ops_table = OPS_PER_EVAL_ROW if args.exp == "row" else OPS_PER_EVAL
    alg_ops_per_launch = float(np.mean(ev_steps)) * ops_table[dom]
    achieved = alg_ops_per_launch / avg_launch_s / 1e12
    peak = fp32_peak / 1e12
    nominal = 148 * 128 * 2.032e9 / 1e12
    default_cfg = (args.exp == "poly" and not args.det and args.tile == 16 and args.fwd_px == 0
                   and args.bwd_px == 0 and args.case == "microscopy" and args.raster == "auto")
    dom_kernel = raster_kernel(dom, args.raster, args.exp)
    traffic, traffic_note = recorded_traffic(dom_kernel) if default_cfg else \
        (None, "recorded for the default configuration only")

    # end to end through host buffers: every step uploads the parameters and the
    # batch's 16 target slices (pinned host -> device), runs the step (render,
    # loss, backward, Adam) and reads back the loss and the updated parameters
    # (device -> pinned host).  The copies run on their own streams against two
    # alternating device buffer sets, so step k+1's upload and step k-1's
    # readback overlap step k's kernels; the timed region runs from the first
    # upload to the last readback.
    host_stack = target.cpu().pin_memory()
    host_out = [[torch.empty(getattr(gs, nm).shape, pin_memory=True) for nm in pnames] for _ in range(2)]
    nloss = 3 if args.loss == "l1dssim" else 1
    host_loss = [torch.empty(nloss, pin_memory=True) for _ in range(2)]
    bufs = [(B.GaussianSet(*[torch.empty_like(getattr(gs, nm)) for nm in pnames], gs.scale_mod),
             torch.empty(S, H, W, device=dev), torch.zeros(nloss, device=dev)) for _ in range(2)]
    h2d = sum(t.numel() * 4 for t in host_params) + S * H * W * 4
    d2h = sum(t.numel() * 4 for t in host_out[0]) + host_loss[0].numel() * 4
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    in_done = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(args.warmup, args.warmup + args.steps):
        kb = k % 2
        gsb, tgt_dev, loss_dev = bufs[kb]
        if k - args.warmup >= 2:
            s_in.wait_event(out_done[kb])  # the readback two steps back reads this buffer
        with torch.cuda.stream(s_in):
            for d, h in zip([getattr(gsb, nm) for nm in pnames], host_params):
                d.copy_(h, non_blocking=True)
            for j, si in enumerate(batches[k]):
                tgt_dev[j].copy_(host_stack[int(si)], non_blocking=True)
            in_done[kb].record(s_in)
        stream.wait_event(in_done[kb])
        flush.zero_()
        B.gp_render_slices(ctx, gsb, zs[k], H, W, SIGMA, out=I, view=view)
        if args.loss == "l1dssim":
            B.gp_l1_dssim_grad(ctx, I, tgt_dev, lam=0.2, dL_dI=G, loss=loss_dev)
        else:
            loss_dev.zero_()
            B.gp_mse_grad(ctx, I, tgt_dev, dL_dI=G, loss=loss_dev)
        B.gp_render_backward(ctx, gsb, zs[k], H, W, SIGMA, G, grads=grads, view=view)
        opt.step(gsb, grads)
        used[kb].record(stream)
        s_out.wait_event(used[kb])
        with torch.cuda.stream(s_out):
            for h, d in zip(host_out[kb], [getattr(gsb, nm) for nm in pnames]):
                h.copy_(d, non_blocking=True)
            host_loss[kb].copy_(loss_dev, non_blocking=True)
            out_done[kb].record(s_out)
    e1.record(s_out)
    e1.synchronize()
    e2e_ms = [e0.elapsed_time(e1) / args.steps] * args.steps
    # every e2e step renders the initial parameters again (uploaded each step)
    e2e_value = world * 2.0 * sum(evals0[args.warmup:]) / (sum(e2e_ms) * 1e-3)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cpu = oracle_baseline(oracle, synth, g, batches[args.warmup], args.ref_px,
                              args.ref_gauss or 2 * oracle.num_threads(), 4242, ev_steps[0])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(WORKLOAD, exp=args.exp, exp_note=EXP_NOTE[args.exp], deterministic=bool(args.det),
                               tile=args.tile, loss=args.loss,
                               view=args.view,
                               backward_bins="re-binned" if args.rebin else "reused from the step's forward",
                               parallelism="replicas" if world > 1 else "single"),
                "slices_per_s": world * S * args.steps / t_total,
                "evals_fwd_per_step": float(np.mean(ev_steps)),
                "pairs_last_call": pairs, "tile_pixels_last_call": issued,
                "evaluated_per_algorithmic": {"fwd": evaluated_ratio[0], "bwd": evaluated_ratio[1]},
                "rasteriser": args.raster, "passes": passes,
                "phase_ms_per_step": {k: v[0] / n_ph for k, v in phases_all.items() if v[2]},
                "phase_timing": f"a separate pass of {n_ph} steps with every phase timed; the timed steps record "
                                "events around the two rasterisers only",
                "roofline": {"bound": "alu", "kernel": dom_kernel, "achieved": achieved, "peak": peak,
                             "unit": "Tinst/s (FP32+INT lane instructions)", "frac": achieved / peak,
                             "traffic": traffic, "traffic_note": traffic_note,
                             "peak_kind": "measured FMA probe, best of 5 bursts, same run",
                             "nominal_peak_2032mhz": nominal, "ops_per_eval": ops_table[dom],
                             **sfu_roofline(sfu_peak, float(np.mean(ev_steps)), avg_launch_s)},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": float(np.mean(e2e_ms)),
                        "overlap": "uploads and readbacks on two copy streams, two device buffer sets"},
                "gpu_launches": launches, "clocks": clk, "wall_s_timed": wall}
        if world == 1 and not args.fit_only:
            # the batched and served forms against their plain launches (after
            # the headline's timed region; their own CUDA-event and wall clocks)
            del target, host_stack, bufs
            torch.cuda.empty_cache()
            line["batched"] = batched_comparison(max(5, min(args.steps, 20)), 3)
            line["serving"] = serving_comparison([float(r) for r in args.fit_rates.split(",")],
                                                 args.serve_requests, args.serve_workers)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ batched workload

def batched_comparison(steps, warmup, n_sets=64):
    """64 uneven sets (1k-200k Gaussians, 128^2-1024^2 slices, 8-64 planes,
    sigma_z in [1, 6]) forward + backward against seeded upstream gradients:
    one autotuned graph launch per step against 64 plain render + backward
    calls, both timed with CUDA events on the launching stream."""
    import torch
    from paper_2603_20611_b300 import binding as B
    from paper_2603_20611_b300 import synth
    dev = f"cuda:{torch.cuda.current_device()}"
    ctx = B.Context(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    gen = torch.Generator(device=dev)
    gen.manual_seed(4004)
    t0 = time.perf_counter()
    items, evals = [], 0
    for bi in synth.batched(n_sets=n_sets):
        gs = B.GaussianSet.from_numpy(bi.gs, dev)
        S = len(bi.z)
        it = {"gs": gs, "z": bi.z, "H": bi.H, "W": bi.W, "sigma_z": bi.sigma_z, "axis": 2,
              "out": torch.empty(S, bi.H, bi.W, device=dev),
              "dL_dI": torch.randn(S, bi.H, bi.W, device=dev, generator=gen),
              "grads": (torch.empty(gs.n, 3, device=dev), torch.empty(gs.n, 3, device=dev),
                        torch.empty(gs.n, 4, device=dev), torch.empty(gs.n, device=dev))}
        evals += B.gp_count_evals(ctx, gs, bi.z, bi.H, bi.W, bi.sigma_z)
        items.append(it)
    t_plan = time.perf_counter()
    plan = B.BatchPlan(ctx, items, autotune=True)
    t_plan = time.perf_counter() - t_plan
    log(f"batched setup {time.perf_counter() - t0:.1f}s (plan + autotune {t_plan:.1f}s), "
        f"{sum(it['gs'].n for it in items)} Gaussians, {evals:.3e} fwd evals/step")

    def plain_step():
        for it in items:
            B.gp_render_slices(ctx, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], out=it["out"])
            B.gp_render_backward(ctx, it["gs"], it["z"], it["H"], it["W"], it["sigma_z"], it["dL_dI"],
                                 grads=it["grads"])

    def timed(fn, n):
        evs = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in evs]

    for _ in range(warmup):
        plan.run()
        plain_step()
    plan.wait()
    torch.cuda.synchronize()
    b_ms = timed(lambda: plan.run(), steps)
    plan.wait()
    p_ms = timed(plain_step, steps)
    info = plan.info()
    plan.close()
    work_gb = sum(2 * it["out"].numel() * 4 for it in items) / 1e9  # images + dL/dI
    return {"workload": f"{n_sets} sets, N log-uniform in [1k, 200k], square slices of side in {{128, 256, 512, 1024}}, "
                        "8-64 planes, sigma_z ~ U(1, 6), fwd + bwd against seeded dL/dI; one autotuned graph "
                        "launch per step",
            "n_items": len(items), "n_gaussians": int(sum(it["gs"].n for it in items)),
            "evals_fwd_per_step": float(evals), "steps": steps, "warmup": warmup,
            "ms_per_step": float(np.mean(b_ms)), "value": 2.0 * evals / (np.mean(b_ms) * 1e-3), "unit": UNIT,
            "slices_per_s": sum(len(it["z"]) for it in items) / (np.mean(b_ms) * 1e-3),
            "plain": {"ms_per_step": float(np.mean(p_ms)), "value": 2.0 * evals / (np.mean(p_ms) * 1e-3),
                      "launch": f"{len(items)} x (gp_render_slices + gp_render_backward) on one stream"},
            "speedup_vs_plain": float(np.mean(p_ms) / np.mean(b_ms)),
            "autotuned": info,
            "l2": f"not flushed: every step writes and reads {work_gb:.1f} GB of images and gradients, "
                  f"{work_gb * 1e3 / 126:.0f}x the 126 MB L2"}


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    # --case small: the first 12 of the sets (a few GB on the device, for profiler captures)
    r = batched_comparison(args.steps, args.warmup, n_sets=12 if args.case == "small" else 64)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched: " + r["workload"], "n_items": r["n_items"],
                       "n_gaussians": r["n_gaussians"], "l2": r["l2"], "autotuned": r["autotuned"]},
            "plain_launches": r["plain"], "speedup_vs_plain": r["speedup_vs_plain"],
            "slices_per_s": r["slices_per_s"]}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- serving workload

SERVE_KINDS = ("slice", "stack", "voxelize")


def serving_stream(rate, n, n_sets, seed):
    """A seeded request stream: Poisson arrival offsets (s) and, per request, its
    kind (a slice of side 256-1024 on a random axis, a 16-slice 512^2 stack, or
    a 256^3 voxelize), set and parameters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    reqs = []
    for kind in rng.choice(3, n):
        sid = int(rng.integers(0, n_sets))
        if kind == 2:
            reqs.append({"kind": 2, "set": sid})
        elif kind == 0:
            side = int(rng.integers(256, 1025))
            reqs.append({"kind": 0, "set": sid, "side": side, "axis": int(rng.integers(0, 3)),
                         "z": np.array([rng.uniform(0, 1024)], np.float32)})
        else:
            z0 = rng.uniform(0, 1024 - 16)
            reqs.append({"kind": 1, "set": sid, "z": (z0 + np.arange(16)).astype(np.float32)})
    return arrivals, reqs


def _latency_summary(lat_ms, n, wall):
    a = np.asarray(lat_ms)
    return {"requests": n, "throughput_req_per_s": n / wall, "p50_ms": float(np.percentile(a, 50)),
            "p99_ms": float(np.percentile(a, 99)), "mean_ms": float(a.mean())}


def serve_served(B, srv, pools, arrivals, reqs):
    """The stream through the server: each request is submitted at its arrival
    time (once an output buffer of its kind is free, as a client with a bounded
    number of outstanding requests would); latency runs from the arrival to the
    completion the server reports."""
    import threading
    kinds = (B.GP_REQ_SLICE, B.GP_REQ_STACK, B.GP_REQ_VOXELIZE)
    free = {k: list(range(len(v))) for k, v in pools.items()}
    lock = threading.Lock()
    lat, pend, batch = [], {}, []
    done_evt = threading.Event()

    def poller():
        while not (done_evt.is_set() and not pend):
            with lock:
                items = list(pend.items())
            if not items:
                time.sleep(0.0005)
                continue
            for t, (kind, slot, lag_ms) in items:
                res = srv.poll(t, timeout_ms=0)
                if res is not None:
                    with lock:
                        lat.append(lag_ms + res["latency_ms"])
                        batch.append(res["batch_size"])
                        free[kind].append(slot)
                        del pend[t]
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for at, r in zip(arrivals, reqs):
        while time.perf_counter() - t0 < at:
            time.sleep(min(0.0005, max(0.0, at - (time.perf_counter() - t0))))
        kind = kinds[r["kind"]]
        while True:
            with lock:
                if free[kind]:
                    slot = free[kind].pop()
                    break
            time.sleep(0.0002)
        buf = pools[kind][slot]
        lag_ms = (time.perf_counter() - t0 - at) * 1e3
        if r["kind"] == 2:
            t = srv.submit(kind, r["set"], buf, X=256, Y=256, Z=256)
        elif r["kind"] == 0:
            sd = r["side"]
            t = srv.submit(kind, r["set"], buf[:sd * sd], z=r["z"], H=sd, W=sd, sigma_z=3.0, axis=r["axis"])
        else:
            t = srv.submit(kind, r["set"], buf, z=r["z"], H=512, W=512, sigma_z=3.0, axis=2)
        with lock:
            pend[t] = (kind, slot, lag_ms)
    done_evt.set()
    th.join()
    wall = time.perf_counter() - t0
    out = _latency_summary(lat, len(reqs), wall)
    out["mean_batch_size"] = float(np.mean(batch))
    return out


def serve_plain(B, ctx, sets, bufs, arrivals, reqs, stream):
    """The same stream through sequential plain calls (gp_render_slices /
    gp_voxelize) on one stream, each waited for before the next starts;
    latency runs from the arrival to the end of the call."""
    lat = []
    t0 = time.perf_counter()
    for at, r in zip(arrivals, reqs):
        while time.perf_counter() - t0 < at:
            time.sleep(min(0.0005, max(0.0, at - (time.perf_counter() - t0))))
        gs = sets[r["set"]]
        if r["kind"] == 2:
            B.gp_voxelize(ctx, gs, 256, 256, 256, vol=bufs[2])
        elif r["kind"] == 0:
            sd = r["side"]
            B.gp_render_slices(ctx, gs, r["z"], sd, sd, 3.0, r["axis"], out=bufs[0][:sd * sd].view(1, sd, sd))
        else:
            B.gp_render_slices(ctx, gs, r["z"], 512, 512, 3.0, 2, out=bufs[1].view(16, 512, 512))
        stream.synchronize()
        lat.append((time.perf_counter() - t0 - at) * 1e3)
    return _latency_summary(lat, len(reqs), time.perf_counter() - t0)


def serving_comparison(rates, n_requests, workers):
    """8 resident sets (50k-2M Gaussians in 1024^3); for each offered rate a
    seeded Poisson stream of n_requests requests, served (continuous batching
    on `workers` workers) and replayed through sequential plain calls."""
    import torch
    from paper_2603_20611_b300 import binding as B
    from paper_2603_20611_b300 import synth
    dev_i = torch.cuda.current_device()
    dev = f"cuda:{dev_i}"
    ctx = B.Context(dev_i)
    pctx = B.Context(dev_i)
    stream = torch.cuda.current_stream()
    sets = [B.GaussianSet.from_numpy(g, dev) for g in synth.serving_sets()]
    srv = B.Server(ctx, workers=workers, max_batch_slices=64)
    for g in sets:
        srv.load_set(g)
    pools = {B.GP_REQ_SLICE: [torch.empty(1024 * 1024, device=dev) for _ in range(48)],
             B.GP_REQ_STACK: [torch.empty(16 * 512 * 512, device=dev) for _ in range(48)],
             B.GP_REQ_VOXELIZE: [torch.empty(256 ** 3, device=dev) for _ in range(24)]}
    bufs = [torch.empty(1024 * 1024, device=dev), torch.empty(16 * 512 * 512, device=dev),
            torch.empty(256, 256, 256, device=dev)]
    # warm-up: every kind on every set through both arms (workspaces grow once)
    arr_w, req_w = serving_stream(1e6, 48, len(sets), 5004)
    serve_served(B, srv, pools, arr_w, req_w)
    serve_plain(B, pctx, sets, bufs, arr_w, req_w, stream)
    per_rate = []
    for k, rate in enumerate(rates):
        arrivals, reqs = serving_stream(rate, n_requests, len(sets), 5005 + k)
        st0 = srv.stats()
        served = serve_served(B, srv, pools, arrivals, reqs)
        st1 = srv.stats()
        served["batches"] = st1["batches"] - st0["batches"]
        plain = serve_plain(B, pctx, sets, bufs, arrivals, reqs, stream)
        per_rate.append({"offered_req_per_s": rate, "served": served, "plain": plain,
                         "throughput_vs_plain": served["throughput_req_per_s"] / plain["throughput_req_per_s"],
                         "p99_vs_plain": served["p99_ms"] / plain["p99_ms"]})
        log(f"serving rate {rate}: served {served['throughput_req_per_s']:.0f} req/s p50 {served['p50_ms']:.2f} "
            f"p99 {served['p99_ms']:.2f} ms; plain {plain['throughput_req_per_s']:.0f} req/s "
            f"p50 {plain['p50_ms']:.2f} p99 {plain['p99_ms']:.2f} ms")
    stats = srv.stats()
    srv.close()
    return {"workload": "8 resident sets of 50k-2M Gaussians in 1024^3; Poisson arrivals; requests uniform over "
                        "{1 slice 256^2-1024^2 on a random axis, 16-slice 512^2 stack, 256^3 voxelize}",
            "workers": workers, "per_rate": per_rate, "server_stats": stats,
            "plain": "the same seeded request stream through sequential gp_render_slices / gp_voxelize calls on "
                     "one stream, each finished before the next starts",
            "latency": "from the request's arrival time to its completion, in both arms"}


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    rates = [float(r) for r in args.rates.split(",")]
    r = serving_comparison(rates, args.serve_requests, args.serve_workers)
    best = max(r["per_rate"], key=lambda x: x["served"]["throughput_req_per_s"])
    line = {"metric": "served requests/s with p50/p99 latency", "value": best["served"]["throughput_req_per_s"],
            "unit": "req/s", "n_gpus": 1, "steps": len(rates), "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: " + r["workload"], "workers": r["workers"],
                       "requests_per_rate": args.serve_requests},
            "per_rate": r["per_rate"], "plain": r["plain"], "latency": r["latency"],
            "server_stats": r["server_stats"]}
    print(json.dumps(line), flush=True)
    return 0


def speckle_blob_volume(torch, dev, shape, seed=2003, n_blobs=16):
    """Ultrasound-shaped target [Z, Y, X] on the device: Rayleigh(1) speckle times
    a sum of 16 isotropic blobs (std U(20, 80) voxels, centres uniform), scaled
    to [0, 1]; seeded."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    Z, Y, X = shape
    z = torch.arange(Z, device=dev, dtype=torch.float32) + 0.5
    y = torch.arange(Y, device=dev, dtype=torch.float32) + 0.5
    x = torch.arange(X, device=dev, dtype=torch.float32) + 0.5
    env = torch.zeros(shape, device=dev)
    for _ in range(n_blobs):
        c = torch.rand(3, generator=g, device=dev) * torch.tensor([X, Y, Z], device=dev, dtype=torch.float32)
        sd = 20.0 + 60.0 * torch.rand(1, generator=g, device=dev)
        gz = torch.exp(-0.5 * ((z - c[2]) / sd) ** 2)
        gy = torch.exp(-0.5 * ((y - c[1]) / sd) ** 2)
        gx = torch.exp(-0.5 * ((x - c[0]) / sd) ** 2)
        env += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    u = torch.rand(shape, generator=g, device=dev).clamp_(min=1e-12)
    vol = torch.sqrt(-2.0 * torch.log(u)) * env  # Rayleigh(1) speckle
    return vol / vol.max()


def run_ultrasound(args):
    """The ultrasound-shaped configuration: 200k Gaussians in 512^3, sigma_z = 5,
    against a speckle-times-blobs target.  --workload ultrasound renders all 512
    slices of 512^2 (forward + MSE + backward); --workload voxelize runs the
    voxelizer (Eq. 12) over the 512^3 grid forward + MSE + backward.  Metric:
    algorithmic evaluations (forward + backward) per second."""
    import torch
    from paper_2603_20611_b300 import binding as B
    from paper_2603_20611_b300 import synth
    torch.cuda.set_device(0)
    dev = "cuda:0"
    # the backward takes the forward's bins (parameters unchanged); --exp picks the
    # rasterisers' exponential (the voxelizer always evaluates exp2 per voxel)
    ctx = B.Context(0, reuse_bins=True, exp_mode=EXP_MODES[args.exp], tile=args.tile,
                    raster=RASTER_FORMS[args.raster])
    # --case small (for kernel profiles): 50k Gaussians in 320^3 (the same density; a
    # 131 MB volume, just above L2) against a two-blob target, so that few launches come
    # before the rasterisers
    small = args.case == "small"
    D = 320 if small else 512
    g = synth.ultrasound(n=50_000, extent=(D, D, D)) if small else synth.ultrasound()
    gs = B.GaussianSet.from_numpy(g, dev)
    target = speckle_blob_volume(torch, dev, (D, D, D), n_blobs=2 if small else 16)
    stream = torch.cuda.current_stream()
    grads = (torch.empty(g.n, 3, device=dev), torch.empty(g.n, 3, device=dev), torch.empty(g.n, 4, device=dev),
             torch.empty(g.n, device=dev))
    out = torch.empty(D, D, D, device=dev)
    G = torch.empty_like(out)
    loss = torch.zeros(1, device=dev)
    z = synth.slice_positions(range(D))
    if args.workload == "ultrasound":
        evals = B.gp_count_evals(ctx, gs, z, D, D, 5.0)
        evaluated = B.gp_count_evaluated(ctx, gs, z, D, D, 5.0)

        def step():
            B.gp_render_slices(ctx, gs, z, D, D, 5.0, out=out)
            B.gp_mse_grad(ctx, out, target, dL_dI=G, loss=loss)
            B.gp_render_backward(ctx, gs, z, D, D, 5.0, G, grads=grads)
        fwd_phase, bwd_phase = "fwd", "bwd"
        ops = (OPS_PER_EVAL_ROW if args.exp == "row" else OPS_PER_EVAL)["bwd"]
        name = (f"ultrasound slice stack: {g.n // 1000}k Gaussians, {D}^3, sigma_z = 5, all {D} slices, "
                "fwd + MSE + bwd")
    else:
        evals = B.gp_count_vox_evals(ctx, gs, D, D, D)
        evaluated = B.gp_count_vox_evaluated(ctx, gs, D, D, D)

        def step():
            B.gp_voxelize(ctx, gs, D, D, D, vol=out)
            B.gp_mse_grad(ctx, out, target, dL_dI=G, loss=loss)
            B.gp_voxelize_backward(ctx, gs, D, D, D, G, grads=grads)
        fwd_phase, bwd_phase = "vox_fwd", "vox_bwd"
        ops = OPS_PER_EVAL["bwd"]  # the voxelizer planes run the slice rasterisers with per-pixel exp2
        name = f"ultrasound voxelize: {g.n // 1000}k Gaussians, {D}^3 grid, Eq. 12 fwd + MSE + bwd"
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    fp32_peak = fp32_probe_peak(ctx, stream)
    sfu_peak = fp32_probe_peak(ctx, stream, mode=3) if args.exp == "hw" and ops else None
    # the timed steps record phase events around the two rasterisers only (the
    # roofline's launch times) and no host synchronisation between them; the
    # whole phase breakdown comes from a separate pass
    ctx.timing(True, phases=(fwd_phase, bwd_phase))
    ctx.timing_read()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    phases = ctx.timing_read()
    n_ph = min(args.steps, 5)
    ctx.timing(True)
    ctx.timing_read()
    for _ in range(n_ph):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    phases_all = ctx.timing_read()
    ctx.timing(False)
    t = float(np.mean(ms))
    line = {"metric": METRIC, "value": 2.0 * evals / (t * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "n_gaussians": g.n, "l2": "flushed between steps (256 MiB write)",
                       "exp": args.exp if args.workload == "ultrasound" else "poly",
                       "exp_note": EXP_NOTE[args.exp if args.workload == "ultrasound" else "poly"]},
            "evals_fwd_per_step": evals, "rasteriser": args.raster,
            "phase_ms_per_step": {k: v[0] / n_ph for k, v in phases_all.items() if v[2]},
            "phase_timing": f"a separate pass of {n_ph} steps with every phase timed; the timed steps record "
                            "events around the two rasterisers only"}
    ops_t = OPS_PER_EVAL_ROW if (args.exp == "row" and args.workload == "ultrasound") else OPS_PER_EVAL
    # one rasteriser launch per step and pass (the voxelizer's backward phase also
    # holds its small gradient-finish kernel)
    line["passes"] = {p: pass_roofline(evals, evals * (evaluated[i] / max(evals, 1)), ops_t[p],
                                       phases[ph][0] * 1e-3 / args.steps, fp32_peak,
                                       raster_kernel(p, args.raster, args.exp, args.workload == "voxelize"))
                      for i, (p, ph) in enumerate((("fwd", fwd_phase), ("bwd", bwd_phase)))}
    if ops:
        bwd_s = phases[bwd_phase][0] * 1e-3 / args.steps
        achieved = evals * ops / bwd_s / 1e12
        line["roofline"] = {"bound": "alu", "kernel": raster_kernel("bwd", args.raster, args.exp,
                                                                    args.workload == "voxelize"),
                            "achieved": achieved,
                            "peak": fp32_peak / 1e12, "frac": achieved / (fp32_peak / 1e12),
                            "unit": "Tinst/s (FP32+INT lane instructions)", "ops_per_eval": ops,
                            "peak_kind": "measured FMA probe, best of 5 bursts, same run",
                            **sfu_roofline(sfu_peak, evals, bwd_s)}
    print(json.dumps(line), flush=True)
    return 0


def run_codec(args):
    """Encode (device quantisation, Morton sort, delta streams) and decode of the
    500k-Gaussian microscopy set, timed with CUDA events; throughput in
    Gaussians/s and algorithmic bytes (44 B of parameters + 22 B of streams per
    Gaussian) against the measured HBM copy bandwidth.  The host LZMA stage is
    timed separately (wall clock)."""
    import torch
    from paper_2603_20611_b300 import binding as B
    from paper_2603_20611_b300 import synth
    torch.cuda.set_device(0)
    ctx = B.Context(0)
    g = microscopy_set(synth, 1002)
    gs = B.GaussianSet.from_numpy(g, "cuda:0")
    stream = torch.cuda.current_stream()
    hdr, streams, _ = B.gp_encode(ctx, gs)
    out = B.gp_decode(ctx, hdr, streams)
    for _ in range(args.warmup):
        B.gp_encode(ctx, gs)
        B.gp_decode(ctx, hdr, streams)
    flush = torch.empty(64 * 1024 * 1024, device="cuda:0")  # 256 MiB > 126 MB L2
    torch.cuda.synchronize()
    enc_ms, dec_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        hdr, streams, _ = B.gp_encode(ctx, gs)  # synchronous (bounding-box readback)
        e1.record(stream)
        B.gp_decode(ctx, hdr, streams)
        e2.record(stream)
        torch.cuda.synchronize()
        enc_ms.append(e0.elapsed_time(e1))
        dec_ms.append(e1.elapsed_time(e2))
    t0 = time.perf_counter()
    blob = B.encode_bytes(ctx, gs)
    t_host = time.perf_counter() - t0
    n = g.n
    peaks = measured_peaks() or {}
    hbm = peaks.get("hbm_gbs", 6400.0)
    e_ms, d_ms = float(np.median(enc_ms)), float(np.median(dec_ms))
    line = {"metric": "codec Gaussians/s (encode + decode on the device)", "value": n / ((e_ms + d_ms) * 1e-3),
            "unit": "Gaussians/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": e_ms + d_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/u16", "data": "synthetic",
            "config": {"workload": "codec of the 500k-Gaussian microscopy set: 14-bit positions, 12-bit log "
                                   "scales, quaternions and intensities, Morton order, zigzag deltas", "n": n,
                       "l2": "flushed before each encode (256 MiB write); the decode reads the streams the "
                             "encode just wrote"},
            "encode_ms": e_ms, "decode_ms": d_ms,
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                         "encode_achieved": n * 66 / (e_ms * 1e-3) / 1e9,
                         "decode_achieved": n * 66 / (d_ms * 1e-3) / 1e9,
                         "algorithmic_bytes_per_gaussian": 66},
            "host_lzma": {"seconds": t_host, "bytes": len(blob), "raw_param_bytes": n * 44,
                          "ratio_vs_fp32_params": n * 44 / len(blob)}}
    line["roofline"]["frac"] = line["roofline"]["decode_achieved"] / hbm
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--exp", default="poly", choices=sorted(EXP_MODES),
                    help="exponential: poly (default), hw (SFU ex2.approx) or row (poly, factored per pixel row)")
    ap.add_argument("--det", action="store_true")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--raster", default="auto", choices=sorted(RASTER_FORMS),
                    help="rasteriser form: auto (row units on voxelizer planes, block-culled on slices), block or rows")
    ap.add_argument("--fwd-px", type=int, default=0)
    ap.add_argument("--bwd-px", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rebin", action="store_true", help="the backward re-bins instead of reusing the forward's")
    ap.add_argument("--loss", default="mse", choices=["mse", "l1dssim"],
                    help="fit-step loss: MSE, or the paper's L1 + 0.2 D-SSIM")
    ap.add_argument("--ref-px", type=int, default=2048)
    ap.add_argument("--ref-gauss", type=int, default=0, help="0 = twice the oracle's threads")
    ap.add_argument("--case", default="microscopy", choices=["microscopy", "small"])
    ap.add_argument("--workload", default="fit", choices=["fit", "batched", "serving", "codec", "ultrasound",
                                                           "voxelize"])
    ap.add_argument("--view", default="axis", choices=["axis", "oblique"],
                    help="fit step on axis-aligned planes, or on a seeded oblique stack through the centre")
    ap.add_argument("--rates", default="1000,3000,10000,30000")
    ap.add_argument("--serve-requests", type=int, default=3000)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--fit-only", action="store_true",
                    help="the fit step alone, without the batched and served comparisons")
    ap.add_argument("--fit-rates", default="3000,30000",
                    help="offered request rates of the served comparison attached to the fit-step line")
    args = ap.parse_args()
    if args.case == "small":
        use_small_case()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.warmup < 3 and args.impl == "native":
        log("note: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "codec":
        return run_codec(args)
    if args.workload in ("ultrasound", "voxelize"):
        return run_ultrasound(args)
    return run_native(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
