#!/usr/bin/env python
"""Benchmark: reconstructions/s and p50/p99 ms per projection on the paper-scale
workload (256x256x120 reference volume at 2x2x2.5 mm, K=3 PCA modes, 512x384
cone-beam detector at 0.776 mm, 10 iterations per projection, warm start from
the previous frame), through the pcarecon C ABI on one B300 per rank.

One step = one full reconstruction (Section 2.2's alternation to its 10-iteration
cap, then the Section 2.3 tumor fixed point) of one projection: frame j at
gantry angle j deg and breathing time j/6 s of the 1.5x-amplitude phantom, with
1% noise of seed j. Arms:

  default        the on-device loop (CUDA graph with a conditional WHILE node),
                 inputs resident in HBM: `value`, p50/p99; the same frames
                 through pr_reconstruct with pinned host y (`e2e`); the plain
                 FP32 host-driven loop (`plain_fp32`); per-kernel CUDA-event
                 times and the roofline of the dominant kernel; the FP64
                 oracle timed on the host cores (`cpu_baseline`).
  --impl reference
                 the FP64 CPU oracle as it stands (the only reference that
                 exists for this method), one bounded sample per step.

Prints one JSON line on rank 0. Multi-GPU runs (torchrun) give each rank its
own independent patient stream; ranks exchange only the timing (barrier and
max/sum of scalars), never data.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reconstructions/s and p50/p99 ms per projection (256²×120, K=3) vs plain FP32 path"
UNIT = "reconstructions/s"
WORKLOAD = "paper-scale plain method, %s storage: 256x256x120 @ 2x2x2.5 mm, K=%d, %s detector, 10 iterations"
# Trials and accepted steps per reconstruction of this library's solver on this
# workload (measured on the GPU arm); used only to scale the oracle's per-step
# sample to a whole reconstruction in the reference arm.
TRIALS_PER_SOLVE = 10.7
ITERS_PER_SOLVE = 9.5


# ----------------------------------------------------------------------------
# distributed plumbing (barrier and max/sum of timings only)
# ----------------------------------------------------------------------------


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group("nccl")
    return dist


def barrier(dist):
    if dist is not None:
        import torch

        dist.barrier()
        torch.cuda.synchronize()


def max_over_ranks(dist, x: float, device: str = "cuda") -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float, device: str = "cuda") -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(dist, units: float, elapsed_s: float, device: str = "cuda") -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return sum_over_ranks(dist, units, device) / max_over_ranks(dist, elapsed_s, device)


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------


def build_model_inputs(detector: str = "512x384", K: int = 3):
    from phantom import build_pca, phantom_volume, training_dvfs, tumor_centre, workload_paper

    w = workload_paper(K=K, detector=detector)
    vol = w["vol"]
    f0 = phantom_volume(vol).astype(np.float32)
    pca = build_pca(training_dvfs(vol), w["K"])
    return w, f0, pca.mean.astype(np.float32), pca.U.astype(np.float32), tumor_centre(vol)


FIXED_ANGLE = None  # gantry angle (deg) of every frame with --fixed-angle


def frame_params(w, j):
    deg = w["frame_angle_deg"](j) if FIXED_ANGLE is None else FIXED_ANGLE
    return math.radians(deg), w["frame_time"](j), w["frame_seed"](j)


def make_targets(ctx, w, f0, frames):
    """Measured projections y_j [F][nv][nu] on the device: the phantom warped by
    the 1.5x analytic field at t_j and projected at angle_j through the
    library's warp and projector (a helper model whose 'modes' are the distinct
    fields, evaluated at unit-vector w), plus 1% noise of seed j."""
    import torch

    from phantom import dvf_analytic, standard_normal

    vol, geom = w["vol"], w["geom"]
    times = sorted({round(frame_params(w, j)[1] % 4.0, 9) for j in frames})
    fields = {t: dvf_analytic(vol, t, w["scale"]).astype(np.float32) for t in times}
    ys = torch.empty((len(frames), geom.nv, geom.nu), dtype=torch.float32, device="cuda")
    zero_mean = np.zeros((3,) + vol.shape, np.float32)
    where = {}
    helpers = []
    for g in [times[i:i + 7] for i in range(0, len(times), 7)]:
        U = np.stack([fields[t] for t in g])
        mid = ctx.load_model(vol, geom, f0, zero_mean, U, np.zeros(3))
        helpers.append(mid)
        for k, t in enumerate(g):
            where[t] = (mid, k, len(g))
    for i, j in enumerate(frames):
        th, t, seed = frame_params(w, j)
        mid, k, K = where[round(t % 4.0, 9)]
        e = np.zeros(K)
        e[k] = 1.0
        p = ctx.forward(mid, e, th)
        noise = torch.from_numpy(standard_normal(seed, (geom.nv, geom.nu)).astype(np.float32)).cuda()
        ys[i] = p + 0.01 * p * noise
    for mid in helpers:
        ctx.release_model(mid)
    return ys


# ----------------------------------------------------------------------------
# roofline helpers
# ----------------------------------------------------------------------------

# Algorithmic FP32 work per projector sample of an nch-channel volume: one
# multiply-add per trilinear tap and channel, 8 taps x 2 flop x nch (the
# weights and the sample position, shared by the channels, are not counted).
def flops_per_sample(nch: int) -> int:
    return 2 * 8 * nch


def timed_frames(steps: int, warmup: int):
    """Frames of a run: `warmup` frames just before the rotation (j = -W..-1),
    then `steps` frames spread evenly over one gantry rotation (j = floor(i
    360 / steps); every frame j >= 360 / steps apart warm-starts from the one
    before it in this list). With 360 steps every projection of the rotation
    is solved once."""
    if steps <= 360:
        timed = [(i * 360) // steps for i in range(steps)]
    else:
        timed = list(range(steps))
    return list(range(-warmup, 0)) + timed


def warp_voxels_evaluated(vol, box, block_voxels: int = 512) -> int:
    """Voxels of the warp pass's chunks (block_voxels consecutive voxels of
    the flat grid each, the kernel's 512) that meet the inclusive voxel box
    ((x0, y0, z0), (x1, y1, z1)); the other chunks write zeros without reading
    a field."""
    (x0, y0, z0), (x1, y1, z1) = box
    ix, iy, iz = np.arange(vol.nx), np.arange(vol.ny), np.arange(vol.nz)
    inside = (((iz >= z0) & (iz <= z1))[:, None, None] & ((iy >= y0) & (iy <= y1))[None, :, None]
              & ((ix >= x0) & (ix <= x1))[None, None, :]).ravel()
    n = inside.size
    pad = np.zeros(-n % block_voxels, dtype=bool)
    blocks = np.concatenate([inside, pad]).reshape(-1, block_voxels).any(axis=1)
    sizes = np.full(blocks.size, block_voxels)
    sizes[-1] = n - block_voxels * (blocks.size - 1)
    return int(sizes[blocks].sum())


def recorded_capture(kernel: str, source: str):
    """The committed ncu record of `kernel` (profiles/traffic.json), only if the
    kernel's source file is unchanged since the capture (else None)."""
    import hashlib

    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        sha = hashlib.sha256(open(os.path.join(ROOT, "paper_1004_0014_b300", "csrc", source), "rb").read()).hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    return rec if rec.get("source_sha256") == sha else None


def recorded_traffic(kernel: str, source: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None."""
    rec = recorded_capture(kernel, source)
    return rec["bytes_per_launch"] if rec else None


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------


def cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(w, f0, mean, U, c0, j=0, openmp=True):
    """Time one whole oracle trial evaluation (warp + projection of every
    detector pixel) and one whole oracle gradient evaluation on frame j of the
    workload, on all host cores (the OpenMP build) or one. The measured
    projection is the oracle's own (its projection of the truth field + noise).
    Returns (t_eval, t_grad, threads)."""
    from oracle import oracle as O
    from phantom import dvf_analytic, standard_normal

    vol, geom = w["vol"], w["geom"]
    th, t, seed = frame_params(w, j)
    threads = O.use_openmp(openmp)
    m = O.Model(vol, f0.astype(np.float64), mean.astype(np.float64), U.astype(np.float64), c0)
    x_t = dvf_analytic(vol, t, w["scale"])
    t0 = time.perf_counter()
    p = O.project(vol, geom, th, O.warp(vol, m.f0, x_t))
    t_eval = time.perf_counter() - t0
    y = p + 0.01 * p * standard_normal(seed, p.shape)
    a, b = O.fit_ab(p, y)
    t0 = time.perf_counter()
    O.gradient(m, geom, th, np.zeros(m.K), a, b, y)
    t_grad = time.perf_counter() - t0
    return t_eval, t_grad, threads


def oracle_recon_seconds(t_eval, t_grad, iters, trials):
    """Oracle time of one reconstruction: Eq. 4 at the start (one evaluation),
    one gradient per accepted step plus the first, one evaluation per trial."""
    return (1 + trials) * t_eval + (1 + iters) * t_grad


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import multiprocessing

    from oracle import oracle as O
    from phantom import dvf_analytic

    w, f0, mean, U, c0 = build_model_inputs(args.detector, args.K)
    vol, geom = w["vol"], w["geom"]
    m_f0 = f0.astype(np.float64)
    frames = timed_frames(args.steps, args.warmup)
    # A step's bounded sample: one whole oracle evaluation of frame j (its warp
    # and its projection of every detector pixel) on all host cores; a
    # reconstruction costs 1 + trials evaluations and 1 + iterations gradients
    # (the GPU arm's counts), the gradient timed once, also whole.
    t_eval1, t_grad1, _ = oracle_sample(w, f0, mean, U, c0, frames[0], openmp=False)  # one core, for context
    _, t_grad, threads = oracle_sample(w, f0, mean, U, c0, frames[0], openmp=True)
    times = []
    for i, j in enumerate(frames):
        th, t, _ = frame_params(w, j)
        x_t = dvf_analytic(vol, t, w["scale"])
        t0 = time.perf_counter()
        O.project(vol, geom, th, O.warp(vol, m_f0, x_t))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t_eval = statistics.mean(times)
    sec = oracle_recon_seconds(t_eval, t_grad, ITERS_PER_SOLVE, TRIALS_PER_SOLVE)
    value = 1.0 / sec
    sec1 = oracle_recon_seconds(t_eval1, t_grad1, ITERS_PER_SOLVE, TRIALS_PER_SOLVE)
    counts = "a reconstruction = %.2f evaluations + %.2f gradients (the GPU arm's measured counts)" % (
        1 + TRIALS_PER_SOLVE, 1 + ITERS_PER_SOLVE)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_eval,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic phantom (seeded)",
        "config": {"workload": WORKLOAD % (args.storage, args.K, args.detector),
                   "frames": "j = %s: angle j deg, t = j/6 s" % frame_list_text(frames[args.warmup:])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu": cpu_model(), "kind": "oracle",
                         "build": "OpenMP (all host cores)", "extrapolated": True,
                         "sample": "per step: one whole FP64 oracle evaluation of frame j (warp + projection of all "
                                   "%d rays), mean %.3f s; one whole gradient %.3f s; %s" %
                                   (geom.n_rays, t_eval, t_grad, counts),
                         "single_core": {"value": 1.0 / sec1, "unit": UNIT, "cores": 1, "extrapolated": True,
                                         "evaluation_s": t_eval1, "gradient_s": t_grad1}},
        "ms_per_step_meaning": "time of one step's sample (one whole oracle evaluation), not of a reconstruction",
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host_cpus": multiprocessing.cpu_count(),
    }
    print(json.dumps(line), flush=True)
    return 0


def frame_list_text(frames) -> str:
    if len(frames) > 1 and all(b - a == frames[1] - frames[0] for a, b in zip(frames, frames[1:])):
        return "%d, %d, ..., %d" % (frames[0], frames[1], frames[-1])
    return ", ".join(str(j) for j in frames)


def run_profile_pass(args):
    """One model at the workload; the solver-pass projector as a line-search
    trial runs it, at --profile-angle degrees: a setup pass (no moments), then
    three trial passes (for ncu: -k regex:k_project_split -s 1 -c 1 takes the
    first trial pass). Prints the CUDA-event time per trial pass."""
    from paper_1004_0014_b300 import PR_BF16, PR_F32, Context, capi

    w, f0, mean, U, c0 = build_model_inputs(args.detector, args.K)
    ctx = Context(0)
    mid = ctx.load_model(w["vol"], w["geom"], f0, mean, U, c0,
                         storage=PR_BF16 if args.storage == "bf16" else PR_F32)
    ctx.set_state(mid, np.array([-1.0, 0.3, 0.05, 0.1, -0.05, 0.0, 0.0][:w["K"]]))
    th = math.radians(args.profile_angle)
    ms = ctx.time_kernel(mid, capi.PR_KERNEL_PROJECT_FH_TRIAL, th, iters=3)
    print(json.dumps({"profile_pass": "k_project_split trial pass", "angle_deg": args.profile_angle, "ms": ms,
                      "samples": ctx.count_samples(mid, th, ctx.get_state(mid))}), flush=True)
    ctx.close()
    return 0


def run_ours(args):
    import torch

    from paper_1004_0014_b300 import PR_LOOP_HOST, Context, capi, default_opts

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world)

    from paper_1004_0014_b300 import PR_BF16, PR_F32

    w, f0, mean, U, c0 = build_model_inputs(args.detector, args.K)
    vol, geom = w["vol"], w["geom"]
    ctx = Context(local)
    bf16 = args.storage == "bf16"
    mid = ctx.load_model(vol, geom, f0, mean, U, c0, storage=PR_BF16 if bf16 else PR_F32)
    W, K = args.warmup, args.steps
    frames = timed_frames(K, W)
    ys = make_targets(ctx, w, f0, frames)
    torch.cuda.synchronize()  # ys was written on torch's stream; the solves read it on ctx.stream
    angles = [frame_params(w, j)[0] for j in frames]
    opts = default_opts(max_iters=w["max_iters"])
    stream = ctx.stream  # every library launch of this context is ordered on this stream

    # ---------------- device-resident, on-device loop ----------------
    ctx.set_state(mid, np.zeros(w["K"]))
    for i in range(W):
        ctx.reconstruct_async(mid, ys[i], angles[i], opts)
    ctx.fetch_result(mid)
    w_start = ctx.get_state(mid)
    st0 = ctx.stats(mid)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for i in range(W, W + K):
            ctx.reconstruct_async(mid, ys[i], angles[i], opts)
            ev[i - W + 1].record(stream)
        ev[K].synchronize()
    torch.cuda.synchronize()
    barrier(dist)
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    elapsed_ms = ev[0].elapsed_time(ev[K])
    last = ctx.fetch_result(mid)
    st1 = ctx.stats(mid)
    launches = st1["kernels"] - st0["kernels"]
    trials = st1["trials"] - st0["trials"]
    max_ms = max_over_ranks(dist, elapsed_ms)
    value = job_throughput(dist, float(K), elapsed_ms / 1000.0)

    # ---------------- end to end: host buffers through pr_reconstruct ----------------
    y_host = ys.cpu().pin_memory()
    # the same W untimed warm-up frames, through the same call, right before
    # the timed ones: the GPU has idled while y_host was staged, and the timed
    # frames start from the state they start from in the device-resident leg
    ctx.set_state(mid, np.zeros(w["K"]))
    for i in range(W):
        capi.pr_reconstruct(ctx._ctx, mid, y_host[i], angles[i], opts)
    e2e_same_start = bool(np.array_equal(ctx.get_state(mid), w_start))
    torch.cuda.synchronize()
    barrier(dist)
    t0 = time.perf_counter()
    for i in range(W, W + K):
        capi.pr_reconstruct(ctx._ctx, mid, y_host[i], angles[i], opts)
    e2e_s = time.perf_counter() - t0
    barrier(dist)
    e2e_value = job_throughput(dist, float(K), e2e_s)
    h2d, d2h = ctx.io_bytes(mid)

    # ---------------- plain FP32 path: host-driven loop ----------------
    plain_opts = default_opts(max_iters=w["max_iters"], loop_mode=PR_LOOP_HOST)
    ctx.set_state(mid, np.zeros(w["K"]))
    for i in range(W):  # the same untimed warm-up, through this path
        capi.pr_reconstruct(ctx._ctx, mid, ys[i], angles[i], plain_opts)
    torch.cuda.synchronize()
    plain = []
    for i in range(W, W + K):
        t0 = time.perf_counter()
        capi.pr_reconstruct(ctx._ctx, mid, ys[i], angles[i], plain_opts)
        plain.append(1000.0 * (time.perf_counter() - t0))
    plain_value = job_throughput(dist, float(K), sum(plain) / 1000.0)

    # ---------------- kernels: CUDA-event times on the library stream ----------------
    ctx.set_state(mid, w_start)
    kern = {}
    for name, which in (("warp_fh", capi.PR_KERNEL_WARP_FH), ("project_fh", capi.PR_KERNEL_PROJECT_FH),
                        ("project_fh_trial", capi.PR_KERNEL_PROJECT_FH_TRIAL),
                        ("regrad", capi.PR_KERNEL_REGRAD), ("warp_f", capi.PR_KERNEL_WARP_F),
                        ("project_f", capi.PR_KERNEL_PROJECT_F)):
        kern[name] = ctx.time_kernel(mid, which, angles[W], iters=20)
    kern["invert_dvf"] = ctx.time_kernel(mid, capi.PR_KERNEL_INVERT, angles[W], iters=5)
    # the dominant kernel over the rotation: the trial pass and its sample
    # count at up to 8 of the timed frames' angles, evenly spaced
    rot_idx = sorted({W + (i * K) // min(K, 8) for i in range(min(K, 8))})
    rot = []
    for i in rot_idx:
        ms_i = ctx.time_kernel(mid, capi.PR_KERNEL_PROJECT_FH_TRIAL, angles[i], iters=10)
        rot.append((math.degrees(angles[i]), ms_i, ctx.count_samples(mid, angles[i], w_start)))
    fixed = None
    if args.adjoint:
        kern["backproject_dot"] = ctx.time_kernel(mid, capi.PR_KERNEL_BACKPROJECT, angles[W], iters=3)
        # fixed gantry angle: the transpose's footprint weights stored once
        t0 = time.perf_counter()
        nb = ctx.fix_angle(mid, angles[W])
        t_build = time.perf_counter() - t0
        kern["backproject_dot_fixed_angle"] = ctx.time_kernel(mid, capi.PR_KERNEL_BACKPROJECT, angles[W], iters=5)
        ctx.fix_angle(mid, float("nan"))
        fixed = {"table_bytes": nb, "build_s": t_build,
                 "adjoint_ms": kern["backproject_dot_fixed_angle"], "adjoint_ms_on_the_fly": kern["backproject_dot"],
                 "table_gbs": (nb + 4 * vol.n * w["K"]) / (kern["backproject_dot_fixed_angle"] / 1000.0) / 1e9}

    # Dominant kernel: the 4-channel projector, bound by instruction issue and
    # FP32 arithmetic (ncu: DRAM ~1%, L1 ~70%, issue ~65%), so its roofline is
    # FP32 flop/s against the FMA peak of 148 SMs x 128 lanes x 2 flop x clock.
    # The warp kernel is the HBM-bound one; its roofline is reported beside it.
    N, R, Km = vol.n, geom.n_rays, w["K"]
    nch = 4 if Km <= 3 else (6 if Km <= 5 else 8)
    # bytes of one voxel's record in the solver volume: nch floats, or the
    # packed 16-byte float32 f + float16 h record of bfloat16 models with K = 4, 5
    rec_bytes = 16 if (bf16 and Km in (4, 5)) else 4 * nch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    # samples the projector evaluates (support box and brick trace, counted by
    # the library with the kernel's own clipping) over the rotation's angles
    samples = sum(r[2] for r in rot) / len(rot)
    t_proj_ms = sum(r[1] for r in rot) / len(rot)
    flops = samples * flops_per_sample(nch)
    per_solve_ms = elapsed_ms / K
    trials_per_solve = trials / K
    share_proj = (1 + trials_per_solve) * t_proj_ms / per_solve_ms
    share_warp = (1 + trials_per_solve) * kern["warp_fh"] / per_solve_ms
    proj_tflops = flops / (t_proj_ms / 1000.0) / 1e12
    bytes_proj = N * rec_bytes + R * 4 * (1 + Km)
    roofline = {"kernel": "k_project_split<%d> (f, h_1..h_%d)" % (nch, Km), "bound": "alu", "achieved": proj_tflops,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": proj_tflops / fp32_peak,
                "traffic": recorded_traffic("k_project_split<4>", "project.cu") if (Km == 3 and not bf16) else None,
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (FMA peak)" % sm_mhz,
                "timed_as": "line-search trial pass (moments and controller included), CUDA events on the library "
                            "stream, averaged over %d angles of the rotation" % len(rot),
                "per_angle": [{"deg": round(d, 1), "ms": t, "samples": int(n)} for d, t, n in rot],
                "samples_per_launch": samples, "flops_per_sample": flops_per_sample(nch),
                "flops_counted": "one multiply-add per trilinear tap and channel (8 x 2 x %d)" % nch,
                "algorithmic_flops_per_launch": flops, "share_of_solve": share_proj,
                "algorithmic_bytes_per_launch": bytes_proj,
                "achieved_gbs": bytes_proj / (t_proj_ms / 1000.0) / 1e9,
                "limiter": "L1 data pipe returning the trilinear corners (ncu, DRAM 1.6%)",
                "l1_data_pipe_pct_of_peak": ((recorded_capture("k_project_split<4>", "project.cu") or {})
                                             .get("l1_data_pipe_pct") if (Km == 3 and not bf16) else None)}
    ts = 2 if bf16 else 4  # bytes per stored value of f0 and U
    # the solver's warp evaluates the 512-voxel chunks that meet the support box at w;
    # with w repeated (the timing loop) the others hold zeros already and are
    # left alone
    n_eval = warp_voxels_evaluated(vol, ctx.warp_box(mid, w_start))
    bytes_warp = n_eval * (12 + 3 * ts * Km + ts + rec_bytes)
    warp_gbs = bytes_warp / (kern["warp_fh"] / 1000.0) / 1e9
    roofline_warp = {"kernel": "k_warp<%d, f+h, %s>" % (Km, "bf16" if bf16 else "float"), "bound": "hbm",
                     "achieved": warp_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": warp_gbs / hbm_peak,
                     "traffic": recorded_traffic("k_warp<3,FH,float>", "warp.cu") if (Km == 3 and not bf16) else None,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)" if peaks else "fallback",
                     "algorithmic_bytes_per_launch": bytes_warp, "share_of_solve": share_warp,
                     "voxels_evaluated": n_eval, "voxels": N}

    # Whole-grid DVF inversion (Section 2.3 with ref. 13), outside the solve:
    # x/dx synthesis (12 + 12K bytes read, 16 written per voxel), then the
    # per-voxel fixed point (the 16-byte field read once, 12 bytes of y written).
    bytes_inv = N * (12 + 3 * ts * Km + 16 + 16 + 12)
    inv_gbs = bytes_inv / (kern["invert_dvf"] / 1000.0) / 1e9
    roofline_invert = {"kernels": "k_dvf_idx + k_invert", "bound": "hbm", "achieved": inv_gbs, "peak": hbm_peak,
                       "unit": "GB/s", "frac": inv_gbs / hbm_peak, "algorithmic_bytes_per_call": bytes_inv,
                       "ms": kern["invert_dvf"], "tol_mm": 1e-5, "max_iter": 64}

    # ---------------- accuracy of the last timed frame (reported, not a parity claim) ----------------
    # Section 3's relative image error e = sqrt(sum (f - f*)^2 / sum f*^2) of the
    # reconstructed image f (the warp at the final w) against the truth image f*
    # (f0 warped by the 1.5x analytic field at the frame's time), and the 3D
    # tumor error against the analytic truth.
    accuracy = None
    if world == 1:
        from phantom import dvf_analytic, tumor_truth

        th_l, t_l, _ = frame_params(w, frames[-1])
        h_mid = ctx.load_model(vol, geom, f0, np.zeros((3,) + vol.shape, np.float32),
                               dvf_analytic(vol, t_l, w["scale"])[None].astype(np.float32), np.zeros(3))
        f_true, _ = ctx.warp(h_mid, np.array([1.0]), with_h=False)
        f_rec, _ = ctx.warp(mid, np.asarray(last["w"]), with_h=False)
        ctx.release_model(h_mid)
        f_true, f_rec = f_true.double(), f_rec.double()
        accuracy = {"frame": int(frames[-1]), "angle_deg": math.degrees(th_l),
                    "relative_image_error": float(torch.linalg.norm(f_rec - f_true) / torch.linalg.norm(f_true)),
                    "relative_image_error_at_w0": None,
                    "tumor_error_mm": float(np.linalg.norm(np.asarray(last["tumor"]) - tumor_truth(vol, t_l, w["scale"])))}
        f_w0, _ = ctx.warp(mid, np.zeros(w["K"]), with_h=False)
        accuracy["relative_image_error_at_w0"] = float(torch.linalg.norm(f_w0.double() - f_true) /
                                                       torch.linalg.norm(f_true))

    # ---------------- BF16 storage of f0 and U: the same frames and loop ----------------
    bf16_arm = None
    if not bf16 and world == 1 and not args.no_extra_arms:
        mid_b = ctx.load_model(vol, geom, f0, mean, U, c0, storage=PR_BF16)
        ctx.set_state(mid_b, np.zeros(w["K"]))
        for i in range(W):
            ctx.reconstruct_async(mid_b, ys[i], angles[i], opts)
        ctx.fetch_result(mid_b)
        sb0 = ctx.stats(mid_b)
        evb = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        torch.cuda.synchronize()
        evb[0].record(stream)
        for i in range(W, W + K):
            ctx.reconstruct_async(mid_b, ys[i], angles[i], opts)
            evb[i - W + 1].record(stream)
        evb[K].synchronize()
        per_b = [evb[i].elapsed_time(evb[i + 1]) for i in range(K)]
        sb1 = ctx.stats(mid_b)
        last_b = ctx.fetch_result(mid_b)
        qb = np.percentile(per_b, [50, 99])
        bf16_arm = {"value": K / (evb[0].elapsed_time(evb[K]) / 1000.0), "unit": UNIT, "p50_ms": float(qb[0]),
                    "p99_ms": float(qb[1]), "trials_per_solve": (sb1["trials"] - sb0["trials"]) / K,
                    "storage": "bfloat16 f0 and U, float32 mean; FP32 arithmetic, FP64 reductions",
                    "w_last": [float(x) for x in last_b["w"]], "J_last": last_b["J"],
                    "vs_fp32_storage": (K / (evb[0].elapsed_time(evb[K]) / 1000.0)) / value}
        ctx.release_model(mid_b)

    # ---------------- short served arm: 16 mixed patients, 8 Hz each, 5 s ----------------
    served = None
    if world == 1 and not args.no_extra_arms:
        sm = serve_measure(16, 8.0, 5.0, "bf16", local, ["batched:2:2", "slots:2"])
        served = {"patients": 16, "rate_hz_each": 8.0, "seconds": 5.0, "frames": len(sm["trace"]),
                  "storage": "served: bfloat16 f0 and U (FP32 arithmetic, FP64 reductions); plain_fp32: float32",
                  "results_identical_to_plain_bf16": bool(sm["same"]),
                  "plain_fp32_one_at_a_time": sm["plain_fp32"],
                  "plain_bf16_one_at_a_time": sm["plain"]}
        for md, r in zip(("batched_2lanes_2frames_per_tick", "slots_2"), sm["runs"]):
            served[md] = {"value": r["value"], "unit": UNIT, "p50_ms": float(np.percentile(r["lat"], 50)),
                          "p99_ms": float(np.percentile(r["lat"], 99)), "gpu_ms_mean": r["gpu_ms_mean"]}

    # ---------------- CPU baseline (rank 0, N = 1) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_eval, t_grad, threads = oracle_sample(w, f0, mean, U, c0, frames[W], openmp=True)
        iters = (st1["iters"] - st0["iters"]) / K
        sec = oracle_recon_seconds(t_eval, t_grad, iters, trials_per_solve)
        cpu = {"value": 1.0 / sec, "unit": UNIT, "cores": threads, "cpu": cpu_model(), "kind": "oracle",
               "build": "OpenMP (all host cores)", "extrapolated": True,
               "sample": "one whole FP64 oracle trial evaluation (warp + projection of all %d rays, %.2f s) and one "
                         "whole gradient evaluation (%.2f s) of frame %d, scaled by this run's %.2f trials and %.2f "
                         "iterations per reconstruction" % (R, t_eval, t_grad, frames[W], trials_per_solve, iters)}

    if rank == 0:
        q = np.percentile(per_step, [50, 99])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": max_ms / K, "p50_ms": float(q[0]), "p99_ms": float(q[1]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic phantom (seeded), measured projections synthesised on the device",
            "config": {"workload": WORKLOAD % (args.storage, Km, args.detector), "volume": [vol.nx, vol.ny, vol.nz],
                       "spacing_mm": [vol.dx, vol.dy, vol.dz], "K": Km, "detector": [geom.nu, geom.nv],
                       "pixel_mm": geom.du, "ray_step_mm": geom.ds, "iterations": w["max_iters"],
                       "frames": ("j = %s (spread over one rotation): angle j deg, t = j/6 s, 1%% noise seed j, "
                                  "each warm-started from the frame before it in this list (warm-up frames j = %d..-1)"
                                  % (frame_list_text(frames[W:]), -W)) if FIXED_ANGLE is None else
                                 ("j = %s at the fixed angle %g deg (fluoroscopy), t = j/6 s, 1%% noise seed j, each "
                                  "warm-started from the frame before it" % (frame_list_text(frames[W:]), FIXED_ANGLE)),
                       "storage": "bfloat16 f0 and U, float32 mean" if bf16 else "float32",
                       "loop": "on-device (CUDA graph, conditional WHILE)",
                       "l2": "inputs larger than L2: %d MB of DVF fields streamed per warp pass"
                             % ((12 + 3 * ts * Km) * N // 2**20),
                       "parallelism": "independent patient streams, one per GPU" if world > 1 else "1 GPU"},
            "plain_fp32": {"value": plain_value, "unit": UNIT, "p50_ms": float(np.percentile(plain, 50)),
                           "p99_ms": float(np.percentile(plain, 99)),
                           "path": "same kernels, host-driven loop (one device-to-host read per trial), no graph",
                           "storage": "same as the served arm (FP32 arithmetic throughout)",
                           "speedup": value / plain_value},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": "pr_reconstruct with pinned host y, result copied back every step",
                    "start_state_identical_to_value_leg": e2e_same_start},
            "gpu_launches": int(launches),
            "solver": {"iters_per_solve": (st1["iters"] - st0["iters"]) / K, "trials_per_solve": trials_per_solve,
                       "line_search_failures": st1["line_search_failures"] - st0["line_search_failures"],
                       "stop_reason_last": last["stop_reason"], "J_last": last["J"],
                       "w_last": [float(x) for x in last["w"]], "tumor_last_mm": [float(x) for x in last["tumor"]]},
            "kernel_ms": kern,
            "roofline": roofline,
            "roofline_warp": roofline_warp,
            "roofline_invert_dvf": roofline_invert,
            "fixed_angle_adjoint": fixed,
            "accuracy": accuracy,
            "bf16_storage": bf16_arm,
            "served": served,
            "clocks": clk.summary(),
            "paper_context": {"s_per_projection": 0.24, "hardware": "Tesla C1060",
                              "workload": "NCAT 256x256x120, K=3, 200x150 projections (context only)"},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# serving arm: many patients streaming frames (--serve)
# ----------------------------------------------------------------------------

SERVE_BINS = 8  # breathing phases per 4 s cycle used to synthesise the frames


def _patient_base(vol):
    """One phantom and its K=5 PCA model at the training amplitude (a process
    pool worker: host arithmetic only)."""
    from phantom import build_pca, phantom_volume, training_dvfs, tumor_centre

    pca = build_pca(training_dvfs(vol), 5)
    return dict(vol=vol, f0=phantom_volume(vol).astype(np.float32), mean=pca.mean.astype(np.float32),
                U=pca.U.astype(np.float32), c0=tumor_centre(vol))


def serve_patients(n_pat: int, workers: int = 0):
    """Patient models of mixed sizes: shape, K and SI amplitude from
    workload_mixed(i). One phantom and K=5 PCA per distinct shape at the
    training amplitude (10 mm SI, 3 mm AP); a patient of amplitude A scales the
    whole field by A / 10 (mean x A / 10, the same unit-norm modes), and keeps
    the first K modes. workers > 0 builds the shapes in that many spawned
    processes."""
    from phantom import workload_mixed

    pats, vols = [], {}
    for i in range(n_pat):
        wl = workload_mixed(i)
        vol = wl["vol"]
        key = (vol.nx, vol.ny, vol.nz)
        vols.setdefault(key, vol)
        pats.append(dict(wl=wl, key=key, alpha=wl["amp_si"] / 10.0, K=wl["K"]))
    keys = list(vols)
    if workers > 0 and len(keys) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp

        with cf.ProcessPoolExecutor(min(workers, len(keys)), mp_context=mp.get_context("spawn")) as ex:
            built = list(ex.map(_patient_base, [vols[k] for k in keys]))
    else:
        built = [_patient_base(vols[k]) for k in keys]
    return dict(zip(keys, built)), pats


def serve_trace(n_pat: int, rate_hz: float, seconds: float, seed: int = 77):
    """Poisson arrivals per patient (exponential gaps of mean 1/rate), the
    gantry advancing 1 degree per frame from a random start; merged in time."""
    ev = []
    for i in range(n_pat):
        rng = np.random.default_rng(seed + i)
        t, f, th0 = float(rng.exponential(1.0 / rate_hz)), 0, float(rng.uniform(0.0, 360.0))
        while t < seconds:
            ev.append((t, i, f, math.radians((th0 + f) % 360.0)))
            t += float(rng.exponential(1.0 / rate_hz))
            f += 1
    ev.sort()
    return ev


def serve_targets(ctx, bases, pats, trace, geom):
    """Measured frames on the host: for each (patient, frame), the patient's
    phantom warped by 1.5 x its amplitude x the analytic field at the frame's
    breathing phase (SERVE_BINS bins per 4 s), projected, 1% noise (seed =
    1000 patient + frame)."""
    import torch

    from phantom import dvf_analytic, standard_normal

    bins = [4.0 * b / SERVE_BINS for b in range(SERVE_BINS)]
    ys = {}
    for key, base in bases.items():
        vol = base["vol"]
        zero = np.zeros((3,) + vol.shape, np.float32)
        fields = np.stack([1.5 * dvf_analytic(vol, t) for t in bins]).astype(np.float32)
        helpers = []
        for g0 in range(0, SERVE_BINS, 7):
            U = fields[g0:g0 + 7]
            helpers.append((g0, U.shape[0], ctx.load_model(vol, geom, base["f0"], zero, U, np.zeros(3))))
        for (t, i, f, th) in trace:
            if pats[i]["key"] != key:
                continue
            b = int(round((t % 4.0) / 4.0 * SERVE_BINS)) % SERVE_BINS
            g0, K, mid = next(h for h in helpers if h[0] <= b < h[0] + h[1])
            e = np.zeros(K)
            e[b - g0] = pats[i]["alpha"]
            p = ctx.forward(mid, e, th)
            noise = torch.from_numpy(standard_normal(1000 * i + f, (geom.nv, geom.nu)).astype(np.float32)).cuda()
            ys[(i, f)] = (p + 0.01 * p * noise).cpu().numpy()
        for _, _, mid in helpers:
            ctx.release_model(mid)
    return ys


def serve_once(ctx, mids, pats, ys, trace, opts, n_slots, local, lanes=0, tick_frames=0):
    """One served pass of the trace with n_slots concurrent solve streams (or,
    lanes > 0, tick-batched with that many ticks in flight and at most
    tick_frames frames per tick), every patient starting from w = 0; latencies
    from the scheduled arrivals."""
    import threading

    for pt, mid in zip(pats, mids):
        ctx.set_state(mid, np.zeros(pt["K"]))
    done = {}
    t_start = [0.0]
    submitted = [0]
    t_submit = [0.0] * len(trace)

    def feeder():
        t0 = time.perf_counter()
        t_start[0] = t0
        for n, (t, i, f, th) in enumerate(trace):
            d = t0 + t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ctx.submit(mids[i], ys[(i, f)], th, opts, tag=n)
            t_submit[n] = time.perf_counter()
            submitted[0] = n + 1

    ctx.serve_start(slots=n_slots, batched_lanes=lanes, tick_frames=tick_frames)
    with ClockSampler(local) as clk:
        th_feed = threading.Thread(target=feeder)
        th_feed.start()
        while len(done) < len(trace):
            if submitted[0] <= len(done):  # nothing outstanding until the next arrival
                time.sleep(0.0002)
                continue
            r = ctx.poll(timeout_ms=120000)
            if r is None or r["status"] != 0:
                raise SystemExit("serving failed: %r" % (r,))
            done[r["tag"]] = (time.perf_counter(), r)
        th_feed.join()
    ctx.serve_stop()
    t_end = max(v[0] for v in done.values())
    lat = np.array([1000.0 * (done[n][0] - (t_start[0] + trace[n][0])) for n in range(len(trace))])
    late = np.array([1000.0 * (t_submit[n] - (t_start[0] + trace[n][0])) for n in range(len(trace))])
    final = {}
    for n, (t, i, f, th) in enumerate(trace):
        final[i] = done[n][1]["w"]
    return dict(lat=lat, late=late, value=len(trace) / (t_end - t_start[0]), final=final, clocks=clk.summary(),
                slots=n_slots, lanes=lanes,
                gpu_ms_mean=float(np.mean([done[n][1]["gpu_ms"] for n in range(len(trace))])))


def _plain_path(ctx, mids, pats, ys, trace):
    """The plain path on a serving trace: the host-driven loop, one frame at a
    time in arrival order, every patient from w = 0. Latency comes from the
    measured service times (start = max(arrival, previous finish)). Returns the
    figures and each patient's final w."""
    from paper_1004_0014_b300 import PR_LOOP_HOST, default_opts

    plain_opts = default_opts(max_iters=10, loop_mode=PR_LOOP_HOST)
    for pt, mid in zip(pats, mids):
        ctx.set_state(mid, np.zeros(pt["K"]))
    svc, final = [], {}
    for (t, i, f, th) in trace:
        t0 = time.perf_counter()
        res = ctx.reconstruct(mids[i], ys[(i, f)], th, plain_opts)
        svc.append(time.perf_counter() - t0)
        final[i] = res["w"]
    finish, lat = 0.0, []
    for (t, i, f, th), s_i in zip(trace, svc):
        finish = max(t, finish) + s_i
        lat.append(1000.0 * (finish - t))
    figures = dict(value=len(trace) / (finish - trace[0][0]), p50_ms=float(np.percentile(lat, 50)),
                   p99_ms=float(np.percentile(lat, 99)), mean_service_ms=1000.0 * float(np.mean(svc)))
    return figures, final


def _load_patients(ctx, bases, pats, geom, storage):
    from paper_1004_0014_b300 import PR_BF16, PR_F32

    mids = []
    for pt in pats:
        b = bases[pt["key"]]
        mids.append(ctx.load_model(b["vol"], geom, b["f0"], pt["alpha"] * b["mean"], b["U"][:pt["K"]], b["c0"],
                                   storage=PR_BF16 if storage == "bf16" else PR_F32))
    return mids


def serve_measure(patients: int, rate: float, seconds: float, storage: str, local: int, modes, workers: int = 8):
    """Serve a Poisson trace of `patients` mixed patients at `rate` Hz each for
    `seconds` once per mode in `modes` ("batched:L:F" = tick-batched with L
    lanes and at most F frames per tick (0 or absent = all), "slots:S" = S solve
    streams), then the plain path (host-driven loop, one frame at a time in
    arrival order) on the same trace with the same models, whose final w the
    served ones must equal bitwise. With bfloat16 storage the plain path also
    runs on float32-storage models of the same patients (`plain_fp32`).
    Returns the runs and the plain paths' figures."""
    from paper_1004_0014_b300 import Context, default_opts

    bases, pats = serve_patients(patients, workers)
    geom = pats[0]["wl"]["geom"]
    trace = serve_trace(patients, rate, seconds)
    ctx = Context(local)
    ys = serve_targets(ctx, bases, pats, trace, geom)
    mids = _load_patients(ctx, bases, pats, geom, storage)
    opts = default_opts(max_iters=10)
    # warm-up: two frames per patient, then every patient restarts from w = 0
    ctx.serve_start(slots=4)
    for i, mid in enumerate(mids):
        for f in range(2):
            ctx.submit(mid, ys[next(k for k in ys if k[0] == i)], 0.0, opts, tag=f)
    for _ in range(2 * len(mids)):
        ctx.poll(timeout_ms=120000)
    ctx.serve_stop()
    runs = []
    for mode in modes:
        kind, n, *rest = mode.split(":")
        runs.append(serve_once(ctx, mids, pats, ys, trace, opts, int(n) if kind == "slots" else 4, local,
                               lanes=int(n) if kind == "batched" else 0, tick_frames=int(rest[0]) if rest else 0))
    plain, final_plain = _plain_path(ctx, mids, pats, ys, trace)
    same = all(np.array_equal(np.asarray(r["final"][i]), np.asarray(final_plain[i])) for r in runs for i in r["final"])
    plain_fp32 = plain
    if storage != "f32":
        for mid in mids:
            ctx.release_model(mid)
        mids32 = _load_patients(ctx, bases, pats, geom, "f32")
        plain_fp32, _ = _plain_path(ctx, mids32, pats, ys, trace)
    ctx.close()
    return dict(runs=runs, plain=plain, plain_fp32=plain_fp32, same=same, trace=trace, pats=pats)


def run_serve(args):
    world, rank, local = dist_env()
    if world > 1:
        raise SystemExit("--serve runs on one GPU")
    if args.serve_mode == "batched":
        modes = ["batched:%s:%s" % (x, f) for x in str(args.lanes).split(",")
                 for f in str(args.tick_frames).split(",")]
    else:
        modes = ["slots:%s" % x for x in str(args.slots).split(",")]
    m = serve_measure(args.patients, args.rate, args.seconds, args.storage, local, modes)
    runs, plain, trace, pats = m["runs"], m["plain"], m["trace"], m["pats"]
    head = runs[0]
    lat, late = head["lat"], head["late"]
    line = {
        "metric": "served reconstructions/s and p50/p99 ms per projection (%d patients, mixed sizes, %g Hz Poisson "
                  "each) vs plain FP32 path" % (args.patients, args.rate),
        "value": head["value"], "unit": UNIT, "n_gpus": 1, "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "higher_is_better": True, "dtype": "f32",
        "data": "synthetic phantoms (seeded)",
        "frames": len(trace), "offered_hz": args.rate * args.patients, "seconds": args.seconds,
        "mode": modes[0],
        "sweep": [{"mode": md, "value": r["value"], "p50_ms": float(np.percentile(r["lat"], 50)),
                   "p99_ms": float(np.percentile(r["lat"], 99)), "gpu_ms_mean": r["gpu_ms_mean"]}
                  for md, r in zip(modes, runs)],
        "config": {"workload": "serving: %d patients, shapes %s, K 3-5, SI amplitude 8-20 mm (whole field scaled), "
                               "512x384 detector, 10 iterations, warm start per patient, %s storage" %
                               (args.patients, sorted(set(str(p["key"]) for p in pats)), args.storage),
                   "frames": "per patient: Poisson arrivals, 1 deg per frame from a random start, breathing phase "
                             "from the arrival time (%d bins per 4 s), 1%% noise" % SERVE_BINS},
        "latency": "scheduled arrival to result on the host clock (queue + solve)",
        "submit_lateness_ms": {"p50": float(np.percentile(late, 50)), "p99": float(np.percentile(late, 99)),
                               "max": float(late.max())},
        "capacity_note": "throughput is capped by the GPU's solve rate when the offered load exceeds it; "
                         "latency then grows with the length of the trace",
        "plain_fp32": dict(m["plain_fp32"], path="host-driven loop (PR_LOOP_HOST), one frame at a time in arrival "
                                                 "order; latency from the measured service times with start = "
                                                 "max(arrival, previous finish)", storage="float32"),
        "plain_same_storage": dict(plain, storage="%s, as the served arm" % args.storage),
        "results_identical_to_plain_same_storage": bool(m["same"]),
        "gpu_ms_mean": head["gpu_ms_mean"],
        "clocks": head["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# batched arm: uneven patients' solves in one graph launch (--batch)
# ----------------------------------------------------------------------------


def run_batch(args):
    from paper_1004_0014_b300 import PR_BF16, PR_F32, PR_LOOP_HOST, Context, default_opts

    world, rank, local = dist_env()
    if world > 1:
        raise SystemExit("--batch runs on one GPU")
    n_pat, per = 8, 8
    bases, pats = serve_patients(n_pat, 8)
    geom = pats[0]["wl"]["geom"]
    trace = []  # (t, patient, frame, angle): 8 random angles and breathing times per patient, seed = patient id
    for i in range(n_pat):
        rng = np.random.default_rng(i)
        for f in range(per):
            trace.append((float(rng.uniform(0.0, 4.0)), i, f, float(rng.uniform(0.0, 2.0 * math.pi))))
    order = [(t, i, f, th) for f in range(per) for (t, i, ff, th) in trace if ff == f]  # interleaved
    ctx = Context(local)
    ys = serve_targets(ctx, bases, pats, order, geom)
    mids = []
    for pt in pats:
        b = bases[pt["key"]]
        mids.append(ctx.load_model(b["vol"], geom, b["f0"], pt["alpha"] * b["mean"], b["U"][:pt["K"]], b["c0"],
                                   storage=PR_BF16 if args.storage == "bf16" else PR_F32))
    opts = default_opts(max_iters=10)
    ids = [mids[i] for (_, i, _, _) in order]
    yl = [ys[(i, f)] for (_, i, f, _) in order]
    angs = [th for (_, _, _, th) in order]

    def reset():
        for pt, mid in zip(pats, mids):
            ctx.set_state(mid, np.zeros(pt["K"]))

    reset()
    ctx.reconstruct_batch(ids, yl, angs, opts)  # builds and instantiates the graph
    reps = 3
    t_batch = []
    with ClockSampler(local) as clk:
        for _ in range(reps):
            reset()
            t0 = time.perf_counter()
            res_b = ctx.reconstruct_batch(ids, yl, angs, opts)
            t_batch.append(time.perf_counter() - t0)
    t_seq, t_plain = [], []
    for mode, acc in ((None, t_seq), (PR_LOOP_HOST, t_plain)):
        o = default_opts(max_iters=10) if mode is None else default_opts(max_iters=10, loop_mode=mode)
        for _ in range(reps):
            reset()
            t0 = time.perf_counter()
            res_s = [ctx.reconstruct(m, y, th, o) for m, y, th in zip(ids, yl, angs)]
            acc.append(time.perf_counter() - t0)
    same = all(np.array_equal(np.asarray(a["w"]), np.asarray(b["w"])) for a, b in zip(res_b, res_s))
    n = len(order)
    line = {
        "metric": "batched reconstructions/s: %d uneven solves in one CUDA graph vs one at a time" % n,
        "value": n / statistics.median(t_batch), "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic phantoms (seeded)",
        "ms_per_batch": 1000.0 * statistics.median(t_batch),
        "config": {"workload": "8 patients, shapes %s, K %s, SI amplitude 8-20 mm (whole field scaled), 8 frames "
                               "each at random angles and breathing times (seed = patient id), interleaved; 512x384 "
                               "detector, 10 iterations" % (sorted(set(str(p["key"]) for p in pats)),
                                                            [p["K"] for p in pats]),
                   "timed": "pr_reconstruct_batch with host frames (H2D staging and result read-back included), "
                            "median of %d" % reps, "storage": args.storage},
        "one_at_a_time_graph": {"value": n / statistics.median(t_seq),
                                "path": "pr_reconstruct per frame (on-device loop), same order"},
        "plain_fp32": {"value": n / statistics.median(t_plain),
                       "path": "pr_reconstruct per frame with the host-driven loop, same order",
                       "storage": "%s, as the batched arm (FP32 arithmetic throughout)" % args.storage},
        "results_identical_to_one_at_a_time": bool(same),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=360)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-arms", action="store_true",
                    help="skip the BF16-storage and short served arms of the default run")
    ap.add_argument("--adjoint", action="store_true", help="also time the gather-adjoint gradient kernel")
    ap.add_argument("--detector", default="512x384", choices=["512x384", "200x150", "1000x750", "40x30", "20x15"],
                    help="detector sampling of the 40x30 cm panel")
    ap.add_argument("--K", type=int, default=3, choices=range(1, 8), help="PCA modes of the paper-scale model")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"], help="storage of f0 and U")
    ap.add_argument("--serve", action="store_true", help="serving arm: patients streaming Poisson frames")
    ap.add_argument("--profile-angle", type=float, default=None,
                    help="run only the projector's trial pass at this gantry angle (for ncu), then exit")
    ap.add_argument("--fixed-angle", type=float, default=None,
                    help="every frame at this gantry angle (fluoroscopy, Section 5) instead of the rotation")
    ap.add_argument("--batch", action="store_true", help="batched arm: 64 uneven solves in one graph launch")
    ap.add_argument("--patients", type=int, default=16)
    ap.add_argument("--rate", type=float, default=15.0, help="frames per second per patient (--serve)")
    ap.add_argument("--seconds", type=float, default=20.0, help="length of the arrival trace (--serve)")
    ap.add_argument("--slots", default="4", help="concurrent solve streams (--serve); a comma list runs each")
    ap.add_argument("--serve-mode", default="batched", choices=["batched", "slots"],
                    help="--serve: tick-batched launches or stream slots")
    ap.add_argument("--lanes", default="2", help="ticks in flight (--serve-mode batched); a comma list runs each")
    ap.add_argument("--tick-frames", default="0",
                    help="most frames per tick (--serve-mode batched, 0 = all pending); a comma list runs each")
    args = ap.parse_args()
    global FIXED_ANGLE
    FIXED_ANGLE = args.fixed_angle
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile_angle is not None:
        return run_profile_pass(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.batch:
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
