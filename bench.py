"""Benchmark of the data-consistency hot path at brain size (320x320 image,
16 coils, variable-density spiral 16 x 2048 = 32768 points, KB width 6,
oversampling 2): DC solves per second to relative residual 1e-4 at mu = 1e-2,
with A^H A applies per second and the per-stage (plain) PCG path beside it.

A step is one DC solve for each slice of a batch of B slices: A^H y
(adjoint NUFFT), rhs = A^H y + mu z, and the preconditioned CG solve of
(A^H A + mu I) x = rhs, each slice with its own phantom and coil maps (one
plan per slice).  By default (--mode batched) the B slices form --streams
groups (2), each a batch on its own stream whose cooperative launches take an
equal share of the resident CTAs (hqs_batch_set_grid), so the groups run side by
side; per group the right-hand sides come from the batched adjoint
(hqs_batch_adjoint_axpy) and the solves run in one cooperative launch
(hqs_batch_dc_solve), each slice to its own tolerance;
--mode fused launches the persistent solve once per slice, --mode plain
the per-stage PCG.  The batch's resident inputs exceed the 129 MB L2, so no
explicit flush is needed between steps.  Inputs are synthetic (seeded
ellipse phantoms, Gaussian-bump coil maps, spiral trajectory).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--mode batched|fused|plain] [--streams S]
                  [--impl ours|reference]
  python bench.py --workload batch64     # 64 uneven slices, batched HQS 20 x 5
  python bench.py --workload mixed320    # A^H A and DC solves at FP32 / BF16x3 / FP16x3
  python bench.py --workload hqs320      # annealed HQS 10 x 5 and PnP-PGD 10 steps, Id / F-1 / Chebyshev
  python bench.py --workload learned320  # learned-preconditioned flexible CG vs DC-PCG

The batch64 workload runs annealed HQS (20 outer x 5 CG iterations, Gaussian
smoothing denoiser) over 64 slices of mixed size {256, 320, 384}^2, 8-20
coils, radial (48-96 spokes x 2n) or spiral (12-24 interleaves x 1024-4096)
trajectories, in one persistent launch replayed from a CUDA graph after the
spreading tile and solve shapes were picked by the autotuner; it reports
slices/s, the batch latency, and the same HQS run slice by slice beside it.
The default line carries a compact run of it (2 timed steps, `batch64_hqs`),
beside the precision variant (`mixed_precision`) and the learned
preconditioner (`learned_precond`), all outside the timed region.

With N > 1 (torchrun) every rank solves its own batch (replicas, weak
scaling); the timed region is bracketed by barriers and the slowest rank's
time is used.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

METRIC = "A^H A applies/s and DC solves/s to 1e-4 residual at 320², 16 coils vs plain PCG"
UNIT = "solves/s"
WORKLOAD = ("brain-sized DC solve: 320x320, 16 coils, spiral 16x2048 (32768 pts), KB W=6, sigma=2, mu=1e-2, "
            "rel. residual 1e-4, DC-preconditioned CG")
MU = 1e-2
TOL = 1e-4
MAX_ITER = 200
# Autotuner cache of this benchmark (one file per rank, removed at the start of
# a run so the shapes are timed on the GPU that runs it).
TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".bench_tune_cache.json")



def read_peaks():
    """Roofline denominators: the measured HBM copy bandwidth and BF16 GEMM
    rates in MEASURED_PEAKS.json at the repository root, or the earlier
    GB300 measurement (6.8 TB/s, 1.9 / 1.7 PFLOP/s) when that file is absent."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]),
                "bf16_tflops_sustained": float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


PEAKS = read_peaks()
HBM_PEAK_GBS = PEAKS["hbm_gbs"]
# FP32 ALU peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop (FMA) per clock
FP32_LANES = 152 * 128


def fp32_peak_tflops(sm_mhz: float) -> float:
    return FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
# Algorithmic bytes of one forward / adjoint at 320^2, 16 coils, G = 640, M = 32768
# (complex64 = 8 B): forward = x + S (fused apodise/coil/pad/row-FFT pass) + grid
# write, column FFT read + write, interpolation read + points + y write;
# adjoint = y + points + grid write (spreading), column IFFT read + write of the
# n kept rows, row IFFT read + S + x write.
_G2L = 640 * 640 * 16 * 8
_ROWS = 320 * 640 * 16 * 8
_S = 320 * 320 * 16 * 8
_Y = 32768 * 16 * 8
_PTS = 32768 * 16 + 32768 * 4
FWD_BYTES = (320 * 320 * 8 + _S + _ROWS) + (_ROWS + _G2L) + (_G2L + _PTS + _Y)
ADJ_BYTES = (_Y + _PTS + _G2L) + (_G2L + _ROWS) + (_ROWS + _S + 320 * 320 * 8)
# DRAM bytes (read + write) of one k_pcg_persistent<640,320> launch from an ncu
# capture of the current kernel (profiles/pcg_persistent_320x16.md); None while
# the kernel has changed since the last capture.
PERSISTENT_TRAFFIC_BYTES = None
# The same for the batched solves of one default step (two concurrent k_pcg_batch
# launches of 8 slices: the sum of both launches' bytes, each captured alone), from
# profiles/pcg_batch_320x16_16slices.md; None while the kernel has changed since the
# last capture (the 68.2 GB there predate the column items over flattened lines).
BATCH_TRAFFIC_BYTES = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="batched", choices=["batched", "fused", "plain"])
    ap.add_argument("--group", type=int, default=64, help="slices per batched launch (at most 64)")
    ap.add_argument("--streams", type=int, default=2,
                    help="batched mode: the slices split into this many groups, each its own batched "
                         "launch on its own stream with an equal share of the resident CTAs")
    ap.add_argument("--phase-trace", action="store_true",
                    help="batched dc320: add the per-phase time of one traced batched solve to the line")
    ap.add_argument("--workload", default="dc320",
                    choices=["dc320", "batch64", "mixed320", "mixedsizes", "hqs320", "learned320", "vol64",
                             "vol128"])
    return ap.parse_args()


# --------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(s[0]) for s in self.samples if len(s) >= 8 and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) >= 8 and s[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            if len(s) < 8:
                continue
            for nm, v in zip(names, s[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- ranks
def max_over_ranks(value: float, dist, device: str = "cuda") -> float:
    """The slowest rank's time (every rank gets it); the value itself at N = 1."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units all ranks processed (each rank the same number: weak scaling)
    per second of the slowest rank."""
    return units_per_rank * world / (ms_max / 1e3)


# --------------------------------------------------------------- workload
def make_slices(B, rank=0):
    import synth
    n, L = 320, 16
    traj = synth.traj_spiral(16, 2048, n)
    slices = []
    for b in range(B):
        seed = 1000 * rank + b
        slices.append(dict(x=synth.phantom(seed, n), smaps=synth.coil_maps(seed, n, L),
                           noise=synth.complex_noise(seed, (L, traj.shape[0]))))
    return n, L, traj, slices


class OracleStep:
    """One step of the benchmark's workload in the FP64 oracle, for one slice
    (the first slice of the GPU step, the same seeded inputs): rhs = A^H y +
    mu z by the gridding adjoint, then DC-preconditioned CG from zero to
    relative residual 1e-4, counting its iterations.  Setting up (the
    Toeplitz kernel and density symbol, y and z) is not timed."""

    def __init__(self):
        from oracle import hqs as ohqs
        from oracle import nufft, toeplitz
        self.nufft, self.toeplitz = nufft, toeplitz
        n, L, traj, sl = make_slices(1)
        s = sl[0]
        self.n, self.traj, self.S = n, traj, s["smaps"]
        t0 = time.perf_counter()
        c = toeplitz.kernel(traj, n, n)
        self.Kh, self.lam = toeplitz.khat(c), toeplitz.chan_symbol(c, n, n)
        self.t_plan = time.perf_counter() - t0
        y = nufft.forward(s["x"], self.S, traj, 6, 2.0)
        sd = math.sqrt(1e-4 * float(np.max(np.sum(np.abs(self.S * s["x"]) ** 2, axis=0))))
        self.y = y + sd * s["noise"]
        self.z = ohqs.gaussian_denoise(nufft.adjoint(self.y, self.S, traj, 6, 2.0), 1.0)

    def __call__(self):
        """Runs one step; returns (seconds, CG iterations)."""
        from oracle import solvers
        t0 = time.perf_counter()
        rhs = self.nufft.adjoint(self.y, self.S, self.traj, 6, 2.0) + MU * self.z
        H = lambda v: self.toeplitz.normal(v, self.S, self.Kh) + MU * v
        M = lambda v: self.toeplitz.precond_apply(v, self.lam, 1.0, MU)
        _, info = solvers.pcg(H, rhs, np.zeros((self.n, self.n)), M, max_iter=MAX_ITER, tol=TOL)
        return time.perf_counter() - t0, info["iters"]


def cpu_oracle_vol_sample(case):
    """The FP64 oracle on the host cores: one 3D gridding forward + adjoint
    (A^H(A x), W = 6) of one coil of the volume; returns seconds."""
    from oracle import nufft3d
    t0 = time.perf_counter()
    y = nufft3d.forward(case["x"], case["smaps"][:1], case["traj"], 6, 2.0)
    nufft3d.adjoint(y, case["smaps"][:1], case["traj"], 6, 2.0)
    return time.perf_counter() - t0


def tests_module(name):
    """A helper module of the test suite (tests/ is not a package)."""
    import importlib
    tdir = os.path.join(ROOT, "tests")
    if tdir not in sys.path:
        sys.path.insert(0, tdir)
    return importlib.import_module(name)


def threads_used():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle arm: each step is one full oracle step of one slice
    (OracleStep), W untimed, K timed; rank 0 alone runs under torchrun."""
    if rank != 0:
        return
    step = OracleStep()
    for _ in range(args.warmup):
        step()
    times, iters = [], []
    for _ in range(args.steps):
        t, it = step()
        times.append(t)
        iters.append(it)
    t_step = float(np.mean(times))
    value = 1.0 / t_step
    sample = (f"per step: one FP64 oracle step of slice 0 (gridding adjoint for A^H y + mu z, then "
              f"DC-preconditioned CG to 1e-4: {np.mean(iters):.1f} iterations), measured, not extrapolated; "
              f"oracle plan {step.t_plan:.1f} s once, untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "batch": 1},
            "oracle_cg_iterations": float(np.mean(iters)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import torch
    import paper_2411_01955_gb300 as hq
    from paper_2411_01955_gb300 import tune

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    B = args.batch
    n, L, traj_np, sl = make_slices(B, rank)
    traj = torch.from_numpy(traj_np).cuda()
    M = traj.shape[0]
    tune_cache = f"{TUNE_CACHE}.{rank}"
    if os.path.exists(tune_cache):
        os.remove(tune_cache)
    plans, ys, zs, rhss, xs = [], [], [], [], []
    for s in sl:
        smaps = torch.from_numpy(s["smaps"].astype(np.complex64)).cuda()
        plan = hq.plan_create(traj, n, n, smaps, 6, 2.0)
        # launch shapes picked by the library's autotuner (timed once per shape, cached)
        tuned = tune.autotune(plan, cache_path=tune_cache)
        x = torch.from_numpy(s["x"].astype(np.complex64)).cuda()
        y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
        hq.forward(plan, x, y)
        y_np = y.cpu().numpy()
        sd = math.sqrt(1e-4 * float(np.max(np.sum(np.abs(s["smaps"] * s["x"]) ** 2, axis=0))))
        y = torch.from_numpy((y_np + sd * s["noise"]).astype(np.complex64)).cuda()
        b0 = torch.empty_like(x)
        hq.adjoint(plan, y, b0)
        z = torch.empty_like(x)
        hq.gaussian_denoise(b0, z, 1.0)       # a plausible HQS iterate for the mu z term
        plans.append(plan)
        ys.append(y)
        zs.append(z)
        rhss.append(torch.empty_like(x))
        xs.append(torch.zeros_like(x))
    nstreams = max(1, args.streams) if args.mode == "batched" else 1
    G_ = max(1, min(args.group, math.ceil(B / nstreams), B))
    groups = [list(range(i, min(i + G_, B))) for i in range(0, B, G_)]
    batches = [hq.Batch([plans[i] for i in g], max_outer=1) for g in groups] if args.mode == "batched" else []
    stream = torch.cuda.current_stream()
    # concurrent groups: each batched launch gets an equal share of the CTAs the batch
    # kernels keep resident (two per SM), so the launches run side by side and one
    # launch's grid barriers do not idle the other's CTAs
    gstreams = [torch.cuda.Stream() for _ in groups] if len(groups) > 1 else [stream]
    if len(groups) > 1:
        cap = 2 * torch.cuda.get_device_properties(dev).multi_processor_count // len(groups)
        for bt in batches:
            bt.set_grid(cap)

    def on_group_streams(fn):
        # fn(group index, stream) on each group's stream, ordered after and before the main stream
        if len(gstreams) == 1:
            for k in range(len(groups)):
                fn(k, stream)
            return
        for gs in gstreams:
            gs.wait_stream(stream)
        for k, gs in enumerate(gstreams):
            with torch.cuda.stream(gs):
                fn(k, gs)
        for gs in gstreams:
            stream.wait_stream(gs)

    def solve_all(mode_):
        if mode_ == "batched":
            on_group_streams(lambda k, gs: batches[k].dc_solve(
                [rhss[i] for i in groups[k]], [xs[i] for i in groups[k]], 1.0, MU, max_iter=MAX_ITER, rel_tol=TOL,
                stream=gs))
            return
        flag = hq.HQS_SOLVE_FUSED if mode_ == "fused" else hq.HQS_SOLVE_PLAIN
        for i in range(B):
            hq.dc_solve(plans[i], 1.0, MU, rhss[i], xs[i], max_iter=MAX_ITER, rel_tol=TOL,
                        precond=hq.HQS_PRECOND_DC, mode=flag | hq.HQS_SOLVE_X0_ZERO, want_info=False)

    def step(mode_=args.mode, ys_=None):
        yy = ys if ys_ is None else ys_
        if mode_ == "batched":
            # per group on its stream: A^H y + mu z of its slices (the FFT passes
            # batched), then its batched solve
            def grp(k, gs):
                g = groups[k]
                batches[k].adjoint_axpy([yy[i] for i in g], MU, [zs[i] for i in g], [rhss[i] for i in g], stream=gs)
                batches[k].dc_solve([rhss[i] for i in g], [xs[i] for i in g], 1.0, MU, max_iter=MAX_ITER,
                                    rel_tol=TOL, stream=gs)
            on_group_streams(grp)
            return
        for i in range(B):
            hq.adjoint_axpy(plans[i], yy[i], MU, zs[i], rhss[i])
        solve_all(mode_)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        return max_over_ranks(ms, dist)

    # iteration counts and residuals (untimed)
    for i in range(B):
        hq.adjoint_axpy(plans[i], ys[i], MU, zs[i], rhss[i])
    if args.mode == "batched":
        solve_all("batched")
        info = [t for bt in batches for t in bt.dc_info()]
        iters = [it for it, _, _ in info]
        assert all(st == 0 and rr <= TOL for _, rr, st in info)
    else:
        iters = []
        flag = hq.HQS_SOLVE_FUSED if args.mode == "fused" else hq.HQS_SOLVE_PLAIN
        for i in range(B):
            inf = hq.dc_solve(plans[i], 1.0, MU, rhss[i], xs[i], max_iter=MAX_ITER, rel_tol=TOL,
                              mode=flag | hq.HQS_SOLVE_X0_ZERO)
            iters.append(inf.iterations)
            assert inf.rel_residual <= TOL

    for _ in range(max(args.warmup, 3)):
        step()
    clk = ClockSampler(dev)
    clk.start()
    ms = timed(step, args.steps)
    clocks = clk.stop()
    value = whole_job_rate(B * args.steps, world, ms)

    # the dominant kernel, timed alone on the launching stream: the batched solve
    # (one launch for all B slices) or the persistent solve (one launch per slice)
    for i in range(B):
        hq.adjoint_axpy(plans[i], ys[i], MU, zs[i], rhss[i])
    torch.cuda.synchronize()
    e_solve = []
    for rep in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solve_all(args.mode if args.mode != "plain" else "fused")
        e1.record(stream)
        e_solve.append((e0, e1))
    torch.cuda.synchronize()
    launch_ms = float(np.mean([a.elapsed_time(b) for a, b in e_solve[1:]]))
    # the unit of the roofline: the concurrent batched launches of all groups together,
    # else one launch
    concurrent = args.mode == "batched" and len(gstreams) > 1
    if args.mode == "batched":
        solves_per_launch = B if concurrent else len(groups[0])
        solve_ms = launch_ms if concurrent else launch_ms / len(groups)
    else:
        solves_per_launch = 1
        solve_ms = launch_ms / B
    mean_iters = float(np.mean(iters))

    # plain PCG (per-stage launches, host-checked residual) and A^H A applies/s
    ms_plain = timed(lambda: step("plain"), max(1, args.steps // 2))
    plain_value = B * max(1, args.steps // 2) * world / (ms_plain / 1e3)
    outs = [torch.empty_like(x) for x in xs]
    reps = 10

    def applies():
        for i in range(B):
            hq.toeplitz_normal(plans[i], zs[i], outs[i])
    for _ in range(3):
        applies()
    ms_aha = timed(applies, reps)
    aha_per_s = B * reps * world / (ms_aha / 1e3)
    # the same applies batched: one launch of hqs_batch_toeplitz_normal per slice group
    aha_batched_per_s = None
    if batches:
        def applies_batched():
            on_group_streams(lambda k, gs: batches[k].toeplitz_normal(
                [zs[i] for i in groups[k]], [outs[i] for i in groups[k]], stream=gs))
        for _ in range(3):
            applies_batched()
        ms_ahab = timed(applies_batched, reps)
        aha_batched_per_s = B * reps * world / (ms_ahab / 1e3)

    # forward A and adjoint A^H of the NUFFT (each slice its own plan and data)
    xs_img = [torch.from_numpy(s["x"].astype(np.complex64)).cuda() for s in sl]
    ys_out = [torch.empty_like(y) for y in ys]

    def forwards():
        for i in range(B):
            hq.forward(plans[i], xs_img[i], ys_out[i])

    def adjoints():
        for i in range(B):
            hq.adjoint(plans[i], ys[i], outs[i])
    forwards()
    adjoints()
    ms_fwd = timed(forwards, reps)
    ms_adj = timed(adjoints, reps)
    fwd_per_s = B * reps * world / (ms_fwd / 1e3)
    adj_per_s = B * reps * world / (ms_adj / 1e3)
    # the same operators batched (hqs_batch_forward / hqs_batch_adjoint_axpy per group)
    fwd_batched_per_s = adj_batched_per_s = None
    if batches:
        def forwards_b():
            on_group_streams(lambda k, gs: batches[k].forward(
                [xs_img[i] for i in groups[k]], [ys_out[i] for i in groups[k]], stream=gs))

        def adjoints_b():
            on_group_streams(lambda k, gs: batches[k].adjoint_axpy(
                [ys[i] for i in groups[k]], 0.0, None, [outs[i] for i in groups[k]], stream=gs))
        forwards_b()
        adjoints_b()
        fwd_batched_per_s = B * reps * world / (timed(forwards_b, reps) / 1e3)
        adj_batched_per_s = B * reps * world / (timed(adjoints_b, reps) / 1e3)
    # the solutions themselves, not only the CG recursion: true relative residual
    # ||rhs - (A^H A + mu I) x|| / ||rhs|| of every slice with the library's operator
    for i in range(B):
        hq.adjoint_axpy(plans[i], ys[i], MU, zs[i], rhss[i])
    solve_all(args.mode)
    true_res = []
    for i in range(B):
        hq.toeplitz_normal(plans[i], xs[i], outs[i])
        r = rhss[i] - (outs[i] + MU * xs[i])
        true_res.append(float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(rhss[i])))
    assert max(true_res) <= 1.5 * TOL, max(true_res)

    # the precision variant (BF16x3 / FP16x3 tensor-core Toeplitz passes): A^H A
    # time, per-stage DC solves to 1e-4 and their distance to the FP32 solutions
    mixed = mixed_precision_summary(hq, plans[:4], rhss[:4], xs[:4], timed)
    # the learned preconditioner on this workload's shapes, compact (outside the
    # timed regions): 2 training seeds x 16 iterates, 200 Adam steps, 2 held-out seeds
    learned = learned_summary(hq, range(1000, 1002), range(5000, 5002), steps=200)
    learned = {k: v for k, v in learned.items() if k != "held_out"}
    # the uneven batch (64 slices of 256^2-384^2, annealed HQS 20 x 5 in one
    # graph-replayed persistent launch), compact: 2 timed steps, outside the timed region
    batch64, _, _, _ = batch64_summary(hq, 2, 3, rank, world, dist)

    # end to end through the public API with host buffers: H2D of y, D2H of x
    y_host = [y.cpu().pin_memory() for y in ys]
    x_host = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in xs]
    y_dev = [torch.empty_like(y) for y in ys]

    def e2e_step():
        for i in range(B):
            y_dev[i].copy_(y_host[i], non_blocking=True)
        step(ys_=y_dev)
        for i in range(B):
            x_host[i].copy_(xs[i], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_step()
    ms_e2e = timed(e2e_step, max(1, args.steps // 2))
    e2e_value = B * max(1, args.steps // 2) * world / (ms_e2e / 1e3)
    h2d = sum(int(y.numel()) * 8 for y in ys)
    d2h = sum(int(x.numel()) * 8 for x in xs)

    phases = None
    if args.phase_trace and args.mode == "batched":
        phases = batch_phase_trace(batches[0], [rhss[i] for i in groups[0]], [xs[i] for i in groups[0]], hq)
    if rank != 0:
        return
    # roofline of the dominant kernel (the batched or persistent solve): its
    # algorithmic FP32 work per launch / duration against the ALU peak of the unit
    # counts at the maximum SM clock; beside it the same launch's compulsory bytes
    # against the measured HBM bandwidth
    flops_iter = aha_flops(n, L) + precond_flops(n) + 12 * 8 * n * n
    flops_launch = flops_iter * mean_iters * solves_per_launch
    achieved = flops_launch / (solve_ms / 1e3) / 1e12
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = fp32_peak_tflops(sm_max)
    bytes_launch = iter_bytes(n, L) * mean_iters * solves_per_launch
    hbm_achieved = bytes_launch / (solve_ms / 1e3) / 1e9
    step0 = OracleStep()
    cpu_t, cpu_iters = step0()
    cpu_value = 1.0 / cpu_t
    # per step the adjoint with the axpy: batched, per slice the reorder of y and the
    # spreading, per group one column-IFFT and one row-IFFT + axpy launch (16 coils,
    # one chunk); per slice otherwise (4 launches each).  Then the solve: one batched
    # launch per group, one persistent launch per slice, or the plain path's 8 set-up
    # launches and 10 per CG iteration (3 A^H A passes, 3 preconditioner passes, the
    # update and 3 scalar kernels)
    if args.mode == "batched":
        launches_per_step = 2 * B + 2 * len(groups) + len(groups)
    elif args.mode == "fused":
        launches_per_step = 4 * B + B
    else:
        launches_per_step = 4 * B + sum(8 + 10 * it for it in iters)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantoms, Gaussian-bump coil maps, VD spiral)",
        "config": {"workload": WORKLOAD,
                   "batch_per_gpu": B, "solver": args.mode,
                   "slices_per_launch": len(groups[0]) if args.mode == "batched" else 1,
                   "concurrent_launches": len(gstreams) if args.mode == "batched" else 1,
                   "parallelism": f"replicas x{world}",
                   "tuning": {"spread_tile": tuned.spread_tile, "pc_lines": tuned.pc_lines,
                              "fused_grid": tuned.fused_grid},
                   "l2": "inputs larger than L2 (batch of distinct slices), no flush"},
        "aha_applies_per_s": aha_per_s,
        "aha_applies_per_s_batched": aha_batched_per_s,
        "forward_per_s": fwd_per_s,
        "adjoint_per_s": adj_per_s,
        "forward_per_s_batched": fwd_batched_per_s,
        "adjoint_per_s_batched": adj_batched_per_s,
        "nufft_hbm": {"unit": "GB/s", "peak": HBM_PEAK_GBS,
                      "forward": FWD_BYTES * fwd_per_s / world / 1e9,
                      "adjoint": ADJ_BYTES * adj_per_s / world / 1e9,
                      "bytes": "per operator, algorithmic bytes of the multi-pass design (x or y, S, the "
                               "oversampled grid written and read per pass, points)"},
        "plain_pcg_solves_per_s": plain_value,
        "speedup_vs_plain_pcg": value / plain_value,
        "mean_cg_iterations": mean_iters,
        "true_rel_residual_max": max(true_res),
        "mixed_precision": mixed,
        "learned_precond": learned,
        "batch64_hqs": batch64,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": BATCH_TRAFFIC_BYTES if args.mode == "batched" else PERSISTENT_TRAFFIC_BYTES,
                     "kernel": ((f"k_pcg_batch ({len(groups)} concurrent launches of {len(groups[0])} slices, "
                                 f"each on {2 * torch.cuda.get_device_properties(dev).multi_processor_count // len(groups)} CTAs)"
                                 if concurrent else f"k_pcg_batch ({len(groups[0])} slices per launch)")
                                if args.mode == "batched" else "k_pcg_persistent<640,320>"),
                     "flops_per_launch": flops_launch, "launch_ms": solve_ms,
                     "peak_source": f"unit counts: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                                    f"(maximum SM clock)",
                     "hbm": {"achieved": hbm_achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                             "frac": hbm_achieved / HBM_PEAK_GBS, "bytes_per_launch": bytes_launch,
                             "bytes": "compulsory per slice-iteration: x, S, Khat and the output of A^H A "
                                      "plus 8 vector passes", "peak_source": PEAKS["source"]}},
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
                         "sample": f"one FP64 oracle step of slice 0 (gridding adjoint for A^H y + mu z, "
                                   f"DC-preconditioned CG to 1e-4 in {cpu_iters} iterations), measured; "
                                   f"oracle plan {step0.t_plan:.1f} s once, untimed"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if phases is not None:
        line["phase_trace_us"] = phases
    print(json.dumps(line), flush=True)


BATCH_PHASES = ["p_update", "rows_fwd", "cols", "rows_adj", "epilogue", "update_pc_rows", "pc_cols_rz"]


def batch_phase_trace(bt, rhs, xs, hq):
    """One batched solve with the kernel's phase trace armed (outside the timed
    region): mean microseconds per CG iteration of each phase between grid
    barriers, over all iterations of the launch, plus the set-up phases."""
    for x in xs:
        x.zero_()
    bt.debug_trace(True)
    bt.dc_solve(rhs, xs, 1.0, MU, max_iter=MAX_ITER, rel_tol=TOL)
    st = bt.debug_trace(False)
    its = [it for it, _, _ in bt.dc_info()]
    d = np.diff(np.array(st, dtype=np.float64)) / 1e3
    body = d[3:-1]
    nit = int(math.ceil(len(body) / 7))
    out = {"setup": [round(float(v), 1) for v in d[:3]], "iterations": nit}
    for k, name in enumerate(BATCH_PHASES):
        v = body[k::7]
        if len(v):
            out[name] = round(float(np.mean(v)), 1)
    out["total_ms"] = round(float((st[-1] - st[0]) / 1e6), 3)
    # per batched iteration: its time and the number of slices still iterating
    out["per_iteration_us"] = [round(float(np.sum(body[7 * k:7 * k + 7])), 1) for k in range(nit)]
    out["active_slices"] = [sum(1 for i in its if i > k) for k in range(nit)]
    out["slice_iterations"] = its
    return out


def make_batch64(rank=0, count=64):
    import synth
    rng = np.random.default_rng(4242 + rank)
    out = []
    for i in range(count):
        n = int(rng.choice([256, 320, 384]))
        L = int(rng.integers(8, 21))
        if rng.random() < 0.5:
            spokes = int(rng.integers(48, 97))
            traj = synth.traj_radial(spokes, 2 * n)
            kind = f"radial {spokes}x{2 * n}"
        else:
            il, ns = int(rng.integers(12, 25)), int(rng.integers(1024, 4097))
            traj = synth.traj_spiral(il, ns, n)
            kind = f"spiral {il}x{ns}"
        seed = 7000 + 100 * rank + i
        out.append(dict(n=n, L=L, traj=traj, kind=kind, x=synth.phantom(seed, n),
                        smaps=synth.coil_maps(seed, n, L),
                        noise=synth.complex_noise(seed, (L, traj.shape[0]))))
    return out


def batch64_summary(hq, steps, warmup, rank, world, dist, count=64):
    """The uneven-batch workload (64 slices, n in {256, 320, 384}, 8-20 coils,
    radial or spiral, annealed HQS 20 x 5 in one graph-replayed persistent
    launch): slices/s, per-step latency and the same work slice by slice through
    hqs_run.  Returns (summary dict, clocks, timed ms, slices)."""
    import torch
    from paper_2411_01955_gb300 import tune
    import synth

    K, CG = 20, 5
    mu = synth.mu_schedule_geometric(1e-1, 1e-3, K).astype(np.float32)
    sigma = mu.copy()
    sl = make_batch64(rank, count)
    plans, ys, xs = [], [], []
    tuned = {}
    for s in sl:
        n, L = s["n"], s["L"]
        plan = hq.plan_create(torch.from_numpy(s["traj"]).cuda(), n, n,
                              torch.from_numpy(s["smaps"].astype(np.complex64)).cuda(), 6, 2.0)
        t = tune.autotune(plan, solve_shapes=False)
        tuned[t.spread_tile] = tuned.get(t.spread_tile, 0) + 1
        x = torch.from_numpy(s["x"].astype(np.complex64)).cuda()
        y = torch.empty((L, s["traj"].shape[0]), dtype=torch.complex64, device="cuda")
        hq.forward(plan, x, y)
        sd = math.sqrt(1e-4 * float(np.max(np.sum(np.abs(s["smaps"] * s["x"]) ** 2, axis=0))))
        y = (y + sd * torch.from_numpy(s["noise"].astype(np.complex64)).cuda()).contiguous()
        plans.append(plan)
        ys.append(y)
        xs.append(torch.zeros_like(x))
    batch = hq.Batch(plans, max_outer=K)
    stream = torch.cuda.current_stream()

    def step():
        for x in xs:
            x.zero_()
        batch.run(ys, xs, mu, sigma, cg_iters=CG, use_graph=True)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps_):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps_):
            fn()
        e1.record(stream)
        barrier()
        ms_ = e0.elapsed_time(e1)
        return max_over_ranks(ms_, dist)

    for _ in range(max(warmup, 3)):
        step()
    res = batch.status()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    ms = timed(step, steps)
    clocks = clk.stop()
    # per-step latency (every slice of a step finishes with the step's one launch)
    lat = []
    for _ in range(max(steps, 5)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))

    def per_slice():
        for i, p in enumerate(plans):
            xs[i].zero_()
            hq.hqs_run(p, ys[i], xs[i], mu, sigma, cg_iters=CG)
    batch.close()
    per_slice()
    ms_seq = timed(per_slice, 1)
    summary = {
        "slices_per_s": whole_job_rate(len(sl) * steps, world, ms),
        "batch_latency_ms": ms / steps,
        "slice_latency_ms_p50_p95": [float(np.percentile(lat, 50)), float(np.percentile(lat, 95))],
        "per_slice_hqs_run_slices_per_s": len(sl) * world / (ms_seq / 1e3),
        "speedup_vs_per_slice": (ms_seq) / (ms / steps),
        "max_final_rel_residual_sq": float(max(res)),
        "sizes": {str(k): sum(1 for s in sl if s["n"] == k) for k in (256, 320, 384)},
        "points": int(sum(s["traj"].shape[0] for s in sl)),
        "coils": int(sum(s["L"] for s in sl)),
        "spread_tiles_picked": {str(k): v for k, v in sorted(tuned.items())},
        "launches_per_step": sum(4 + (1 if p.info().coils > 16 else 0) for p in plans) + 1,
    }
    for p in plans:
        p.close()
    return summary, clocks, ms, sl


def run_batch64(args, rank, world, dist):
    import torch
    import paper_2411_01955_gb300 as hq

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    summ, clocks, ms, sl = batch64_summary(hq, args.steps, args.warmup, rank, world, dist)
    if rank != 0:
        return
    line = {
        "metric": "batched annealed HQS slices/s (64 uneven slices, 20 x 5 CG)", "value": summ["slices_per_s"],
        "unit": "slices/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantoms, Gaussian-bump coil maps, radial/spiral)",
        "config": {"workload": "64 slices, n in {256,320,384}, 8-20 coils, radial 48-96 spokes x 2n or "
                               "spiral 12-24 x 1024-4096, KB W=6, sigma=2, HQS 20 outer x 5 CG, "
                               "mu 1e-1 -> 1e-3, Gaussian denoiser; one graph-replayed persistent launch",
                   "sizes": summ["sizes"], "points": summ["points"], "coils": summ["coils"],
                   "spread_tiles_picked": summ["spread_tiles_picked"],
                   "l2": "inputs larger than L2 (64 distinct slices), no flush"},
        "batch_latency_ms": summ["batch_latency_ms"],
        "slice_latency_ms_p50_p95": summ["slice_latency_ms_p50_p95"],
        "per_slice_hqs_run_slices_per_s": summ["per_slice_hqs_run_slices_per_s"],
        "speedup_vs_per_slice": summ["speedup_vs_per_slice"],
        "max_final_rel_residual_sq": summ["max_final_rel_residual_sq"],
        # per step: each slice's adjoint (reorder, spreading, column and row passes, and
        # the chunk sum where a slice has several coil chunks, replayed from the graph),
        # then the persistent launch
        "gpu_launches": summ["launches_per_step"] * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_mixed320(args, rank, world, dist):
    """A^H A applies/s and DC solves/s (plain PCG, DC preconditioner, 1e-4) of
    the 320^2 x 16-coil workload with the Toeplitz passes in FP32 (in-house
    FFTs) and as BF16x3 / FP16x3 tensor-core DFT-GEMMs."""
    import torch
    import paper_2411_01955_gb300 as hq

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    B = args.batch
    n, L, traj_np, sl = make_slices(B, rank)
    traj = torch.from_numpy(traj_np).cuda()
    plans, rhss, xs = [], [], []
    for s in sl:
        plan = hq.plan_create(traj, n, n, torch.from_numpy(s["smaps"].astype(np.complex64)).cuda(), 6, 2.0)
        x = torch.from_numpy(s["x"].astype(np.complex64)).cuda()
        y = torch.empty((L, traj.shape[0]), dtype=torch.complex64, device="cuda")
        hq.forward(plan, x, y)
        rhs = torch.empty_like(x)
        hq.adjoint(plan, y, rhs)
        plans.append(plan)
        rhss.append(rhs)
        xs.append(torch.zeros_like(x))
    stream = torch.cuda.current_stream()
    outs = [torch.empty_like(x) for x in xs]

    def timed(fn, steps):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return max_over_ranks(ms, dist)

    res = {}
    clk = ClockSampler(dev)
    clk.start()
    for name, prec in (("fp32", hq.HQS_PREC_FP32), ("bf16x3", hq.HQS_PREC_BF16X3), ("fp16x3", hq.HQS_PREC_FP16X3)):
        def applies():
            for i in range(B):
                hq.toeplitz_normal(plans[i], rhss[i], outs[i], precision=prec)

        def solves():
            for i in range(B):
                hq.dc_solve(plans[i], 1.0, MU, rhss[i], xs[i], max_iter=MAX_ITER, rel_tol=TOL, precision=prec,
                            mode=hq.HQS_SOLVE_X0_ZERO, want_info=False)
        iters = [hq.dc_solve(plans[i], 1.0, MU, rhss[i], xs[i], max_iter=MAX_ITER, rel_tol=TOL, precision=prec,
                             mode=hq.HQS_SOLVE_X0_ZERO).iterations for i in range(B)]
        for _ in range(max(args.warmup, 3)):
            applies()
        ms_a = timed(applies, args.steps)
        solves()
        ms_s = timed(solves, max(1, args.steps // 2))
        res[name] = {"aha_applies_per_s": B * args.steps * world / (ms_a / 1e3),
                     "aha_us": ms_a * 1e3 / (B * args.steps),
                     "dc_solves_per_s": B * max(1, args.steps // 2) * world / (ms_s / 1e3),
                     "mean_cg_iterations": float(np.mean(iters))}
    clocks = clk.stop()
    if rank != 0:
        return
    # tensor-pipe work of one mixed A^H A: 4 real GEMMs x 3 products
    gemm_flops = 3 * 2 * (L * n * 4 * n * 2 * n + L * 2 * n * 4 * n * 2 * n + L * 2 * n * 2 * n * 4 * n
                          + n * L * 2 * n * 4 * n)
    peak = PEAKS["bf16_tflops"]
    for name in ("bf16x3", "fp16x3"):
        res[name]["tensor_tflops"] = gemm_flops / (res[name]["aha_us"] * 1e-6) / 1e12
        res[name]["tensor_frac_of_measured_bf16_peak"] = res[name]["tensor_tflops"] / peak
    line = {
        "metric": "A^H A applies/s and DC solves/s at 320^2, 16 coils: FP32 vs BF16x3 / FP16x3 DFT-GEMM",
        "value": res["bf16x3"]["dc_solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3", "data": "synthetic (seeded ellipse phantoms, Gaussian-bump coil maps, VD spiral)",
        "config": {"workload": "320x320, 16 coils, spiral 16x2048, KB W=6, sigma=2, mu=1e-2, rel. residual 1e-4, "
                               "plain PCG with DC preconditioner",
                   "batch_per_gpu": B, "l2": "inputs larger than L2 (batch of distinct slices), no flush"},
        "precisions": res, "gemm_flops_per_aha": gemm_flops,
        "gpu_launches_per_mixed_aha": 6, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_mixed_sizes(args, rank, world, dist):
    """A^H A microseconds per apply with the Toeplitz passes as FP32 in-house
    FFTs and as BF16x3 / FP16x3 tensor-core DFT-GEMMs, over the image sizes
    the DFT-GEMM path supports (n a multiple of 64, <= 384), 16 coils, a
    variable-density spiral scaled with n; CUDA events over 50 applies."""
    import torch
    import paper_2411_01955_gb300 as hq
    import synth
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    L = 16
    rows = {}
    clk = ClockSampler(dev)
    clk.start()
    for n in (64, 128, 256, 320, 384):
        traj = torch.from_numpy(synth.traj_spiral(16, max(256, int(2048 * n / 320)), n)).cuda()
        smaps = torch.from_numpy(synth.coil_maps(0, n, L).astype(np.complex64)).cuda()
        plan = hq.plan_create(traj, n, n, smaps, 6, 2.0)
        x = torch.from_numpy(synth.phantom(0, n).astype(np.complex64)).cuda()
        y = torch.empty_like(x)
        row = {}
        for name, prec in (("fp32", hq.HQS_PREC_FP32), ("bf16x3", hq.HQS_PREC_BF16X3), ("fp16x3", hq.HQS_PREC_FP16X3)):
            for _ in range(max(args.warmup, 3)):
                hq.toeplitz_normal(plan, x, y, precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(50):
                hq.toeplitz_normal(plan, x, y, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            row[name] = e0.elapsed_time(e1) * 1e3 / 50
        rows[n] = row
        plan.close()
    clocks = clk.stop()
    if rank != 0:
        return
    line = {"metric": "A^H A microseconds per apply: FP32 in-house FFTs vs BF16x3 / FP16x3 DFT-GEMMs, 16 coils",
            "value": rows[320]["bf16x3"] / rows[320]["fp32"], "unit": "BF16x3 / FP32 time at 320^2",
            "n_gpus": world, "higher_is_better": False, "data": "synthetic (seeded phantoms, coil maps, VD spiral)",
            "config": {"workload": "image sizes 64-384, 16 coils, spiral 16 interleaves scaled with n, W 6, sigma 2"},
            "aha_us": {str(k): v for k, v in rows.items()}, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_hqs320(args, rank, world, dist):
    """Annealed PnP-HQS on the 320^2 x 16-coil workload (10 outer steps x 5 CG
    iterations, mu 1e-1 -> 1e-3, Gaussian smoothing denoiser) in the metric
    P = c0 I + c1 A^H A: Id (1, 0), F-1 (2, -alpha), Chebyshev (4, -10 alpha / 3),
    alpha = 1 / ||A^H A|| by power iteration; HQS runs per second."""
    import torch
    import paper_2411_01955_gb300 as hq
    import synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    B = args.batch
    n, L, traj_np, sl = make_slices(B, rank)
    traj = torch.from_numpy(traj_np).cuda()
    K, CG = 10, 5
    mu = synth.mu_schedule_geometric(1e-1, 1e-3, K).astype(np.float32)
    plans, ys, xs = [], [], []
    for s in sl:
        plan = hq.plan_create(traj, n, n, torch.from_numpy(s["smaps"].astype(np.complex64)).cuda(), 6, 2.0)
        x = torch.from_numpy(s["x"].astype(np.complex64)).cuda()
        y = torch.empty((L, traj.shape[0]), dtype=torch.complex64, device="cuda")
        hq.forward(plan, x, y)
        sd = math.sqrt(1e-4 * float(np.max(np.sum(np.abs(s["smaps"] * s["x"]) ** 2, axis=0))))
        y = (y + sd * torch.from_numpy(s["noise"].astype(np.complex64)).cuda()).contiguous()
        plans.append(plan)
        ys.append(y)
        xs.append(torch.zeros_like(x))
    alpha = 1.0 / hq.power_iteration(plans[0], 50)
    metrics = {"id": (1.0, 0.0), "f1": (2.0, -alpha), "chebyshev": (4.0, -10.0 * alpha / 3.0)}
    stream = torch.cuda.current_stream()
    res = {}
    clk = ClockSampler(dev)
    clk.start()
    for name, (c0, c1) in metrics.items():
        def runs():
            for i in range(B):
                xs[i].zero_()
                hq.hqs_run(plans[i], ys[i], xs[i], mu, mu, cg_iters=CG, c0=c0, c1=c1)
        for _ in range(max(args.warmup, 3)):
            runs()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            runs()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist)
        res[name] = {"hqs_runs_per_s": whole_job_rate(B * args.steps, world, ms),
                     "ms_per_run": ms / (B * args.steps), "c0": c0, "c1": c1}
    # PnP-PGD, 10 steps, gamma = 0.9 / (c0 ||A^H A||), same metrics
    gam_base = 0.9 * alpha
    for name, (c0, c1) in metrics.items():
        gam = np.full(K, gam_base / c0, dtype=np.float32)
        sg = np.full(K, 0.5, dtype=np.float32)

        def pruns():
            for i in range(B):
                xs[i].zero_()
                hq.pgd_run(plans[i], ys[i], xs[i], gam, sg, c0=c0, c1=c1)
        for _ in range(max(args.warmup, 3)):
            pruns()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pruns()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist)
        res["pgd_" + name] = {"pgd_runs_per_s": whole_job_rate(B * args.steps, world, ms),
                              "ms_per_run": ms / (B * args.steps), "c0": c0, "c1": c1}
    # the two other pieces of a reconstruction run here: S-map estimation from the
    # 20 x 20 Hamming-windowed k-space centre (once per scan) and the GPU conv denoiser
    # D_sigma (once per outer step in place of the Gaussian smoothing)
    learned = tests_module("learned_training")
    smaps_out = torch.empty((L, n, n), dtype=torch.complex64, device="cuda")
    net = hq.Net()
    net.set_params(learned.initial_params(0))
    den_out = torch.empty_like(xs[0])

    def timed_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist) / reps
    smaps_ms = timed_ms(lambda: hq.estimate_smaps(traj, ys[0], n, smaps_out), max(args.steps, 3))
    # the network's 32 -> 32 layers on the tensor cores (the default) and on the FP32 cores
    denoise_ms = timed_ms(lambda: net.denoise(xs[0], den_out, 0.05), 10 * max(args.steps, 3))
    net.set_precision(hq.HQS_PREC_FP32)
    denoise_fp32_ms = timed_ms(lambda: net.denoise(xs[0], den_out, 0.05), 10 * max(args.steps, 3))
    net.set_precision(hq.HQS_PREC_BF16X3)
    net.status()
    clocks = clk.stop()
    if rank != 0:
        return
    line = {
        "metric": "annealed PnP-HQS runs/s at 320^2, 16 coils (10 outer x 5 CG), Id / F-1 / Chebyshev metrics",
        "value": res["id"]["hqs_runs_per_s"], "unit": "HQS runs/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded ellipse phantoms, Gaussian-bump coil maps, VD spiral)",
        "config": {"workload": "320x320, 16 coils, spiral 16x2048, KB W=6, sigma=2, HQS 10 x 5 CG, "
                               "mu 1e-1 -> 1e-3, Gaussian smoothing denoiser, DC-preconditioned CG",
                   "batch_per_gpu": B, "alpha": alpha},
        "metrics": res, "clocks": clocks,
        "smaps_estimation_ms": smaps_ms, "conv_denoiser_ms": denoise_ms, "conv_denoiser_fp32_layers_ms": denoise_fp32_ms,
    }
    print(json.dumps(line), flush=True)


def learned_summary(hq, train_seeds, held_seeds, steps, iterates=16):
    """Learned preconditioner at 320^2 x 16 coils: the network is trained on the
    GPU (library kernels; its 32 -> 32 layers on the tensor cores) on DC-PCG
    iterates of training seeds 1000+ (mu log-uniform in [1e-3, 1e-1]), then
    flexible CG with it and DC-PCG solve held-out seeds 5000+ to relative
    residual 1e-4: iterations, solve time, fallback counts."""
    import time as _time
    import torch
    learned = tests_module("learned_training")
    import synth

    n, L = 320, 16
    traj_np = synth.traj_spiral(16, 2048, n)
    traj = torch.from_numpy(traj_np).cuda()
    rng = np.random.default_rng(77)

    def slice_(seed):
        plan = hq.plan_create(traj, n, n, torch.from_numpy(synth.coil_maps(seed, n, L).astype(np.complex64)).cuda(),
                              6, 2.0)
        x = torch.from_numpy(synth.phantom(seed, n).astype(np.complex64)).cuda()
        y = torch.empty((L, traj.shape[0]), dtype=torch.complex64, device="cuda")
        hq.forward(plan, x, y)
        rhs = torch.empty_like(x)
        hq.adjoint(plan, y, rhs)
        return plan, rhs
    t0 = _time.time()
    examples = []
    for seed in train_seeds:
        plan, rhs = slice_(seed)
        mu = float(10 ** rng.uniform(-3, -1))
        for r, e in learned.solve_pairs(plan, rhs, mu, iterates=iterates):
            examples.append(learned.network_example(plan, mu, r, e))
    net = hq.Net()
    net.set_params(learned.initial_params(0))   # zero last layer: the untrained network is DC-PCG
    losses = learned.train(net, examples, steps=steps, batch=16, crop=64, lr=1e-3)
    torch.cuda.synchronize()
    train_s = _time.time() - t0
    rows = []
    for seed in held_seeds:
        plan, rhs = slice_(seed)
        mu = float(10 ** rng.uniform(-3, -1))
        out = {}
        for name, pc in (("dc", hq.HQS_PRECOND_DC), ("learned", hq.HQS_PRECOND_LEARNED)):
            hq.plan_set_net(plan, net if name == "learned" else None)
            x = torch.zeros_like(rhs)
            hq.dc_solve(plan, 1.0, mu, rhs, x, max_iter=400, rel_tol=1e-4, precond=pc)   # warm-up
            x.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            info = hq.dc_solve(plan, 1.0, mu, rhs, x, max_iter=400, rel_tol=1e-4, precond=pc)
            e1.record()
            torch.cuda.synchronize()
            out[name] = {"iterations": info.iterations, "ms": e0.elapsed_time(e1), "fallback": info.fallback,
                         "rel_residual": info.rel_residual}
        hq.plan_set_net(plan, None)
        rows.append({"seed": seed, "mu": mu, **out})
    net.status()
    return {
        "learned_iterations": float(np.mean([r["learned"]["iterations"] for r in rows])),
        "dc_iterations": float(np.mean([r["dc"]["iterations"] for r in rows])),
        "learned_solves_per_s": 1e3 / float(np.mean([r["learned"]["ms"] for r in rows])),
        "dc_solves_per_s": 1e3 / float(np.mean([r["dc"]["ms"] for r in rows])),
        "learned_fallbacks": int(sum(r["learned"]["fallback"] for r in rows)),
        "train_pairs": len(examples), "train_steps": steps, "train_seconds": train_s,
        "train_loss_first_last": [losses[0], float(np.mean(losses[-20:]))],
        "held_out": rows,
    }


def run_learned320(args, rank, world, dist):
    """The learned-preconditioner summary at full size: args.batch training
    seeds x 16 DC-PCG iterates, 400 Adam steps on 64 x 64 crops, 4 held-out
    seeds."""
    import torch
    import paper_2411_01955_gb300 as hq

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    res = learned_summary(hq, range(1000, 1000 + args.batch), range(5000, 5004), steps=400)
    if rank != 0:
        return
    line = {
        "metric": "DC solves to 1e-4 at 320^2, 16 coils: learned-preconditioned flexible CG vs DC-PCG",
        "value": res["learned_iterations"], "unit": "CG iterations (mean)",
        "n_gpus": world, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded ellipse phantoms, Gaussian-bump coil maps, VD spiral)",
        "config": {"workload": "320x320, 16 coils, spiral 16x2048, KB W=6, sigma=2, mu log-uniform [1e-3, 1e-1]; "
                               f"training: {args.batch} seeds x 16 DC-PCG iterates, 400 Adam steps on 64x64 crops",
                   "train_pairs": res["train_pairs"]},
        "dc_mean_iterations": res["dc_iterations"],
        **{k: v for k, v in res.items() if k not in ("learned_iterations", "dc_iterations", "train_pairs")},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) of the launches of one 64^3 x 16-coil A^H A, from one ncu capture of
# the current kernels (None until re-measured after a change)
VOL_AHA_TRAFFIC_BYTES = 480437760 + 181145600


def vol_pass_bytes(shape, L):
    """Bytes the launches of one 3D Toeplitz A^H A move by their pass
    structure (each FFT pass reads its input lines and writes its output):
    with U = Nvox L 8 bytes, x-FFT 1U (maps) + 2U, y-FFT 2U + 4U, z-FFT with
    Khat 4U + 4U, inverse y 4U + 2U, inverse x 2U + 1U (maps); then, with the
    coil sum fused into the inverse x pass (L divides 16), nothing more, else
    1U written and read back by the separate coil sum; plus x and out (8 Nvox
    each) and Khat (32 Nvox)."""
    nvox = shape[0] * shape[1] * shape[2]
    U = nvox * L * 8
    return (26 if 16 % L == 0 else 28) * U + 16 * nvox + 32 * nvox


def run_vol64(args, rank, world, dist):
    """Volumetric operator at 64^3 (vol64: stack of 64 VD spirals, 8 x 1024
    samples each) or 128^3 (vol128: 128 spirals of 16 x 1024), 16 coils:
    forward / adjoint / Toeplitz A^H A per call, DC solves (PCG, mu 1e-2,
    1e-4) per second and one annealed HQS run; every rank runs its own volume."""
    import torch
    import paper_2411_01955_gb300 as hq
    import synth

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    big = args.workload == "vol128"
    nv = 128 if big else 64
    shape, L = (nv, nv, nv), 16
    case = synth.volume_case(rank, shape, L, 16 if big else 8, 1024)
    traj = torch.from_numpy(case["traj"]).cuda()
    smaps = torch.from_numpy(case["smaps"].astype(np.complex64)).cuda()
    plan = hq.plan3d_create(traj, shape, smaps, 6, 2.0)
    M = traj.shape[0]
    x = torch.from_numpy(case["x"].astype(np.complex64)).cuda()
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq.forward3d(plan, x, y)
    rhs = torch.empty_like(x)
    hq.adjoint3d(plan, y, rhs)
    out = torch.empty_like(x)
    xs = torch.zeros_like(x)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist)

    def solve(precond=hq.HQS_PRECOND_DC):
        xs.zero_()
        return hq.dc_solve3d(plan, 1.0, MU, rhs, xs, max_iter=MAX_ITER, rel_tol=TOL, precond=precond)

    W = max(args.warmup, 3)
    K = max(args.steps, 1)
    clk = ClockSampler(dev)
    clk.start()
    for _ in range(W):
        hq.forward3d(plan, x, y)
        hq.adjoint3d(plan, y, rhs)
        hq.toeplitz_normal3d(plan, rhs, out)
    ms_f = timed(lambda: hq.forward3d(plan, x, y), K)
    ms_a = timed(lambda: hq.adjoint3d(plan, y, rhs), K)
    ms_t = timed(lambda: hq.toeplitz_normal3d(plan, x, out), K)
    ms_pc = timed(lambda: hq.precond_apply3d(plan, 1.0, MU, rhs, out), K)
    plain = solve(hq.HQS_PRECOND_NONE)
    ms_plain = timed(lambda: solve(hq.HQS_PRECOND_NONE), max(1, K // 2))
    info = solve()
    ms_s = timed(solve, max(1, K // 2))
    # end to end: pinned host rhs in, solution out, inside the timed region
    h_rhs = rhs.cpu().pin_memory()
    h_x = torch.empty_like(h_rhs).pin_memory()

    def solve_e2e():
        rhs.copy_(h_rhs, non_blocking=True)
        solve()
        h_x.copy_(xs, non_blocking=True)
    ms_e = timed(solve_e2e, max(1, K // 2))
    # annealed HQS on the volume: 10 outer steps x 5 PCG iterations, mu 1e-1 -> 1e-3,
    # built-in Gaussian smoothing (A^H y, 10 DC steps, 10 denoiser calls per run)
    mu_h = np.geomspace(1e-1, 1e-3, 10).astype(np.float32)
    xh = torch.zeros_like(x)

    def hqs_run():
        xh.zero_()
        hq.hqs_run3d(plan, y, xh, mu_h, mu_h, cg_iters=5, gauss=(1.5, float(mu_h[0])))
    hqs_run()
    ms_h = timed(hqs_run, max(1, K // 5))
    clocks = clk.stop()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not big:
        t_cpu = cpu_oracle_vol_sample(case)
        cpu = {"value": 1.0 / (t_cpu * L), "unit": "A^H(A x) applies/s", "cores": threads_used(), "kind": "oracle",
               "sample": "one coil of one 64^3 gridding forward + adjoint (oracle nufft3d, W=6, 524288 points), "
                         f"{t_cpu:.1f} s, scaled to 16 coils; compare aha_applies_per_s"}
    nsol = max(1, K // 2)
    t_us = ms_t * 1e3 / K
    traffic = vol_pass_bytes(shape, L)
    achieved = traffic / (t_us * 1e-6) / 1e9
    npts = case["traj"].shape[0]
    line = {
        "metric": f"3D DC solves/s to 1e-4 at {nv}^3, 16 coils (PCG on the 2N^3 Toeplitz A^H A)",
        "value": nsol * world / (ms_s / 1e3), "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_s / nsol, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded ellipsoid phantom, Gaussian-bump coil maps, stack of VD spirals)",
        "config": {"workload": f"{nv}x{nv}x{nv}, 16 coils, stack of {nv} spirals x {16 if big else 8} x 1024 "
                               f"({npts} points), KB W=6, sigma=2, mu=1e-2, rel. residual 1e-4, PCG with the 3D "
                               "density preconditioner",
                   "l2": f"grids ({(2 * nv) ** 3 // 2 * L * 8 // 2 ** 20} MB per Toeplitz pass) larger than L2, "
                         "no flush"},
        "cg_iterations": info.iterations, "plain_cg_iterations": plain.iterations,
        "plain_cg_solves_per_s": max(1, K // 2) * world / (ms_plain / 1e3), "precond_us": ms_pc * 1e3 / K,
        "forward_us": ms_f * 1e3 / K, "adjoint_us": ms_a * 1e3 / K, "aha_us": t_us,
        "aha_applies_per_s": K * world / (ms_t / 1e3),
        "hqs_10x5_ms": ms_h / max(1, K // 5),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                     "frac": achieved / HBM_PEAK_GBS, "traffic": None if big else VOL_AHA_TRAFFIC_BYTES,
                     "kernel": "the five launches of one A^H A (pass-structure bytes, measured peak)"},
        "e2e": {"value": nsol * world / (ms_e / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": int(rhs.numel() * 8), "d2h_bytes_per_step": int(xs.numel() * 8)},
        # per solve: initial A^H A (5: coil sum fused at 16 coils) + init + scalar + preconditioner
        # step (5 + 3), then the 17-kernel iteration graph replayed in chunks of 4 (replays past
        # convergence return at once)
        "gpu_launches": nsol * (15 + 17 * 4 * math.ceil(info.iterations / 4)), "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def fft_flops(N):
    return 5.0 * N * math.log2(N)


def aha_flops(n, L):
    """Algorithmic FLOPs of one Toeplitz A^H A apply: per coil n row FFTs and
    2n column FFT pairs of size 2n, n inverse row FFTs (5 N log2 N each),
    plus the coil multiply/sum (8 flops per pixel per coil each way) and Khat."""
    N2 = 2 * n
    ffts = L * (n + 2 * N2 + n) * fft_flops(N2)
    return ffts + L * (2 * 8 * n * n + 2 * N2 * n)


def precond_flops(n):
    return 2 * 2 * n * fft_flops(n) + 6 * n * n


def iter_bytes(n, L):
    """Compulsory HBM bytes of one CG iteration of one slice: the A^H A apply's
    x, coil maps, Khat and output (complex64 images and maps, real Khat on the
    2n grid) and 8 passes over complex64 n x n vectors (p, q, x, r, z)."""
    img = n * n * 8
    return img + L * img + (2 * n) * (2 * n) * 4 + img + 8 * img


def mixed_precision_summary(hq, plans, rhss, xs_fp32, timed):
    """A^H A microseconds and per-stage DC solves to 1e-4 in BF16x3 and FP16x3
    (tensor-core DFT-GEMM Toeplitz passes, fp64 CG scalars) on a few slices,
    with each solution's relative distance to the FP32 path's solution."""
    import torch
    out = {}
    outs = [torch.empty_like(x) for x in xs_fp32]
    for name, prec in (("fp32", hq.HQS_PREC_FP32), ("bf16x3", hq.HQS_PREC_BF16X3), ("fp16x3", hq.HQS_PREC_FP16X3)):
        def applies():
            for p, r, o in zip(plans, rhss, outs):
                hq.toeplitz_normal(p, r, o, precision=prec)
        xs = [torch.zeros_like(x) for x in xs_fp32]

        def solves():
            for p, r, x in zip(plans, rhss, xs):
                hq.dc_solve(p, 1.0, MU, r, x, max_iter=MAX_ITER, rel_tol=TOL, precision=prec,
                            mode=hq.HQS_SOLVE_X0_ZERO, want_info=False)
        applies()
        reps = 5
        ms_a = timed(applies, reps)
        its = [hq.dc_solve(p, 1.0, MU, r, x, max_iter=MAX_ITER, rel_tol=TOL, precision=prec,
                           mode=hq.HQS_SOLVE_X0_ZERO).iterations for p, r, x in zip(plans, rhss, xs)]
        ms_s = timed(solves, 1)
        diff = max(float(torch.linalg.vector_norm(x - x0) / torch.linalg.vector_norm(x0))
                   for x, x0 in zip(xs, xs_fp32))
        out[name] = {"aha_us": ms_a * 1e3 / (reps * len(plans)),
                     "dc_solves_per_s": len(plans) / (ms_s / 1e3),
                     "mean_cg_iterations": float(np.mean(its)),
                     "rel_diff_vs_fp32_solution": diff}
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.gpus != world:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE is {world}; launch N > 1 with "
              f"python -m torch.distributed.run --nproc-per-node {args.gpus} bench.py --gpus {args.gpus}",
              file=sys.stderr)
        sys.exit(2)
    dist = None
    if world > 1:
        import torch.distributed as td
        backend = "gloo" if args.impl == "reference" else "nccl"
        td.init_process_group(backend)
        dist = td
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch64":
        run_batch64(args, rank, world, dist)
    elif args.workload == "mixed320":
        run_mixed320(args, rank, world, dist)
    elif args.workload == "mixedsizes":
        run_mixed_sizes(args, rank, world, dist)
    elif args.workload == "hqs320":
        run_hqs320(args, rank, world, dist)
    elif args.workload == "learned320":
        run_learned320(args, rank, world, dist)
    elif args.workload in ("vol64", "vol128"):
        run_vol64(args, rank, world, dist)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
