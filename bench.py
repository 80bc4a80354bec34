#!/usr/bin/env python
"""Throughput of the Vegas hot path on one B300 (or N independent replicas).

Workload (one "step"): the d=8 Lepage Gaussian (Eq. 1, a = 0.1, centres 1/2),
50 bins per dimension, uniform starting grid, damping alpha = 1.5:
10 adapting iterations of 1e7 samples (each followed by a grid refinement),
then 5 fixed-grid iterations of 1e8 samples -- 6e8 samples per step.  The
headline value is samples/s of the FP32-eval / FP64-accumulate path; the plain
FP64 path runs the same workload (same counters, hence equal error) and is
reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) the headline integral is sharded over the ranks: every
rank keeps the per-GPU sample counts (weak scaling), computes its range of
sample indices and the partial sums are all-reduced once per iteration; the
other legs run on each rank independently.  Rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Vegas samples/s, d=8 Gaussian: FP32-eval vs plain FP64 at equal error; % FP peak"
DIM, NBINS, A, ALPHA = 8, 50, 0.1, 1.5
N_ADAPT, IT_ADAPT, N_FIXED, IT_FIXED = 10_000_000, 10, 100_000_000, 5
SAMPLES_PER_STEP = N_ADAPT * IT_ADAPT + N_FIXED * IT_FIXED
WORKLOAD = "gauss_d8_a0.1_N50_10x1e7adapt+5x1e8fixed"
EXACT = math.erf(0.5 / A) ** DIM

# Issue-slot peak from unit counts and clock: 148 SMs x 4 schedulers x 32 lanes
# at the 2032 MHz maximum SM clock (lane-instructions per second).
SMS, LANES_PER_SM, SM_MAX_MHZ = 148, 128, 2032.0
ALU_PEAK_TOPS = SMS * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12

# DRAM bytes per launch of the fixed-grid FP32 iterate kernel (read 71.2 KB,
# write 0 per 1e8-sample launch; the kernel compiled for 50 bins) from an ncu
# capture of this kernel build.
ITERATE_TRAFFIC_BYTES = 71168


def products_per_sample(d):
    """32x32 -> 64-bit products of one sample: Philox rounds 0 and 1 shared by
    the sample's calls (2), rounds 2-9 of each call (16 per call), and the bin
    split of each dimension (1)."""
    return 2 + 16 * ((d + 3) // 4) + d


def pipe_fractions(V, fixed_ms, adapt_ms):
    """The measured peak of each pipe (vegas_pipe_peak, best of 3) and the
    share of it that the d=8 FP32 iterate kernels reach: the products (the
    binding pipe), the exponential's special-function step (one per sample)
    and, when adapting, the histogram's float shared-memory atomic adds (d per
    sample)."""
    peaks = V.binding.pipe_peaks(reps=3)

    def frac(name, per_sample, samples_per_s):
        got = per_sample * samples_per_s
        return {"per_sample": per_sample, "achieved_per_s": got, "peak_per_s": peaks[name]["per_s"],
                "frac": got / peaks[name]["per_s"]}

    fixed_rate = N_FIXED / (fixed_ms / 1e3)
    out = {"measured": {k: {"per_s": v["per_s"], "per_sm_per_clk": v["per_sm_per_clk"],
                            "sm_mhz": v["sm_mhz"]} for k, v in peaks.items()},
           "basis": "vegas_pipe_peak: 8 independent chains per thread, every SM filled, "
                    "CUDA-event time of one launch, best of 3",
           "fixed_kernel": {"kernel": "vegas_iterate_kernel<float,8,GAUSS,fixed,N=50>",
                            "samples_per_s": fixed_rate,
                            "product": frac("product", products_per_sample(DIM), fixed_rate),
                            "ex2": frac("ex2", 1, fixed_rate)}}
    if adapt_ms:
        adapt_rate = N_ADAPT / (adapt_ms / 1e3)
        out["adapt_kernel"] = {"kernel": "vegas_iterate_kernel<float,8,GAUSS,adapt>",
                               "ms_per_iteration": adapt_ms, "samples_per_s": adapt_rate,
                               "product": frac("product", products_per_sample(DIM), adapt_rate),
                               "atoms_f32": frac("atoms_f32", DIM, adapt_rate)}
    return out


def add_product_fractions(peak, adjoint, batch, mix16, gauss20, genz16):
    """Each FP32 leg's rate of 32x32 -> 64-bit products (the binding pipe of
    every float kernel) as a fraction of the measured product peak, written
    into the leg's fp32 record as product_frac_of_measured."""
    def put(rec, products_per_s):
        rec["product_frac_of_measured"] = products_per_s / peak

    if adjoint:
        for k in ("forward_ms", "backward_ms"):
            adjoint["fp32"]["product_frac_" + k[:-3] + "_of_measured"] = (
                products_per_sample(8) * adjoint["fp32"]["samples"] / (adjoint["fp32"][k] / 1e3)
                / peak)
    if batch:
        put(batch["fp32"], batch["products_per_run"] / (batch["fp32"]["graph_ms"] / 1e3))
    for leg, d in ((mix16, 16), (gauss20, 20)):
        if leg:
            put(leg["fp32"], products_per_sample(d) * leg["fp32"]["samples_per_s"])
    if genz16:
        for fam in genz16.values():
            put(fam["fp32"], products_per_sample(16) * fam["fp32"]["samples_per_s"])


def alg_ops_per_sample(d):
    """Issue slots of one FP32 fixed-grid sample as the method's steps count
    them (the roofline's `achieved`): Philox4x32-10 at 60 per call (10 rounds
    x (2 wide multiplies + 2 xors + 2 round-key additions)); per dimension 7
    (the bin split's wide multiply, the integer-to-float conversion, the map's
    fma, the Jacobian multiply, the shared-memory load of the bin, and the
    Gaussian's subtraction and fma); per sample 12 (the exponential, 3
    multiplies for the weight, 8 for the compensated sums of f J and its
    square).  188 at d = 8."""
    return 60 * ((d + 3) // 4) + 7 * d + 12


def kernel_ops_per_sample(d):
    """The leaner count of the same sample as the kernel issues it: the round
    keys k + r W depend only on the seed, so they are computed once per launch
    rather than per call (40 per call: 10 rounds x (2 wide multiplies + 2
    three-input xors)); per dimension the bin/position multiplies, the
    fraction (2), the grid load, the map fma, the Jacobian multiply and two
    integrand fmas (9); one N^4 multiply per call; and 13 per sample
    (exponential 2, weight 1, Kahan 8 + square 1, finiteness 1).  167 at d = 8."""
    calls = (d + 3) // 4
    return 40 * calls + 9 * d + calls + 13


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="fp64,e2e,pipes,graph,adjoint,batch,mix16,gauss20,genz16",
                    help="measurements besides the headline FP32 steps (comma list of "
                         "fp64, e2e, pipes, graph, adjoint, batch, mix16, gauss20, genz16; '' for none)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons every 50 ms while it
    runs; each row is stamped with the host time it arrived, so that the summary
    covers only the rows inside a given window (the timed region)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        import threading

        self.rows = []
        self.gpu_id = gpu_id
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(gpu_id)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append((time.time(), parts))

    def wait_ready(self, timeout=5.0):
        """Block until the sampler has produced a row (or `timeout` seconds)."""
        t_end = time.time() + timeout
        while self.proc is not None and not self.rows and time.time() < t_end:
            time.sleep(0.01)

    def stop(self, window=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "gpu": self.gpu_id}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=5)
        rows = self.rows
        if window is not None:
            t0, t1 = window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            rows = inside
        rows = [r for _, r in rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in window"],
                    "samples": 0, "gpu": self.gpu_id}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in rows if num(r[0])]
        mx = [num(r[1]) for r in rows if num(r[1])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        loaded = [s for s in sm if s >= 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows), "gpu": self.gpu_id,
                "power_w_max": max((num(r[2]) or 0.0) for r in rows)}


def smi_gpu_id(device):
    """nvidia-smi's name for CUDA device `device`: its UUID.  nvidia-smi numbers
    GPUs in PCI order and ignores CUDA_VISIBLE_DEVICES, so the CUDA index can
    name another job's GPU on a shared machine; the UUID cannot."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(device).uuid)
    except (AttributeError, RuntimeError):
        return str(device)
    return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u


def clocks_rejected(clk):
    """Whether a timed window's clock record rejects its number: a hardware or
    thermal slowdown, or a median SM clock below 85% of the maximum with no
    reason reported (a clock lock left by someone else).  sw_power_cap is kept."""
    if {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"} & set(clk.get("reasons",
                                                                                  ())):
        return True
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.85 * mx and not clk.get("reasons"))


def l2_flush(buf):
    buf.zero_()


def run_step(V, ws, stream, mode, seed, fixed_events=None):
    """Enqueue one whole workload step; returns the handle (not synchronised)."""
    import torch

    from paper_2002_12921_b300 import workloads as W

    h = V.vegas_init_grid(DIM, NBINS, seed, mode, V.VEGAS_GAUSS, W.gauss_params(DIM, A),
                          IT_ADAPT + IT_FIXED, ws.data_ptr(), ws.numel(), stream.cuda_stream)
    for _ in range(IT_ADAPT):
        V.vegas_iterate(h, N_ADAPT, 1)
        V.vegas_refine(h, ALPHA)
    for _ in range(IT_FIXED):
        if fixed_events is not None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            V.vegas_iterate(h, N_FIXED, 0)
            e1.record(stream)
            fixed_events.append((e0, e1))
        else:
            V.vegas_iterate(h, N_FIXED, 0)
    return h


def run_step_sharded(V, stream, mode, seed, world, fixed_events=None):
    """One step of the same integral sharded over `world` ranks (weak scaling:
    every rank keeps the per-GPU sample counts, so an iteration has `world`
    times as many samples): each rank computes its counter range, the partial
    sums and histogram are all-reduced (NCCL), every rank refines."""
    import torch

    from paper_2002_12921_b300 import workloads as W
    from paper_2002_12921_b300.shard import GpuShardEngine, ShardedVegas

    v = V.Vegas(DIM, NBINS, seed, mode, V.VEGAS_GAUSS, W.gauss_params(DIM, A),
                max_iters=IT_ADAPT + IT_FIXED, stream=stream)
    # the ranks' grids are compared once per step (after the last refinement);
    # the comparison is read after the timed steps (ShardedVegas.verify), so no
    # host synchronisation interrupts a step
    # the five fixed-grid iterations' sums are exchanged together, in one
    # all-reduce after the last of them (ShardedVegas.flush)
    sv = ShardedVegas(GpuShardEngine(v, logged=0), check_every=IT_ADAPT, defer_checks=True,
                      defer_fixed=True)
    v.sharded = sv
    for _ in range(IT_ADAPT):
        sv.iterate(N_ADAPT * world, True, ALPHA)
    for _ in range(IT_FIXED):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.iterate(N_FIXED * world, False)
        e1.record(stream)
        if fixed_events is not None:
            fixed_events.append((e0, e1))
    sv.flush()
    return v


# one FP32 step: init + staging of the float grid, iterate + refine per adapting
# iteration, iterate per fixed-grid iteration
LAUNCHES_PER_STEP = 2 + IT_ADAPT * 2 + IT_FIXED


def time_mode(V, mode, steps, warmup, seed0, ws, flush, stream, world=1):
    """Device time of `steps` whole steps (events on the library's stream);
    step s uses seed seed0 + s, and the result returned is the last step's.
    world > 1: the step is sharded over the ranks (run_step_sharded)."""
    import torch

    def step(seed, fixed=None):
        if world > 1:
            return run_step_sharded(V, stream, mode, seed, world, fixed)
        return run_step(V, ws, stream, mode, seed, fixed)

    handles = []
    for w in range(warmup):
        handles.append(step(seed0 + 1000 + w))
    torch.cuda.synchronize()
    time_mode.window_start = time.time()
    step_events, fixed = [], []
    for s in range(steps):
        l2_flush(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        handles.append(step(seed0 + s, fixed))
        e1.record(stream)
        step_events.append((e0, e1))
    torch.cuda.synchronize()
    time_mode.window_end = time.time()
    ms = [a.elapsed_time(b) for a, b in step_events]
    fixed_ms = [a.elapsed_time(b) for a, b in fixed]
    last = handles[-1]
    # device time of each adapting iteration of the last step (the kernels'
    # own global-timer stamps; single-GPU runs)
    time_mode.adapt_ns = (list(V.vegas_get_iteration_times(last, IT_ADAPT + IT_FIXED)[:IT_ADAPT])
                          if world == 1 else None)
    if world > 1:
        res = last.result(IT_ADAPT)
        for v in handles:
            v.sharded.verify()  # raises GridMismatch if any step's grids diverged
            v.close()
    else:
        res = V.vegas_result(last, IT_ADAPT)
        for h in handles:
            V.vegas_destroy(h)
    return ms, fixed_ms, res


def adjoint_timing(V, stream, reps=3):
    """The differentiable d=8 workload (centres mu_i ~ U(0.3, 0.7) from PCG64(3),
    a = 0.15): a grid adapted by 5 iterations of 1e6, then forward (I) and
    backward (I and its 9 derivatives) over 1e8 samples regenerated from their
    counters, per precision.  Returns ms per pass and the result."""
    import torch

    from paper_2002_12921_b300 import workloads as W

    p = W.gauss_params(8, 0.15, W.c3_centres(3, 8))
    n = 100_000_000
    res = {}
    for name, mode in (("fp32", V.VEGAS_FP32_EVAL), ("fp64", V.VEGAS_FP64)):
        v = V.Vegas(8, 50, 3, mode, V.VEGAS_GAUSS, p, max_iters=8, stream=stream)
        v.run([(1_000_000, 1)] * 5)
        times = {}
        for grad in (False, True):
            v.gauss_adjoint(p, 5, n, grad)  # warm-up
            ev = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = v.gauss_adjoint(p, 5, n, grad)
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            times["backward" if grad else "forward"] = statistics.median(
                a.elapsed_time(b) for a, b in ev)
        o = out.cpu().numpy()
        v.close()
        res[name] = {"forward_ms": times["forward"], "backward_ms": times["backward"],
                     "samples": n, "I": float(o[0]), "dI_dmu": [float(x) for x in o[1:9]],
                     "dI_da": float(o[9]), "sigma_dI_da": float(o[19] ** 0.5)}
    return res


def graph_timing(V, stream, reps=5):
    """The d=8 step's schedule (10 x 1e7 adapting + 5 x 1e8 fixed, FP32) as one
    CUDA graph replayed on a state, against the same schedule enqueued call by
    call on an identical state (the paper's graph versus eager modes).  Both
    states continue from their adapted grid after the first step, so both time
    the same work; ms per step, median of `reps`."""
    import torch

    from paper_2002_12921_b300 import workloads as W

    sched = [(N_ADAPT, 1)] * IT_ADAPT + [(N_FIXED, 0)] * IT_FIXED
    iters = (reps + 1) * len(sched)
    p = W.gauss_params(DIM, A)
    stream = torch.cuda.Stream()  # CUDA captures only non-default streams
    out = {}
    for name in ("graph", "eager"):
        v = V.Vegas(DIM, NBINS, 2, V.VEGAS_FP32_EVAL, V.VEGAS_GAUSS, p, max_iters=iters,
                    stream=stream)
        step = v.capture(sched).replay if name == "graph" else (lambda v=v: v.run(sched))
        step()  # warm-up
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        assert v.result(0)[3] == iters
        v.close()
        out[name + "_ms_per_step"] = statistics.median(ms)
    out["launches_per_step"] = LAUNCHES_PER_STEP - 2  # the state's init and staging are not in it
    return out


def batch_timing(V, stream, reps=5):
    """256 independent Gaussians (d ~ U{2..16}, n log-uniform in [1e4, 1e6],
    a ~ U(0.05, 0.3), centres ~ U(0.2, 0.8), 50 bins) x 8 adapting iterations:
    autotuned block size (128, 256, 512), samples per thread (tile = block x
    1 .. 512) and tile per dimension bucket, the whole schedule captured in one
    CUDA graph; samples/s of graph replays and of the same schedule enqueued
    eagerly, per precision (tuned_ms: the tuner's best single adapting
    iteration)."""
    import torch

    from paper_2002_12921_b300 import workloads as W

    wls = W.c4_batch()
    dims = [w.dim for w in wls]
    ns = [w.schedule[0][0] for w in wls]
    params = [w.params for w in wls]
    total = 8 * sum(ns)
    res = {"integrals": len(wls), "iterations": 8, "samples_per_run": total,
           "products_per_run": 8 * sum(n * products_per_sample(d) for d, n in zip(dims, ns))}
    for name, mode in (("fp32", V.VEGAS_FP32_EVAL), ("fp64", V.VEGAS_FP64)):
        B = V.VegasBatch(dims, ns, 50, wls[0].seed, mode, params, max_iters=8, stream=stream)
        choice, cands = V.binding.autotune_batch(B, reps=1)
        graph = B.capture(8)
        graph.replay()
        torch.cuda.synchronize()
        times = {}
        for how in ("graph", "eager"):
            ev = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if how == "graph":
                    graph.replay()
                else:
                    B.run(8)
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            times[how] = statistics.median(a.elapsed_time(b) for a, b in ev)
        B.close()
        res[name] = {"graph_ms": times["graph"], "eager_ms": times["eager"],
                     "samples_per_s": total / (times["graph"] / 1e3),
                     "block_threads": choice[0], "tile_samples": choice[1],
                     "samples_per_thread": choice[1] // choice[0],
                     "tiles_by_dim": {str(d): t for d, t in sorted(choice[2].items())},
                     "tuned_ms": min(cands.values()), "candidates": len(cands)}
    return res


def mix16_timing(V, stream):
    """d=16 two-peak mixture (centres 1/3, 2/3), a = 0.1, 100 bins, adapting
    iterations of 1e9 samples streamed in 1e8-sample launches: the full 20
    iterations in FP32, 2 iterations in FP64 for its rate.  Reports the result
    against the erf closed form and how many bins of each dimension's grid sit
    at each peak: the separable grid tends to lock onto one of the two
    diagonal peaks (so does the oracle), and the estimate then converges to
    half the integral."""
    import numpy as np
    import torch

    from paper_2002_12921_b300 import workloads as W

    wl = W.c5_mix16()
    a = wl.params[0]
    J = lambda c: 0.5 * (math.erf((1 - c) / a) + math.erf(c / a))  # noqa: E731
    exact = 0.5 * (J(1 / 3) ** 16 + J(2 / 3) ** 16)
    # one peak's share, J(1/3)^16 / 2 (= J(2/3)^16 / 2): the value a grid locked
    # onto one peak converges to
    locked = 0.5 * J(1 / 3) ** 16
    res = {"exact": exact, "locked_peak_value": locked,
           "note": "a separable grid cannot hold both diagonal peaks; it locks onto one, as "
                   "the FP64 oracle's does (tests/test_oracle_iterate.py), and the estimate "
                   "tends to half the integral: pull measures that against the full "
                   "integral, pull_locked against the locked peak's value"}
    rows = {}
    for name, mode, iters in (("fp32", V.VEGAS_FP32_EVAL, 20), ("fp64", V.VEGAS_FP64, 2)):
        v = V.Vegas(16, 100, wl.seed, mode, V.VEGAS_GAUSS_MIX2, wl.params, max_iters=32,
                    stream=stream)
        v.config(chunk_samples=wl.chunk)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        v.run([(wl.schedule[0][0], 1)] * iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        m, sg, c2, n, bad = v.result(iters // 2)
        e = v.grid()
        rows[name] = v.iterations()
        v.close()
        # bins whose centre lies within 0.1 of each peak, averaged over dimensions
        mids = (e[:, :-1] + e[:, 1:]) / 2
        near_a = float(np.mean((np.abs(mids - 1 / 3) < 0.1).sum(axis=1)))
        near_b = float(np.mean((np.abs(mids - 2 / 3) < 0.1).sum(axis=1)))
        res[name] = {"iterations": iters, "ms": ms,
                     "samples_per_s": iters * wl.schedule[0][0] / (ms / 1e3),
                     "mean": m, "sigma": sg, "chi2_dof": c2, "pull": (m - exact) / sg,
                     "pull_locked": (m - locked) / sg,
                     "bins_near_1/3": near_a, "bins_near_2/3": near_b}
    # the two precisions on the same iterations (same counters): iteration 0
    # on the same uniform grid, iteration 1 on each one's own first refinement
    res["fp32_vs_fp64_same_iterations"] = [
        {"iteration": t, "I_fp32": float(rows["fp32"][t][4]), "I_fp64": float(rows["fp64"][t][4]),
         "abs_diff_in_sigma": abs(rows["fp32"][t][4] - rows["fp64"][t][4])
         / math.sqrt(rows["fp64"][t][5]),
         "sigma_ratio_fp32_fp64": math.sqrt(rows["fp32"][t][5] / rows["fp64"][t][5])}
        for t in range(2)]
    return res


def timed_schedule(V, stream, dim, seed, mode, fid, params, reps=3):
    """The d=8 workload's schedule (10 x 1e7 adapting, 5 x 1e8 fixed) on a
    fresh state of this integrand: one untimed run first (it loads every kernel
    the schedule uses), then `reps` timed runs on fresh states; the median ms
    and the last run's combined result over the fixed-grid iterations."""
    import torch

    sched = [(N_ADAPT, 1)] * IT_ADAPT + [(N_FIXED, 0)] * IT_FIXED
    ms, res = [], None
    for r in range(reps + 1):
        v = V.Vegas(dim, NBINS, seed, mode, fid, params, max_iters=IT_ADAPT + IT_FIXED,
                    stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        v.run(sched, ALPHA)
        e1.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            ms.append(e0.elapsed_time(e1))
        res = v.result(IT_ADAPT)
        v.close()
    return statistics.median(ms), res


def gauss20_timing(V, stream):
    """The 20-dimensional symmetric Gaussian of Table 1 (Eq. 1, centres 1/2,
    a = 0.1 as in the d=8 workload, 50 bins) on the d=8 workload's schedule:
    10 adapting iterations of 1e7 samples, then 5 fixed-grid iterations of 1e8,
    in both precisions; the result combines the fixed-grid iterations and is
    compared with erf(5)^20."""
    from paper_2002_12921_b300 import workloads as W

    dim, a = 20, 0.1
    exact = math.erf(0.5 / a) ** dim
    res = {"exact": exact}
    for name, mode in (("fp32", V.VEGAS_FP32_EVAL), ("fp64", V.VEGAS_FP64)):
        ms, (m, sg, c2, n, bad) = timed_schedule(V, stream, dim, 20, mode, V.VEGAS_GAUSS,
                                                 W.gauss_params(dim, a),
                                                 reps=3 if name == "fp32" else 1)
        res[name] = {"ms": ms, "samples_per_s": SAMPLES_PER_STEP / (ms / 1e3), "mean": m,
                     "sigma": sg, "chi2_dof": c2, "pull": (m - exact) / sg}
    return res


def genz16_timing(V, stream):
    """Table 1's 16-dimensional Genz integrands (Eq. 2 discontinuous, Eq. 3
    product peak, normalised to 1; seeded a_i, c_i), 50 bins, on the d=8
    workload's schedule (10 x 1e7 adapting, 5 x 1e8 fixed) in both precisions;
    the result combines the fixed-grid iterations and is compared with 1."""
    from paper_2002_12921_b300 import workloads as W

    res = {}
    for fname, fid in (("genz_disc", V.VEGAS_GENZ_DISC), ("genz_ppeak", V.VEGAS_GENZ_PPEAK)):
        p = W.genz_params(16, seed=16, kind=fid)
        res[fname] = {}
        for name, mode in (("fp32", V.VEGAS_FP32_EVAL), ("fp64", V.VEGAS_FP64)):
            ms, (m, sg, c2, n, bad) = timed_schedule(V, stream, 16, 16, mode, fid, p,
                                                     reps=3 if name == "fp32" else 1)
            res[fname][name] = {"ms": ms, "samples_per_s": SAMPLES_PER_STEP / (ms / 1e3),
                                "mean": m, "sigma": sg, "chi2_dof": c2, "pull": (m - 1.0) / sg}
    return res


def e2e_mode(V, mode, steps, seed0, ws, stream):
    """Same workload through the public API with host buffers: per step the
    starting grid and the integrand parameters come from pinned host memory and
    the iteration log is read back to the host for the combined result."""
    import numpy as np
    import torch

    from paper_2002_12921_b300 import workloads as W

    grid = torch.empty((DIM, NBINS + 1), dtype=torch.float64).pin_memory()
    grid.copy_(torch.from_numpy(np.tile(np.arange(NBINS + 1) / NBINS, (DIM, 1))))
    grid_np = grid.numpy()
    params = W.gauss_params(DIM, A)
    times = []
    for s in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = V.vegas_init_grid(DIM, NBINS, seed0 + s, mode, V.VEGAS_GAUSS, params,
                              IT_ADAPT + IT_FIXED, ws.data_ptr(), ws.numel(), stream.cuda_stream)
        V.vegas_set_grid(h, grid_np)
        for _ in range(IT_ADAPT):
            V.vegas_iterate(h, N_ADAPT, 1)
            V.vegas_refine(h, ALPHA)
        for _ in range(IT_FIXED):
            V.vegas_iterate(h, N_FIXED, 0)
        V.vegas_result(h, IT_ADAPT)
        times.append(time.perf_counter() - t0)
        V.vegas_destroy(h)
    h2d = DIM * (NBINS + 1) * 8 + len(params) * 8
    d2h = (IT_ADAPT + IT_FIXED) * 8 * 8 + 64 * 4
    return times, h2d, d2h


def cpu_baseline(fast=False):
    """The FP64 CPU oracle, as it stands, on all host cores, on a bounded sample
    of the workload: 2 adapting iterations of 1e7 then 2 fixed-grid iterations
    of 2e7 samples (6e7 samples)."""
    import oracle
    from paper_2002_12921_b300 import workloads as W

    cores = os.cpu_count() or 1
    sched = [(N_ADAPT, 1)] * 2 + [(2 * N_ADAPT, 0)] * 2
    if fast:
        sched = [(N_ADAPT // 2, 1), (N_ADAPT, 0)]
    oracle.lib()
    t0 = time.perf_counter()
    r = oracle.run(DIM, NBINS, 2, W.GAUSS, W.gauss_params(DIM, A), sched, alpha=ALPHA,
                   nthreads=cores)
    dt = time.perf_counter() - t0
    n = sum(s for s, _ in sched)
    out = {"value": n / dt, "unit": "samples/s", "cores": cores, "kind": "oracle",
           "sample": f"{WORKLOAD}: " + " + ".join(f"{s:.0e}{'a' if a else 'f'}" for s, a in sched)
           + f" = {n:.1e} samples, FP64, {cores} threads", "seconds": dt,
           "result": r["mean"], "cpu_model": cpu_model()}
    if not fast:
        # the same oracle on one thread, on a smaller sample of the workload
        sched1 = [(N_ADAPT // 10, 1), (N_ADAPT // 5, 0)]
        t0 = time.perf_counter()
        oracle.run(DIM, NBINS, 2, W.GAUSS, W.gauss_params(DIM, A), sched1, alpha=ALPHA,
                   nthreads=1)
        dt1 = time.perf_counter() - t0
        n1 = sum(s for s, _ in sched1)
        out["single_core"] = {"value": n1 / dt1, "unit": "samples/s",
                              "sample": f"{n1:.1e} samples (1e6 adapting + 2e6 fixed), 1 thread"}
        # the d=16 two-peak mixture: one 1e8-sample launch chunk of its first
        # (adapting, uniform-grid) iteration, as the GPU streams it
        wl = W.c5_mix16()
        t0 = time.perf_counter()
        oracle.iterate_range(oracle.uniform_grid(16, 100), wl.seed, 0, 0, wl.chunk,
                             W.GAUSS_MIX2, wl.params, True, nthreads=cores)
        dt16 = time.perf_counter() - t0
        out["mix16"] = {"value": wl.chunk / dt16, "unit": "samples/s", "seconds": dt16,
                        "sample": f"d=16 mixture, one {wl.chunk:.0e}-sample chunk of an "
                                  f"adapting iteration (the GPU's launch size), {cores} threads"}
        # the oracle's rate against its thread count (the paper's CPU scaling
        # with cores, Sec. 3.3-3.4): one fixed-grid d=8 iteration of 1e7
        # samples on the uniform grid per thread count, the better of two runs
        # (the host is shared, so a single run can catch another job's load)
        sweep, t = {}, 1
        e8 = oracle.uniform_grid(DIM, NBINS)
        while t <= cores:
            best = 0.0
            for _ in range(2):
                t0 = time.perf_counter()
                oracle.iterate(e8, 2, 0, N_ADAPT, W.GAUSS, W.gauss_params(DIM, A), False,
                               nthreads=t)
                best = max(best, N_ADAPT / (time.perf_counter() - t0))
            sweep[str(t)] = best
            t = t * 2 if t * 2 <= cores or t == cores else cores
        out["thread_scaling"] = {"unit": "samples/s", "samples_per_s_by_threads": sweep,
                                 "sample": "d=8 Gaussian, one fixed-grid iteration of 1e7 "
                                           "samples on the uniform grid per thread count, "
                                           "the better of two runs"}
    return out


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def reference_arm(args, rank, world):
    """The oracle timed as the reference implementation (rank 0 only)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(fast=True)
    vals, secs = [], []
    for _ in range(args.steps):
        cb = cpu_baseline(fast=True)
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    value = statistics.median(vals)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "dim": DIM, "nbins": NBINS,
                       "sample_per_step": cb["sample"]},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch

    import paper_2002_12921_b300 as V

    # one rank per GPU; ranks beyond the visible devices share them (only with a
    # host-side backend, for exercising this path on fewer GPUs)
    torch.cuda.set_device(local % torch.cuda.device_count())
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(os.environ.get("VEGAS_BENCH_DIST_BACKEND", "nccl"))
    V.lib()
    stream = torch.cuda.current_stream()
    ws = torch.empty(V.vegas_workspace_bytes(DIM, NBINS, IT_ADAPT + IT_FIXED), dtype=torch.uint8,
                     device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    seed0 = 2 + 100_000 * rank

    # FP32-eval (headline), with clocks sampled during the timed steps; a window
    # that saw a hardware or thermal slowdown, or clocks well below the maximum
    # with no reason given, is timed once more (every rank, if any rank saw it)
    seed_main = 2 if world > 1 else seed0  # N > 1: one integral sharded over the ranks
    rejected = None
    for attempt in range(2):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(smi_gpu_id(torch.cuda.current_device()))
        clocks.wait_ready()
        ms32, fixed32, res32 = time_mode(V, V.VEGAS_FP32_EVAL, args.steps, max(3, args.warmup),
                                         seed_main, ws, flush, stream, world)
        clk = clocks.stop((time_mode.window_start, time_mode.window_end))
        adapt32_ns = time_mode.adapt_ns
        bad = clocks_rejected(clk)
        if dist:
            flag = torch.tensor([1.0 if bad else 0.0], device="cuda")
            dist.all_reduce(flag, op=dist.ReduceOp.MAX)
            bad = flag.item() > 0
        if not bad or attempt == 1:
            break
        rejected = clk
    if rejected is not None:
        clk["remeasured_after"] = rejected
    total_ms = sum(ms32)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = SAMPLES_PER_STEP * args.steps * world / (total_ms / 1e3)

    legs = {x for x in args.legs.split(",") if x}
    # plain FP64 on the same counters (equal error)
    # (its last step uses the same seed as the FP32 run's last step)
    fp64 = None
    if "fp64" in legs:
        ms64, fixed64, res64 = time_mode(V, V.VEGAS_FP64, args.fp64_steps, 1,
                                         seed0 + args.steps - args.fp64_steps, ws, flush, stream)
        value64 = SAMPLES_PER_STEP * args.fp64_steps / (sum(ms64) / 1e3)
        fp64 = {"value": value64, "unit": "samples/s", "ms_per_step": sum(ms64) / args.fp64_steps,
                "kernel_ms_fixed_iteration": statistics.mean(fixed64)}

    # end to end through the public API with host buffers
    e2e = None
    if "e2e" in legs:
        # every rank runs the workload as an independent replica through the
        # public API; the whole job's rate takes the slowest rank's step time
        if dist:
            dist.barrier()
        e2e_t, h2d, d2h = e2e_mode(V, V.VEGAS_FP32_EVAL, max(3, min(args.steps, 5)), seed0, ws,
                                   stream)
        t_step = statistics.median(e2e_t)
        if dist:
            t = torch.tensor([t_step], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_step = float(t.item())
        e2e = {"value": SAMPLES_PER_STEP * world / t_step, "unit": "samples/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    fixed_ms = statistics.mean(fixed32)
    ops = alg_ops_per_sample(DIM) * N_FIXED
    achieved = ops / (fixed_ms / 1e3) / 1e12
    kernel_achieved = kernel_ops_per_sample(DIM) * N_FIXED / (fixed_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS,
                "unit": "Tops/s", "frac": achieved / ALU_PEAK_TOPS,
                "frac_issue": achieved / ALU_PEAK_TOPS,
                "frac_issue_kernel_count": kernel_achieved / ALU_PEAK_TOPS,
                "traffic": ITERATE_TRAFFIC_BYTES,
                "kernel": "vegas_iterate_kernel<float,8,GAUSS,fixed,N=50>",
                "kernel_ms": fixed_ms, "ops_per_sample": alg_ops_per_sample(DIM),
                "ops_per_sample_kernel_count": kernel_ops_per_sample(DIM),
                "ops_basis": "the method's steps per sample, Philox round-key additions "
                             "included (frac, frac_issue); the kernel computes the round keys "
                             "once per launch (frac_issue_kernel_count)",
                "peak_basis": "148 SMs x 128 lanes x 2032 MHz (recipe unit counts and max clock)",
                # the unit that binds inside that envelope (ncu full capture of this
                # kernel build: fraction of elapsed cycles the pipe was busy)
                "binding_pipe": {"pipe": "fmaheavy: integer multiplies (34 Philox + 8 bin "
                                         "32x32->64 products per d=8 sample)",
                                 "busy_ncu": 0.800}}
    if rank == 0 and "pipes" in legs:
        roofline["pipes"] = pipe_fractions(V, fixed_ms, statistics.median(adapt32_ns) / 1e6
                                           if adapt32_ns else None)
        roofline["frac_binding_pipe_measured"] = roofline["pipes"]["fixed_kernel"]["product"]["frac"]
    if clk.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (SMS * LANES_PER_SM * clk["sm_mhz"] * 1e6
                                                         / 1e12)

    graph = graph_timing(V, stream) if rank == 0 and "graph" in legs else None
    adjoint = adjoint_timing(V, stream) if rank == 0 and "adjoint" in legs else None
    batch = batch_timing(V, stream) if rank == 0 and "batch" in legs else None
    mix16 = mix16_timing(V, stream) if rank == 0 and "mix16" in legs else None
    gauss20 = gauss20_timing(V, stream) if rank == 0 and "gauss20" in legs else None
    genz16 = genz16_timing(V, stream) if rank == 0 and "genz16" in legs else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model",
                                  "single_core", "mix16", "thread_scaling")}

    if rank == 0 and roofline.get("pipes"):
        add_product_fractions(roofline["pipes"]["measured"]["product"]["per_s"], adjoint, batch,
                              mix16, gauss20, genz16)

    if rank == 0:
        m32, s32 = res32[0], res32[1]
        result = {"fp32": {"mean": m32, "sigma": s32, "pull": (m32 - EXACT) / s32},
                  "exact": EXACT}
        if fp64:
            m64, s64 = res64[0], res64[1]
            result["fp64"] = {"mean": m64, "sigma": s64, "pull": (m64 - EXACT) / s64}
            result["sigma_ratio_fp32_fp64"] = s32 / s64
            result["abs_diff_fp32_fp64_in_sigma"] = abs(m32 - m64) / s64
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dim": DIM, "nbins": NBINS, "a": A, "alpha": ALPHA,
                       "samples_per_step": SAMPLES_PER_STEP, "mode": "fp32_eval_fp64_accumulate",
                       "l2": "256 MiB buffer written between timed steps, outside the step events",
                       "parallelism": (f"one integral sharded over {world} ranks: counter "
                                       "ranges, NCCL all-reduce of S1, S2 and the histogram "
                                       "per adapting iteration, of the fixed-grid rows' "
                                       "S1, S2 once per step" if world > 1 else "1 GPU")},
            "clocks": clk,
            "e2e": e2e,
            # sharded: one more kernel per adapting iteration installs the
            # reduced sums, one installs the fixed-grid iterations' rows, and
            # one per step digests the grid for the ranks' comparison
            "gpu_launches": (LAUNCHES_PER_STEP + (IT_ADAPT + 1 + 1 if world > 1 else 0))
            * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "fp64_plain": fp64,
            "speedup_fp32_over_fp64": value / fp64["value"] if fp64 else None,
            "adjoint_d8_a0.15_1e8": adjoint,
            "batch_256_gauss_8iters": batch,
            "graph_vs_eager_d8_step": graph,
            "mix2_d16_N100_1e9_per_iter": mix16,
            "symgauss_d20_a0.1_N50_10x1e7adapt+5x1e8fixed": gauss20,
            "genz_d16_N50_10x1e7adapt+5x1e8fixed": genz16,
            "result": result,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
