#!/usr/bin/env python3
"""Benchmark of the GB300 explicit DOM transient step of the non-gray phonon BTE.

One "step" is one time step of Eq. (disretized_transientBTE) over the whole workload: the
fused forward kernel over every (band, direction, cell) plus the T_L finalize pass.  Default
workload: the 3-D laser-heated block (128x128x64 cells, 40 bands, 96 directions, FP32 state),
the largest of the paper-shaped configurations that runs on one GPU.  Inputs are resident in
HBM before the timed region; the state (16.1 GB a copy) is far larger than L2, so no flush is
needed between steps.  The same run then measures, one context at a time, the sub-records:
the laser block with 16-bit storage, the 2-D hot spot (FP32 and 16-bit), the adjoint/forward
step-time ratio of the two adjoint workloads, an in-plane film run to steady state by the
residual stop, and the transient thermal grating over its xi sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--storage f32|f16|bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own GPU
(weak scaling, no data-path collective); the time is the max over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell·dir·band updates/s and % HBM roofline; adjoint/forward step time"
UNIT = "cell·dir·band updates/s"
FALLBACK_HBM_GBS = 6800.0
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
KERNEL = {"auto": 0, "generic": 1, "tiled": 2, "persistent": 3}


def workloads():
    from paper_2306_14181_gb300 import inputs
    return {
        "hotspot_2d": inputs.hotspot_2d,
        "laser_3d": inputs.laser_3d,
        "film_1d": inputs.film_1d,
        "film_adjoint_2d": inputs.film_adjoint_2d,
        "block_adjoint_3d": inputs.block_adjoint_3d,
    }


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="laser_3d")
    p.add_argument("--storage", default="f32", choices=sorted(STORAGE))
    p.add_argument("--kernel", default="auto", choices=sorted(KERNEL))
    p.add_argument("--rounding", default="nearest", choices=["nearest", "stochastic"],
                   help="rounding of 16-bit codes")
    p.add_argument("--t-scale", type=float, default=1.0, help="16-bit code scale T_scale (K)")
    p.add_argument("--adj-steps", type=int, default=None,
                   help="adjoint workloads: steps of the timed bte_adjoint call (default: the workload's)")
    p.add_argument("--ckpt", type=int, default=None, help="adjoint checkpoint spacing (default: the workload's)")
    p.add_argument("--limiter", type=int, default=2)
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--nb", type=int, default=None, help="override the workload's band count (profiling runs)")
    p.add_argument("--no-sub-records", action="store_true",
                   help="skip the sub-records (the other workloads and storage forms, the adjoint ratios)")
    a = p.parse_args()
    if a.warmup < 3:
        p.error("--warmup must be >= 3")
    return a


# ------------------------------------------------------------------------------------------
# distributed plumbing: one process per GPU, barrier + max over ranks
# ------------------------------------------------------------------------------------------
class Dist:
    def __init__(self, backend):
        import torch
        import torch.distributed as dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = dist if self.world > 1 else None
        if self.dist is not None and not dist.is_initialized():
            dist.init_process_group(backend=backend)
        self.torch = torch

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        if self.dist is None:
            return float(x)
        dev = "cuda" if self.torch.cuda.is_available() and self.dist.get_backend() == "nccl" else "cpu"
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def whole_job_rate(units_per_step, steps, world, t_max_ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_step * steps * world / (t_max_ms / 1e3)


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
REASONS = ["clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
           "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," + ",".join(REASONS)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        load = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# roofline helpers
# ------------------------------------------------------------------------------------------
def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def code_only(text):
    """C/C++/CUDA source without its comments and whitespace (a comment edit leaves the kernel
    unchanged)."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    return "".join("".join(out).split())


def kernel_source_hash():
    """Hash of the tiled forward kernel's code, comments and whitespace aside (the kernel the
    traffic figure describes)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_14181_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if (name.startswith("bte_tiled") and name.endswith((".cu", ".cuh", ".h"))) or name == "bte_internal.h":
            h.update(code_only(open(os.path.join(csrc, name), encoding="utf-8").read()).encode())
    return h.hexdigest()[:12]


def measured_traffic(workload, storage, kernel_name):
    """DRAM bytes per launch of the forward kernel from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        m = re.match(r"^(\S+)\s+(\S+)\s+(\S+)\s+(\S+)\s+([0-9.eE+]+)\s*$", line.strip())
        if m and m.group(1) == workload and m.group(2) == storage and m.group(3) == kernel_name and m.group(4) == src:
            return float(m.group(5))
    return None


# ------------------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------------------
def oracle_for(cfg, sample_n=None, limiter=2):
    from oracle import Problem
    from oracle import quadrature as oq
    c = dict(cfg)
    if sample_n is not None:
        c["n"] = tuple(sample_n)
    s, w, mirror = oq.polar_1d(c["quad"][1]) if c["quad"][0] == "gl1d" else oq.octant_rule(c["quad"][1], c["quad"][2])
    return c, Problem(c["dim"], c["n"], c["h"], c["C"], c["v"], c["tau"], s, w, mirror, c["bc"], c["Tw"], c["dt"],
                      limiter)


def cpu_sample_grid(cfg, updates):
    """Grid of the host sample: the workload with its slowest axes cut (down to 2 cells) until a
    step has about `updates` (band, direction, cell) updates.  All bands and directions are kept."""
    n = list(cfg["n"])
    per_cell = cfg["nb"] * (cfg["quad"][1] if cfg["quad"][0] == "gl1d" else 8 * cfg["quad"][1] * cfg["quad"][2])
    for ax in reversed(range(1, cfg["dim"])):
        rest = per_cell * math.prod(n) // n[ax]
        n[ax] = max(2, min(n[ax], int(updates // max(rest, 1))))
    return tuple(n)


def time_oracle(cfg, seconds, limiter=2, updates=40e6, max_steps=None):
    """Oracle steps on a cut of the workload until `seconds` of host time is used (at least one)."""
    from paper_2306_14181_gb300 import inputs
    c, P = oracle_for(cfg, cpu_sample_grid(cfg, updates), limiter)
    Q = inputs.source_field(c) if cfg.get("source") is not None else None
    e = P.equilibrium(0.0)
    nel = P.nb * P.nd * P.ncell
    t0 = time.perf_counter()
    e = P.step(e, Q, 1.0)
    t1 = time.perf_counter()
    n = 1
    while t1 - t0 < seconds and (max_steps is None or n < max_steps):
        e = P.step(e, Q, 1.0)
        n += 1
        t1 = time.perf_counter()
    return nel * n / (t1 - t0), n, c["n"], t1 - t0


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def time_oracle_one_thread(workload, seconds, limiter):
    """The oracle on one host thread (a child process with OMP_NUM_THREADS=1, so the OpenMP
    runtime of this process keeps its thread count)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "cfg = bench.workloads()[%r](); v, n, g, t = bench.time_oracle(cfg, %r, %r, 4e6, 50); "
            "print(json.dumps([v, n, list(g), t]))" % (ROOT, workload, float(seconds), int(limiter)))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=seconds * 4 + 120)
        v, n, g, t = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None
    return {"value": v, "unit": UNIT, "cores": 1,
            "sample": "%d FP64 oracle steps on a %s cut of the workload, %.1f s" % (n, "x".join(map(str, g)), t)}


# ------------------------------------------------------------------------------------------
def run_reference(args):
    d = Dist("gloo")
    if d.rank != 0:
        d.barrier()
        d.close()
        return
    cfg = make_workload(args)
    from oracle import build_oracle
    build_oracle()
    # about 75 s of oracle work at ~2e8 updates/s over the whole --steps + --warmup run
    updates = min(4e7, max(2e6, 1.5e10 / (args.steps + args.warmup)))
    c, P = oracle_for(cfg, cpu_sample_grid(cfg, updates), args.limiter)
    from paper_2306_14181_gb300 import inputs
    Q = inputs.source_field(c) if cfg.get("source") is not None else None
    e = P.equilibrium(0.0)
    for _ in range(args.warmup):
        e = P.step(e, Q, 1.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e = P.step(e, Q, 1.0)
    t = time.perf_counter() - t0
    nel = P.nb * P.nd * P.ncell
    value = nel * args.steps / t
    sample = "%d oracle steps on a %s cut of %s (all bands and directions)" % (args.steps, "x".join(map(str, c["n"])),
                                                                             cfg["name"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "storage": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "sample_grid": list(c["n"]), "bands": c["nb"], "dirs": P.nd,
                       "limiter": args.limiter},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": omp_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    d.barrier()
    d.close()


def l2_note(info):
    """How the timed steps relate to L2: each step reads one state copy and writes the other."""
    import torch
    from paper_2306_14181_gb300 import bte
    l2 = getattr(torch.cuda.get_device_properties(torch.cuda.current_device()), "L2_cache_size", 0) or (126 << 20)
    ws = 2 * info.state_bytes
    if info.kernel == bte.BTE_KERNEL_PERSISTENT:
        return "state held in shared memory for the whole call; no DRAM traffic to flush"
    if ws > l2:
        return "step reads %.2f GB and writes %.2f GB (> %d MB L2), no flush" % (
            info.state_bytes / 1e9, info.state_bytes / 1e9, l2 >> 20)
    return "step working set %.0f MB fits the %d MB L2: steps run L2-warm, no flush" % (ws / 2**20, l2 >> 20)


def make_workload(args):
    kw = {} if args.nb is None else {"nb": args.nb}
    return workloads()[args.workload](**kw)


def kernel_name_of(info):
    from paper_2306_14181_gb300 import bte
    return {bte.BTE_KERNEL_TILED: "tiled", bte.BTE_KERNEL_PERSISTENT: "persistent"}.get(info.kernel, "generic")


def make_context(cfg, storage, limiter, kernel, T_scale, rounding, amps_len):
    """A context of the workload with its source field (device) and amplitudes set."""
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    Q = inputs.source_field(cfg)
    amps = inputs.source_amplitudes(cfg, amps_len)
    stream = torch.cuda.current_stream()
    ctx = bte.bte_from_workload(cfg, storage=storage, limiter=limiter, kernel=kernel, stream=stream.cuda_stream,
                                T_scale=T_scale, rounding=rounding, seed=1)
    if Q is not None:
        bte.bte_set_source(ctx, torch.from_numpy(Q.reshape(-1)).cuda(), amps)
    return ctx, Q, amps


def timed_forward(ctx, steps, d=None, clocks=None):
    """Device time of `steps` bte_step calls (CUDA events on the context's stream) with the
    library's per-launch tracing: (total ms, forward ms, forward launches, finalize ms,
    finalize launches)."""
    import torch
    from paper_2306_14181_gb300 import bte
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    if d is not None:
        d.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    bte.bte_profile(ctx, True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    bte.bte_step(ctx, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if d is not None:
        d.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks is not None else None
    fwd_ms, nfwd, fin_ms, nfin = bte.bte_profile_read(ctx)
    bte.bte_profile(ctx, False)
    bte.bte_synchronize(ctx)  # a bounded wait that gave up is reported here
    return ev0.elapsed_time(ev1), fwd_ms, nfwd, fin_ms, nfin, ck


def roofline_of(info, steps, fwd_ms, nfwd, fin_ms, nfin, peak, peak_kind, traffic=None):
    """Roofline of the forward kernel: algorithmic bytes = read e + write e per update, over the
    mean device time of one launch."""
    from paper_2306_14181_gb300 import bte
    persistent = info.kernel == bte.BTE_KERNEL_PERSISTENT
    # a persistent launch covers all the steps of its bte_step call
    steps_per_launch = steps / max(nfwd, 1) if persistent else 1
    bytes_per_launch = info.nelem * 2 * info.elem_bytes * steps_per_launch
    fwd_avg_s = fwd_ms / max(nfwd, 1) / 1e3
    achieved = bytes_per_launch / fwd_avg_s / 1e9
    r = {"bound": "latency" if persistent else "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": traffic, "kernel": "forward step (%s)" % kernel_name_of(info),
         "peak_source": peak_kind, "bytes_per_launch": bytes_per_launch, "kernel_ms": fwd_avg_s * 1e3,
         "finalize_ms": fin_ms / max(nfin, 1)}
    if persistent:
        # the state stays in shared memory: report the step time, not a DRAM fraction
        r["us_per_step"] = fwd_avg_s * 1e6 / steps_per_launch
        r["note"] = "one single-CTA launch per bte_step call; the state never leaves shared memory"
        r["finalize_ms"] = 0.0
    return r


def adjoint_record(ctx, cfg, info, fwd_step_ms, nadj, kck, Q, amps, peak):
    """One traced bte_adjoint call (forward sweep + checkpointed reverse sweep) of J = mean T_L
    over the workload's probe: adjoint-step and forward-step device times and their ratio."""
    import numpy as np
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    probe = inputs.probe_weights(cfg)
    bte.bte_init_temperature(ctx, None)
    if Q is not None:
        bte.bte_set_source(ctx, torch.from_numpy(Q.reshape(-1)).cuda(), amps)
    torch.cuda.synchronize()
    bte.bte_profile(ctx, True)
    t0 = time.perf_counter()
    J, gQ, gt = bte.bte_adjoint(ctx, nadj, probe, kck)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    adj_ms, nadj_k, rec_ms, nrec = bte.bte_adjoint_profile_read(ctx)
    bte.bte_profile(ctx, False)
    adj_step = adj_ms / max(nadj_k, 1)
    adj_bytes = info.nelem * (8 + info.elem_bytes)
    return {"steps": nadj, "ckpt": kck, "J": J, "adj_step_ms": adj_step, "fwd_step_ms": fwd_step_ms,
            "ratio": adj_step / fwd_step_ms, "recompute_steps": nrec, "recompute_ms": rec_ms, "wall_s": wall,
            "bytes_per_adj_step": adj_bytes, "achieved_gbs": adj_bytes / (adj_step / 1e3) / 1e9,
            "frac": adj_bytes / (adj_step / 1e3) / 1e9 / peak,
            "grad_finite": bool(np.all(np.isfinite(gQ)) and np.all(np.isfinite(gt)))}


# Sub-records measured in the same run after the headline, one context at a time: (workload,
# storage, T_scale, timed forward steps, adjoint steps or None, checkpoint spacing, kernel).
# The 3-D adjoint runs 100 of its 1000 steps (checkpoints every 50) to keep the run within
# minutes.  The hot spot also runs on the generic kernel (one thread per cell and band), the
# path grids of any shape take.
SUB_RECORDS = [
    ("laser_3d", "f16", 1.0, 30, None, None, "auto"),
    ("hotspot_2d", "f32", 1.0, 100, None, None, "auto"),
    ("hotspot_2d", "f16", 10.0, 100, None, None, "auto"),
    ("hotspot_2d", "f32", 1.0, 20, None, None, "generic"),
    ("film_adjoint_2d", "f32", 1.0, 100, 2000, 100, "auto"),
    ("block_adjoint_3d", "f16", 1.0, 10, 100, 50, "auto"),
]


def sub_record(args, name, storage, T_scale, steps, nadj, kck, peak, peak_kind, kernel="auto"):
    import gc
    import torch
    from paper_2306_14181_gb300 import bte
    cfg = workloads()[name]()
    warm = 3
    ctx, Q, amps = make_context(cfg, STORAGE[storage], args.limiter, KERNEL[kernel], T_scale, 0,
                                warm + steps + 8)
    info = ctx.info
    bte.bte_step(ctx, warm)
    t_ms, fwd_ms, nfwd, fin_ms, nfin, _ = timed_forward(ctx, steps)
    rec = {"workload": cfg["name"], "storage": storage, "kernel": kernel_name_of(info), "steps": steps,
           "warmup": warm, "ms_per_step": t_ms / steps, "value": info.nelem * steps / (t_ms / 1e3), "unit": UNIT,
           "updates_per_step": info.nelem,
           "roofline": roofline_of(info, steps, fwd_ms, nfwd, fin_ms, nfin, peak, peak_kind)}
    if storage != "f32":
        rec["T_scale"] = T_scale
    if nadj is not None:
        fwd_step = (fwd_ms / max(nfwd, 1)) + fin_ms / max(nfin, 1)
        rec["adjoint"] = adjoint_record(ctx, cfg, info, fwd_step, nadj, kck, Q, amps, peak)
    bte.bte_destroy(ctx)
    del ctx
    gc.collect()
    torch.cuda.empty_cache()
    return rec


def steady_record(args):
    """f1: the in-plane film run to steady state by the residual stop of the transient solver
    (eps_T and eps_q below 1e-7, checked every 200 steps): steps, device time and the in-plane
    conductivity q L / dT against the bulk sum C v^2 tau / 3."""
    import gc
    import numpy as np
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    cfg = inputs.inplane_film_2d()
    ctx = bte.bte_from_workload(cfg, limiter=args.limiter, stream=torch.cuda.current_stream().cuda_stream)
    info = ctx.info
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n, eT, eq = bte.bte_run_steady(ctx, cfg["steps"], 200, 1e-7, 1e-7)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _, _, q = bte.bte_moments(ctx)
    L = cfg["n"][0] * cfg["h"][0]
    kappa = float(np.mean(q[0])) * L / cfg["jump"][0]
    kbulk = float(np.sum(cfg["C"] * cfg["v"] ** 2 * cfg["tau"]) / 3.0)
    rec = {"workload": cfg["name"], "storage": "f32", "kernel": kernel_name_of(info), "steps": n, "converged": bool(
        eT < 1e-7 and eq < 1e-7), "eps_T": eT, "eps_q": eq, "wall_s": wall, "ms_per_step": 1e3 * wall / max(n, 1),
           "kappa_inplane": kappa, "kappa_bulk": kbulk, "kappa_ratio": kappa / kbulk,
           "note": "residual stop of Algorithm 2 (eps_T, eps_q < 1e-7, checked every 200 steps); "
                   "wall time includes the FP64 residual reductions"}
    bte.bte_destroy(ctx)
    del ctx
    gc.collect()
    return rec


def ttg_record(args, xi):
    """f2: the transient thermal grating (1000 cells, 512 directions, gray Si) at xi = 2 pi Kn over
    t* = t/tau up to 10/xi: device time of the steps and the grating amplitude at the end."""
    import gc
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    cfg = inputs.ttg_1d(xi)
    ctx = bte.bte_from_workload(cfg, limiter=args.limiter, stream=torch.cuda.current_stream().cuda_stream)
    info = ctx.info
    bte.bte_init_temperature(ctx, inputs.ttg_initial_temperature(cfg).reshape(-1))
    # CUDA events around the one bte_step call, without per-launch tracing: a long call replays
    # captured step graphs, which tracing would turn off
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    bte.bte_step(ctx, cfg["steps"])
    ev1.record(stream)
    torch.cuda.synchronize()
    bte.bte_synchronize(ctx)
    t_ms = ev0.elapsed_time(ev1)
    T, _, _ = bte.bte_moments(ctx)
    rec = {"workload": cfg["name"], "xi": xi, "storage": "f32", "kernel": kernel_name_of(info), "steps": cfg["steps"],
           "t_star_end": cfg["steps"] * cfg["dt"] / cfg["tau_ref"], "ms_per_step": t_ms / cfg["steps"],
           "value": info.nelem * cfg["steps"] / (t_ms / 1e3), "unit": UNIT,
           "amplitude_end": inputs.grating_amplitude(cfg, T) / cfg["A0"]}
    bte.bte_destroy(ctx)
    del ctx
    gc.collect()
    return rec


def implicit_record(args, explicit):
    """f4: the in-plane film solved by the steady implicit DOM (sequential iterations, Sec.
    3.3-3.5) to eps_T, eps_q < 1e-6 (checked every 5 iterations; the FP32 right-hand side keeps
    the change between iterates near 1e-7): iterations, device time per
    iteration (CUDA events over the whole solve, residual checks included) and the in-plane
    conductivity, beside the time-marched solve of the same problem."""
    import gc
    import numpy as np
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    cfg = inputs.inplane_film_2d()
    stream = torch.cuda.current_stream()
    ctx = bte.bte_from_workload(cfg, limiter=args.limiter, stream=stream.cuda_stream)
    info = ctx.info
    bte.bte_sis_iterate(ctx, 2)  # warm-up (module load, first launches)
    bte.bte_init_temperature(ctx, None)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n, eT, eq = bte.bte_run_steady_implicit(ctx, 2000, 5, 1e-6, 1e-6)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1)
    _, _, q = bte.bte_moments(ctx)
    L = cfg["n"][0] * cfg["h"][0]
    kappa = float(np.mean(q[0])) * L / cfg["jump"][0]
    rec = {"workload": cfg["name"], "method": "steady implicit DOM, sequential iterations", "storage": "f32",
           "forward_kernel": kernel_name_of(info), "iterations": n, "converged": bool(eT < 1e-6 and eq < 1e-6),
           "eps_T": eT, "eps_q": eq, "ms_total": t_ms, "ms_per_iteration": t_ms / max(n, 1),
           "kappa_inplane": kappa}
    if explicit is not None and explicit.get("steps"):
        rec["time_marching"] = {"steps": explicit["steps"], "wall_s": explicit["wall_s"],
                                "kappa_inplane": explicit["kappa_inplane"]}
        rec["speedup_vs_time_marching"] = explicit["wall_s"] * 1e3 / t_ms
    bte.bte_destroy(ctx)
    del ctx
    gc.collect()
    # one iteration at the hot spot's size (5120 planes of 256 x 256 cells): forward step (8 B an
    # update), sweep (12 B) and moment pass (4 B) over the iteration's device time
    hcfg = inputs.hotspot_2d()
    hctx = bte.bte_from_workload(hcfg, limiter=args.limiter, stream=stream.cuda_stream)
    Q = inputs.source_field(hcfg)
    bte.bte_set_source(hctx, torch.from_numpy(Q.reshape(-1)).cuda())
    bte.bte_sis_iterate(hctx, 2)
    torch.cuda.synchronize()
    its = 10
    ev0.record(stream)
    bte.bte_sis_iterate(hctx, its)
    ev1.record(stream)
    torch.cuda.synchronize()
    it_ms = ev0.elapsed_time(ev1) / its
    nel = hctx.info.nelem
    gbs = nel * 24 / (it_ms / 1e3) / 1e9
    rec["hotspot_iteration"] = {"workload": hcfg["name"], "iterations": its, "ms_per_iteration": it_ms,
                                "bytes_per_iteration": nel * 24, "achieved_gbs": gbs,
                                "frac": gbs / hbm_peak()[0], "unit": "GB/s",
                                "note": "forward step 8 B + sweep 12 B + moment pass 4 B per update"}
    bte.bte_destroy(hctx)
    del hctx
    gc.collect()
    torch.cuda.empty_cache()
    # the near-diffusive film: sequential against synthetic iterations (Sec. 3.5) to 1e-5
    dcfg = inputs.diffusive_film_1d()
    schemes = {}
    for name, scheme in (("sequential", bte.BTE_SCHEME_SEQUENTIAL), ("synthetic", bte.BTE_SCHEME_SYNTHETIC)):
        dctx = bte.bte_from_workload(dcfg, limiter=args.limiter, stream=stream.cuda_stream)
        bte.bte_set_steady_scheme(dctx, scheme)
        bte.bte_sis_iterate(dctx, 2)
        bte.bte_init_temperature(dctx, None)
        torch.cuda.synchronize()
        ev0.record(stream)
        n, eT, eq = bte.bte_run_steady_implicit(dctx, 20000, 5, 1e-5, 1e-5)
        ev1.record(stream)
        torch.cuda.synchronize()
        _, _, q = bte.bte_moments(dctx)
        schemes[name] = {"iterations": n, "converged": bool(eT < 1e-5 and eq < 1e-5), "ms_total": ev0.elapsed_time(ev1),
                         "q_mean_w_m2": float(np.mean(q[0]))}
        bte.bte_destroy(dctx)
        del dctx
    rec["diffusive_film"] = {"workload": dcfg["name"], "tol": 1e-5, **schemes}
    gc.collect()
    return rec


def interface_record(args, peak, peak_kind):
    """f3: the two-material interface pair (both sides' forward steps and the interface kernel
    each step), timed with CUDA events over 100 coupled steps after 3 warm-up ones; the
    roofline counts both sides' algorithmic bytes over the pair step."""
    import gc
    import torch
    from paper_2306_14181_gb300 import bte, inputs
    cfg = inputs.interface_2d()
    stream = torch.cuda.current_stream()
    ctxs = []
    for side, w in (("A", cfg["wall_a"]), ("B", cfg["wall_b"])):
        c = dict(cfg[side])
        c["bc"] = [bte.BTE_BC_INTERFACE if j == w else b for j, b in enumerate(c["bc"])]
        ctxs.append(bte.bte_from_workload(c, limiter=args.limiter, stream=stream.cuda_stream))
    A, B = ctxs
    Q = inputs.source_field(cfg["A"])
    bte.bte_set_source(A, torch.from_numpy(Q.reshape(-1)).cuda())
    bte.bte_interface(A, cfg["wall_a"], B, cfg["wall_b"], cfg["beta_ab"], cfg["beta_ba"])
    bte.bte_step_pair(A, B, 3)
    steps = 100
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    bte.bte_step_pair(A, B, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    bte.bte_synchronize(A)
    bte.bte_synchronize(B)
    t_ms = ev0.elapsed_time(ev1)
    n = A.info.nelem + B.info.nelem
    bytes_step = n * 2 * A.info.elem_bytes
    achieved = bytes_step / (t_ms / steps / 1e3) / 1e9
    _, FA = bte.bte_energy(A)
    _, FB = bte.bte_energy(B)
    rec = {"workload": cfg["name"], "storage": "f32", "kernel": kernel_name_of(A.info), "steps": steps, "warmup": 3,
           "ms_per_step": t_ms / steps, "value": n * steps / (t_ms / 1e3), "unit": UNIT, "updates_per_step": n,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": "pair step (two forward steps, two finalizes, the interface kernel)",
                        "peak_source": peak_kind, "bytes_per_step": bytes_step},
           "interface_flow_w_per_m": [FA[cfg["wall_a"]], FB[cfg["wall_b"]]],
           "launches_per_step": A.info.launches_per_step + B.info.launches_per_step + 1}
    bte.bte_destroy(B)
    bte.bte_destroy(A)
    del A, B, ctxs
    gc.collect()
    torch.cuda.empty_cache()
    return rec


def run_gb300(args):
    import gc
    import numpy as np
    import torch

    d = Dist("nccl")
    torch.cuda.set_device(d.local)
    from paper_2306_14181_gb300 import bte, build
    build.build()
    cfg = make_workload(args)
    storage = STORAGE[args.storage]
    total = args.warmup + args.steps + args.e2e_steps + 8
    ctx, Q, amps = make_context(cfg, storage, args.limiter, KERNEL[args.kernel], args.t_scale,
                                1 if args.rounding == "stochastic" else 0, total)
    info = ctx.info
    kernel_name = kernel_name_of(info)
    bte.bte_step(ctx, args.warmup)
    clocks = ClockSampler(torch.cuda.current_device())
    t_ms, fwd_ms, nfwd, fin_ms, nfin, ck = timed_forward(ctx, args.steps, d, clocks)
    t_max = d.max(t_ms)
    value = whole_job_rate(info.nelem, args.steps, d.world, t_max)
    peak, peak_kind = hbm_peak()
    persistent = info.kernel == bte.BTE_KERNEL_PERSISTENT
    roofline = roofline_of(info, args.steps, fwd_ms, nfwd, fin_ms, nfin, peak, peak_kind,
                           measured_traffic(args.workload, args.storage, kernel_name))

    # end to end through the C ABI with host buffers: upload the step's source (pinned), step,
    # read the step's lattice temperature back
    e2e = None
    if not args.no_e2e:
        Qh = torch.from_numpy(np.ascontiguousarray(Q.reshape(-1))).pin_memory() if Q is not None else None
        TLh = np.empty(info.ncell)
        torch.cuda.synchronize()
        d.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            if Qh is not None:
                bte.bte_set_source(ctx, Qh.numpy(), amps)
            bte.bte_step(ctx, 1)
            bte.bte_lattice_temperature(ctx, TLh)
        torch.cuda.synchronize()
        te = d.max(time.perf_counter() - t0)
        e2e = {"value": info.nelem * args.e2e_steps * d.world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(info.ncell * 4 if Qh is not None else 0),
               "d2h_bytes_per_step": int(info.ncell * 4)}
    # adjoint workloads as the headline: one traced bte_adjoint call
    adjoint = None
    if "probe" in cfg:
        nadj = args.adj_steps if args.adj_steps is not None else cfg["steps"]
        kck = args.ckpt if args.ckpt is not None else cfg.get("ckpt", 0)
        fwd_step = fwd_ms / max(nfwd, 1) + fin_ms / max(nfin, 1)
        adjoint = adjoint_record(ctx, cfg, info, fwd_step, nadj, kck, Q, amps, peak)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "storage": args.storage, "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": list(cfg["n"]), "bands": info.nbands, "dirs": info.ndirs,
                       "storage": args.storage, "limiter": args.limiter, "kernel": kernel_name,
                       **({"rounding": args.rounding, "T_scale": args.t_scale} if args.storage != "f32" else {}),
                       "updates_per_step": info.nelem, "l2": l2_note(info),
                       "parallelism": "replicas" if d.world > 1 else "single"},
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e,
            "gpu_launches": int(nfwd if persistent else nfwd * info.launches_per_step), "clocks": ck}
    if adjoint is not None:
        line["adjoint"] = adjoint
    bte.bte_destroy(ctx)
    del ctx
    gc.collect()
    torch.cuda.empty_cache()
    # the other workloads, storage forms and the adjoint ratios (one GPU runs only)
    if d.world == 1 and not args.no_sub_records:
        subs = []
        for name, st, ts, steps, nadj, kck, kern in SUB_RECORDS:
            if name == args.workload and st == args.storage and nadj is None and kern == args.kernel:
                continue
            subs.append(sub_record(args, name, st, ts, steps, nadj, kck, peak, peak_kind, kern))
        subs.append(steady_record(args))
        subs.append(implicit_record(args, subs[-1]))
        subs.append(interface_record(args, peak, peak_kind))
        for xi in (0.1, 1.0, 10.0):
            subs.append(ttg_record(args, xi))
        line["sub_records"] = subs
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        v, n, grid, secs = time_oracle(cfg, args.cpu_seconds, args.limiter)
        cpu = {"value": v, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": "%d FP64 oracle steps on a %s cut of the workload (all bands and directions), %.1f s"
                         % (n, "x".join(map(str, grid)), secs)}
        one = time_oracle_one_thread(args.workload, min(args.cpu_seconds, 10.0), args.limiter)
        if one is not None:
            cpu["single_thread"] = one
        line["cpu_baseline"] = cpu
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.barrier()
    d.close()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gb300(a)
