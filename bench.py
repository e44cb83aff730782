#!/usr/bin/env python3
"""Benchmark of the short-range gravity hot path on one GB300 (or N replicas).

One step = the whole path on one synthetic particle set with inputs resident
in HBM: og_keys_sort -> og_tree_build -> og_shortrange_accel (FP32+Kahan) ->
og_shortrange_adjoint (FP32, frozen decisions).  value = interactions per
step / step time.  The all-FP64 walk (the comparison variant) is timed on
the same tree in the same run and reported under "fp64".

Default workload: the largest single-GPU set, 256^3 = 16,777,216 particles
with 60% of the mass in 2000 NFW haloes and 40% uniform background,
eps = 1/7680, r_s = 1.25/512, rcut = 4.5 r_s, theta = 0.5.  The 128^3
Zel'dovich lattice and the 10.5M-particle zoom set are timed beside it.
Inputs are larger than L2, which is flushed (256 MiB write) between timed
steps anyway.

Measured on the device in the same run: the FP32 (FFMA), packed FP32
(FFMA2), special-function (MUFU) and FP64 (DFMA) pipe rates (og_probe_pipe),
which the roofline fractions use beside the unit-count peak; and the error of
the GPU walk against the FP64 oracle (tree at the same theta on the CPU
baseline's sampled targets, direct sum on a bounded sample, theta = 0 on the
4096-particle set).

--impl reference times the CPU oracle (single-threaded FP64) on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs an
independent replica (no collective on the data path; "scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "short-range interactions/s and particles/s (fwd, fwd+adjoint) on 1 GB300, FP32 vs FP64"
UNIT = "interactions/s"
# FP32 flops per interaction (FFMA = 2).  "Algorithmic" is the canonical form
# of one term: displacement 3, r^2 5, r 1, u 1, exp argument 2, erfcx
# polynomial 20, f 3, m K f 4, accumulation 6 (plus 2 MUFU: rsqrt, ex2).  The
# adjoint adds F'/r 6, d.w 5, (F'/r)(d.w) 1, J w 9, the target-side m J w 6 and
# the source-side (J w, w.g) 4 after dropping the forward accumulation.
# "Implemented" counts walk.cu as written (split-float displacement, degree-11
# polynomial, Kahan fold).
FWD_FLOPS = 45
ADJ_FLOPS = 70
FWD_FLOPS_IMPL = 51
ADJ_FLOPS_IMPL = 75
MUFU_PER_INTERACTION = 2
FP64_FLOPS = 45      # the same canonical form in FP64 (CUDA's erfc / exp calls not counted)

WORKLOADS = {
    "zeldovich128": "128^3 Zel'dovich lattice, P(k)~k^-2, rms disp 0.5 cells, eps=1/3840, r_s=1.25/256, theta=0.5",
    "nfw256": "256^3 clustered: 60% mass in 2000 NFW haloes, 40% uniform, eps=1/7680, r_s=1.25/512, theta=0.5",
    "nfw128_adjoint": "128^3 clustered (NFW haloes + background), eps=1/3840, r_s=1.25/256, theta=0.5",
    "zoom8m": "2^23 high-res NFW sphere + 2^21 low-res (64 m) background, eps 5e-5/2e-4, r_s=1.25/512, theta=0.5",
    "uniform4096": "4096 uniform points, eps=1/480, r_s=1.25/16, theta=0.5",
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest value of x over the ranks (x itself on one rank): the
    replicas' time is that of the slowest one."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, ms: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in ms."""
    return ws * units_per_rank / (ms * 1e-3)


def walk_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of a walk kernel ("forward" or "adjoint") on this
    workload from the committed ncu summary, if it was taken on the current
    walk.cu (else None)."""
    path = os.path.join(ROOT, "profiles", f"walk_fp32_{workload}.md")
    src = os.path.join(ROOT, "paper_2606_17145_gb300", "csrc", "walk.cu")
    try:
        text = open(path).read()
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m = re.search(r"walk\.cu sha256\[:16\]:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch_%s:\s*([0-9.eE+]+)" % kernel, text)
    if not m or not t or m.group(1) != digest:
        return None
    return float(t.group(1))


class Clocks:
    """nvidia-smi sampling of SM clock / throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"og_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[2], parts[3:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, _, flags in rows:
            for nm, v in zip(names[1:], flags[1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def host_info():
    """Host core count and CPU model (lscpu), for the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"host_cores": os.cpu_count(), "cpu_model": model}


def pipe_peaks(og, L, dev):
    """Measured pipe rates (og_probe_pipe, CUDA events, best of 3 launches)."""
    import ctypes as C
    import torch
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    out = {}
    for kind, name, iters in ((0, "ffma", 4096), (1, "ffma2", 2048), (2, "mufu", 1024), (3, "dfma", 256)):
        ops = C.c_uint64()
        best = None
        for _ in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            code = L.og_probe_pipe(kind, iters, C.c_void_p(sink.data_ptr()), C.byref(ops),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
            b.record()
            torch.cuda.synchronize()
            if code != 0:
                raise SystemExit(f"og_probe_pipe({name}) failed: {code}")
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[name] = ops.value / (best * 1e-3)   # operations per second
    return {"fp32_tflops": 2 * out["ffma"] / 1e12, "fp32x2_tflops": 2 * out["ffma2"] / 1e12,
            "mufu_per_s": out["mufu"], "fp64_tflops": 2 * out["dfma"] / 1e12,
            "how": "og_probe_pipe: independent FMA / f32x2 FMA / rsqrt+ex2 / DFMA chains, 4 blocks x 256 "
                   "threads per SM, best of 4 launches timed with CUDA events"}


# ----------------------------------------------------------------- CPU oracle

def oracle_throughput(w, theta, budget_s=12.0, min_targets=1024, seed=5, T=None):
    """Single-threaded FP64 oracle forward walk on sampled targets (tree built
    once, untimed).  Returns (interactions/s, particles/s, sample text,
    targets, oracle accelerations of those targets)."""
    import numpy as np
    import oracle
    t0 = time.time()
    own = T is None
    if own:
        T = oracle.Tree(w.pos, w.mass, 2.8 * w.eps)
    build_s = time.time() - t0
    rng = np.random.default_rng(seed)
    perm = rng.permutation(w.n)
    done, inter, spent = 0, 0, 0.0
    chunk = min_targets
    accs = []
    while done < w.n and (spent < budget_s or done < min_targets):
        tg = perm[done:done + chunk]
        t1 = time.time()
        a, cnt = T.walk(w.r_s, w.rcut, theta, tg)
        spent += time.time() - t1
        accs.append(a)
        inter += int(cnt.sum())
        done += len(tg)
    if own:
        T.close()
    sample = (f"oracle tree walk (1 thread, FP64, -O2) of {done} random targets of the {w.n}-particle set "
              f"(tree over all particles built once, {build_s:.1f} s, untimed); forward walk only")
    return inter / spent, done / spent, sample, perm[:done], np.concatenate(accs)


def rel_stats(a, ref):
    """Per-particle relative error |a_i - ref_i| / |ref_i|: rms, median, p99, max."""
    import numpy as np
    r = np.linalg.norm(a - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return {"rms": float(np.sqrt(np.mean(r * r))), "median": float(np.median(r)),
            "p99": float(np.percentile(r, 99)), "max": float(r.max()), "n": int(len(r))}


def accuracy_c1(og, dev):
    """GPU FP32 walk on the 4096-particle uniform set against the oracle direct
    sum: rms at theta = 0 and p99 for a range of theta."""
    import numpy as np
    import ics
    import oracle
    import torch
    w = ics.make("uniform4096")
    pos = torch.tensor(w.pos, device=dev)
    mass = torch.tensor(w.mass, device=dev)
    eps = torch.tensor(w.eps, device=dev)
    k, o = og.keys_sort(pos, w.box)
    tree = og.tree_build(k, o, pos, mass, eps, w.box)
    ad, _ = oracle.direct(w.pos, w.mass, 2.8 * w.eps, w.box, w.r_s, w.rcut)
    out = {}
    for th in (0.0, 0.2, 0.3, 0.5):
        a, _, _ = og.shortrange_accel(tree, w.r_s, th)
        out[f"theta_{th}"] = rel_stats(a.double().cpu().numpy(), ad)
    ok = [th for th in (0.5, 0.3, 0.2) if out[f"theta_{th}"]["p99"] <= 5e-3]
    return {"set": "uniform4096 (4096 uniform, eps=1/480, r_s=1.25/16) vs oracle direct sum",
            "theta0_rms": out["theta_0.0"]["rms"], "p99_by_theta": {k: v["p99"] for k, v in out.items()},
            "largest_theta_with_p99_le_5e-3": max(ok) if ok else None}


def run_reference(args, w, ws, rank):
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.build()
    T = oracle.Tree(w.pos, w.mass, 2.8 * w.eps)
    rng = np.random.default_rng(11)
    per_step = args.ref_targets
    times, inters = [], []
    for it in range(args.warmup + args.steps):
        tg = rng.choice(w.n, per_step, replace=False)
        t0 = time.time()
        _, cnt = T.walk(w.r_s, w.rcut, args.theta, tg)
        dt = time.time() - t0
        if it >= args.warmup:
            times.append(dt)
            inters.append(int(cnt.sum()))
    value = sum(inters) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n": w.n, "theta": args.theta,
                       "step": f"oracle forward walk of {per_step} random targets"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} random targets per step, tree over all {w.n} particles "
                                       "built once (untimed); forward walk only", **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm

def timed_ms(fn, reps, flush, warm=0):
    """Mean CUDA-event time of fn over reps calls (L2 flushed before each)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sum(ts) / len(ts)


def side_workload(og, L, name, dev, theta, steps, flush):
    """Keys, tree, FP32 forward and adjoint walks on another workload (stream
    launches, L2 flushed): per-phase times and rates."""
    import ctypes as C
    import ics
    import torch
    w = ics.make(name)
    pos = torch.tensor(w.pos, device=dev)
    mass = torch.tensor(w.mass, device=dev)
    eps = torch.tensor(w.eps, device=dev)
    wt = torch.tensor(ics.loss_weights(w.n, 2002), dtype=torch.float32, device=dev)
    wsk = og._workspace(L.og_keys_sort_ws_bytes(w.n), dev)
    k, o = og.keys_sort(pos, w.box, ws=wsk)
    tree = og.tree_build(k, o, pos, mass, eps, w.box)
    ws = og._workspace(L.og_accel_ws_bytes(C.byref(tree.header), 0), dev)
    wsa = og._workspace(L.og_adjoint_ws_bytes(C.byref(tree.header), 1), dev)
    acc = torch.empty((w.n, 3), dtype=torch.float32, device=dev)
    tot = torch.zeros(1, dtype=torch.int64, device=dev)
    og.shortrange_accel(tree, w.r_s, theta, ws=ws, out=acc, total=tot)
    og.shortrange_adjoint(tree, w.r_s, theta, wt, ws=wsa)
    inter = int(tot.item())
    t_keys = timed_ms(lambda: og.keys_sort(pos, w.box, check=False, ws=wsk, keys=k, order=o), steps, flush)
    t_tree = timed_ms(lambda: og.tree_build(k, o, pos, mass, eps, w.box, check=False, mem=tree.mem), steps, flush)
    t_fwd = timed_ms(lambda: og.shortrange_accel(tree, w.r_s, theta, check=False, ws=ws, out=acc, total=tot),
                     steps, flush)
    t_adj = timed_ms(lambda: og.shortrange_adjoint(tree, w.r_s, theta, wt, check=False, ws=wsa), steps, flush)
    og.shortrange_accel_adjoint(tree, w.r_s, theta, wt, ws=wsa)
    t_fu = timed_ms(lambda: og.shortrange_accel_adjoint(tree, w.r_s, theta, wt, check=False, ws=wsa), steps, flush)
    step = t_keys + t_tree + t_fwd + t_adj
    return {"workload": f"{name}: {WORKLOADS[name]}", "n": w.n, "interactions_per_step": inter,
            "ms": {"keys_sort": t_keys, "tree_build": t_tree, "accel_fp32": t_fwd, "adjoint_fp32": t_adj,
                   "step": step, "fused_fwd_adjoint": t_fu},
            "interactions_per_s": inter / (step * 1e-3), "fwd_interactions_per_s": inter / (t_fwd * 1e-3),
            "adj_interactions_per_s": inter / (t_adj * 1e-3), "fwd_particles_per_s": w.n / (t_fwd * 1e-3),
            "timed_steps": steps, "launch": "stream launches, L2 flushed"}


def autograd_leg(og, dev, theta, steps, flush):
    """The adjoint configuration through torch.autograd: L = sum w . a on the
    128^3 clustered set with seeded w; ShortRangeAccel.forward runs keys,
    sort, tree and the forward walk, backward the adjoint walk and the
    push-down (decisions frozen).  Stream launches, L2 flushed."""
    import ics
    import torch
    w = ics.make("nfw128_adjoint")
    pos = torch.tensor(w.pos, device=dev, requires_grad=True)
    mass = torch.tensor(w.mass, device=dev, requires_grad=True)
    eps = torch.tensor(w.eps, device=dev)
    wt = torch.tensor(w.w, dtype=torch.float32, device=dev)

    def run():
        acc = og.ShortRangeAccel.apply(pos, mass, eps, w.box, w.r_s, theta)
        return torch.autograd.grad((acc * wt).sum(), (pos, mass))

    def run_fused():
        loss = og.ShortRangeLinearLoss.apply(pos, mass, eps, wt, w.box, w.r_s, theta)
        return torch.autograd.grad(loss, (pos, mass))

    run()
    run_fused()
    torch.cuda.synchronize()
    t = timed_ms(run, steps, flush)
    tf = timed_ms(run_fused, steps, flush)
    k, o = og.keys_sort(pos.detach(), w.box)
    tree = og.tree_build(k, o, pos.detach(), mass.detach(), eps, w.box)
    _, tot, _ = og.shortrange_accel(tree, w.r_s, theta)
    inter = int(tot.item())
    return {"workload": f"nfw128_adjoint: {WORKLOADS['nfw128_adjoint']}", "n": w.n, "interactions_per_pass": inter,
            "ms": t, "interactions_per_s": inter / (t * 1e-3), "particles_per_s": w.n / (t * 1e-3),
            "linear_loss_fused": {"ms": tf, "interactions_per_s": inter / (tf * 1e-3), "speedup": t / tf,
                                  "what": "ShortRangeLinearLoss: the same loss and gradients from one fused walk"},
            "timed_steps": steps,
            "what": "ShortRangeAccel.apply + torch.autograd.grad of sum(w . a) for pos and mass: keys, sort, "
                    "tree, forward walk; adjoint walk, push-down; stream launches, L2 flushed"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nfw256", choices=sorted(WORKLOADS))
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-targets", type=int, default=None,
                    help="oracle targets per reference-arm step (default: 1024, or 8192 for zeldovich128)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--side", default="zeldovich128,zoom8m",
                    help="other workloads timed beside the line (comma list, empty for none)")
    ap.add_argument("--no-graph", action="store_true", help="launch every kernel instead of replaying a CUDA graph")
    ap.add_argument("--scale", type=int, default=None,
                    help="a smaller instance of the workload (particles per side; for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.ref_targets is None:
        args.ref_targets = 8192 if args.workload == "zeldovich128" else 1024
    ws, rank, local = dist_env()

    import numpy as np
    import ics
    w = ics.make(args.workload, args.scale)

    if args.impl == "reference":
        return run_reference(args, w, ws, rank)

    import torch
    import __graft_entry__
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)  # before any collective: each rank on its own GPU
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        dist.barrier(device_ids=[local])
        __graft_entry__.build()
    import paper_2606_17145_gb300 as og
    L = og.lib()

    # resident inputs, preallocated outputs and workspaces (no allocation in the timed region)
    pos = torch.tensor(w.pos, dtype=torch.float64, device=dev)
    mass = torch.tensor(w.mass, dtype=torch.float64, device=dev)
    eps = torch.tensor(w.eps, dtype=torch.float64, device=dev)
    wt = torch.tensor(ics.loss_weights(w.n, 2002), dtype=torch.float32, device=dev)
    n = w.n
    ws_keys = og._workspace(L.og_keys_sort_ws_bytes(n), dev)
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    order = torch.empty(n, dtype=torch.int32, device=dev)
    p = og.params()
    import ctypes as C
    tree_mem = og._workspace(L.og_tree_bytes(n, C.byref(p)), dev)
    k0, o0 = og.keys_sort(pos, w.box, ws=ws_keys)
    tree = og.tree_build(k0, o0, pos, mass, eps, w.box, p=p, mem=tree_mem)
    ws_acc = og._workspace(L.og_accel_ws_bytes(C.byref(tree.header), 0), dev)
    ws_adj = og._workspace(L.og_adjoint_ws_bytes(C.byref(tree.header), 1), dev)
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    acc64 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    total64 = torch.zeros(1, dtype=torch.int64, device=dev)
    dpos = torch.empty((n, 3), dtype=torch.float64, device=dev)
    dmass = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    peaks = pipe_peaks(og, L, dev)

    state = {}

    def part_keys():
        state["ko"] = og.keys_sort(pos, w.box, check=False, ws=ws_keys, keys=keys, order=order)

    def part_tree():
        k, o = state["ko"]
        state["tree"] = og.tree_build(k, o, pos, mass, eps, w.box, p=p, check=False, mem=tree_mem)

    def part_accel():
        og.shortrange_accel(state["tree"], w.r_s, args.theta, check=False, ws=ws_acc, out=acc, total=total)

    def part_adjoint():
        og.shortrange_adjoint(state["tree"], w.r_s, args.theta, wt, check=False, ws=ws_adj, dpos=dpos, dmass=dmass)

    def step(ev=None):
        part_keys()
        if ev: ev[1].record()
        part_tree()
        if ev: ev[2].record()
        part_accel()
        if ev: ev[3].record()
        part_adjoint()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # The library never allocates or synchronises inside a call and its grids
    # are fixed (per-level sizes live on the device), so a whole step can be
    # captured once and replayed as one CUDA graph.
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()

    def run_step(ev=None):
        if graph is None or ev is not None:
            step(ev)
        else:
            graph.replay()
    for buf, name in ((ws_keys, "keys_sort"), (tree_mem, "tree_build"), (ws_acc, "accel"), (ws_adj, "adjoint")):
        code = og.poll_status(buf)
        if code != 0:
            raise SystemExit(f"{name} failed on the device: {L.og_status_str(code).decode()}")
    interactions = int(total.item())

    phases = ["keys_sort", "tree_build", "accel_fp32", "adjoint_fp32"]
    per = {k: [] for k in phases}
    step_ms = []
    if ws > 1:
        torch.distributed.barrier(device_ids=[local])
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall = time.time()
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            run_step()
            b.record()
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        wall = time.time() - t_wall
    # per-phase breakdown (separately launched steps with events between phases)
    for _ in range(min(args.steps, 3)):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        step(ev)
        ev[4].record()
        torch.cuda.synchronize()
        for i, k in enumerate(phases):
            per[k].append(ev[i].elapsed_time(ev[i + 1]))
    clocks = clk.summary()
    ms = max_over_ranks(sum(step_ms) / len(step_ms), ws, dev)
    value = job_rate(interactions, ws, ms)
    pms = {k: sum(v) / len(v) for k, v in per.items()}

    # end to end through the public API with host buffers
    pos_h = pos.cpu().pin_memory()
    mass_h = mass.cpu().pin_memory()
    eps_h = eps.cpu().pin_memory()
    wt_h = wt.cpu().pin_memory()
    acc_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    dpos_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    dmass_h = torch.empty(n, dtype=torch.float64).pin_memory()
    h2d = pos_h.numel() * 8 + mass_h.numel() * 8 + eps_h.numel() * 8 + wt_h.numel() * 4
    d2h = acc_h.numel() * 4 + dpos_h.numel() * 8 + dmass_h.numel() * 8

    # End to end, pipelined over steps as a production loop runs it: two
    # device buffer sets; step k+1's inputs go up on one copy stream while
    # step k computes on the other set, and step k's results come down on a
    # second copy stream while step k+1 computes.  Every step's copies lie
    # inside the timed region; the first upload and the last download are
    # exposed.  (The steps are independent: the same synthetic set each time.)
    up = torch.cuda.Stream(device=dev)
    down = torch.cuda.Stream(device=dev)
    sets = []
    for si in range(2):
        if si == 0:
            S = dict(pos=pos, mass=mass, eps=eps, wt=wt, acc=acc, dpos=dpos, dmass=dmass)
        else:
            S = {k: torch.empty_like(v) for k, v in
                 dict(pos=pos, mass=mass, eps=eps, wt=wt, acc=acc, dpos=dpos, dmass=dmass).items()}
        for e in ("ev_in", "ev_acc", "ev_done", "ev_out"):
            S[e] = torch.cuda.Event()
        S["used"] = False
        sets.append(S)

    def upload(S):
        with torch.cuda.stream(up):
            if S["used"]:
                up.wait_event(S["ev_done"])      # the set's last step has read its inputs
            S["pos"].copy_(pos_h, non_blocking=True)
            S["mass"].copy_(mass_h, non_blocking=True)
            S["eps"].copy_(eps_h, non_blocking=True)
            S["wt"].copy_(wt_h, non_blocking=True)
            S["ev_in"].record(up)

    def compute(S):
        main = torch.cuda.current_stream()
        main.wait_event(S["ev_in"])
        if S["used"]:
            main.wait_event(S["ev_out"])         # the set's last results are on the host
        flush.zero_()
        k, o = og.keys_sort(S["pos"], w.box, check=False, ws=ws_keys, keys=keys, order=order)
        tr = og.tree_build(k, o, S["pos"], S["mass"], S["eps"], w.box, p=p, check=False, mem=tree_mem)
        og.shortrange_accel(tr, w.r_s, args.theta, check=False, ws=ws_acc, out=S["acc"], total=total)
        S["ev_acc"].record(main)
        og.shortrange_adjoint(tr, w.r_s, args.theta, S["wt"], check=False, ws=ws_adj, dpos=S["dpos"],
                              dmass=S["dmass"])
        S["ev_done"].record(main)
        S["used"] = True

    def download(S):
        with torch.cuda.stream(down):
            down.wait_event(S["ev_acc"])
            acc_h.copy_(S["acc"], non_blocking=True)
            down.wait_event(S["ev_done"])
            dpos_h.copy_(S["dpos"], non_blocking=True)
            dmass_h.copy_(S["dmass"], non_blocking=True)
            S["ev_out"].record(down)

    def run_e2e(nsteps):
        main = torch.cuda.current_stream()
        upload(sets[0])
        for k in range(nsteps):
            compute(sets[k % 2])
            if k + 1 < nsteps:
                upload(sets[(k + 1) % 2])
            download(sets[k % 2])
        main.wait_stream(up)
        main.wait_stream(down)

    run_e2e(2)
    torch.cuda.synchronize()
    e2e_steps = min(args.steps, 6)
    with Clocks(local) as clk_e2e:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run_e2e(e2e_steps)
        b.record()
        torch.cuda.synchronize()
    e2e_ms = [a.elapsed_time(b) / e2e_steps]
    e2e_mean = max_over_ranks(sum(e2e_ms) / len(e2e_ms), ws, dev)

    # FP64 walk on the same tree (comparison variant)
    tr = state["tree"]
    f64 = []
    for _ in range(max(1, args.fp64_steps)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        og.shortrange_accel(tr, w.r_s, args.theta, prec="fp64", check=False, ws=ws_acc, out=acc64, total=total64)
        b.record()
        torch.cuda.synchronize()
        f64.append(a.elapsed_time(b))
    f64_ms = sum(f64) / len(f64)
    inter64 = int(total64.item())
    code = og.poll_status(ws_acc)
    if code != 0:
        raise SystemExit(f"fp64 walk failed on the device: {L.og_status_str(code).decode()}")
    # the FP32 accelerations of the same tree (the graph's last replay wrote acc)
    og.shortrange_accel(tr, w.r_s, args.theta, ws=ws_acc, out=acc, total=total)
    rel = (acc.double() - acc64).norm(dim=1) / acc64.norm(dim=1).clamp_min(1e-300)
    fp32_vs_fp64 = {"rms_rel": float(rel.pow(2).mean().sqrt()), "max_rel": float(rel.max())}
    acc_host = acc.double().cpu().numpy()

    # fused forward + adjoint (one walk; a loss whose weights are known before
    # the forces): timed on the same tree, its accelerations checked against
    # the separate forward walk's bit for bit
    acc_fu = torch.empty_like(acc)
    total_fu = torch.zeros(1, dtype=torch.int64, device=dev)
    og.shortrange_accel_adjoint(tr, w.r_s, args.theta, wt, ws=ws_adj, out=acc_fu, total=total_fu, dpos=dpos,
                                dmass=dmass)
    fu_ms = timed_ms(lambda: og.shortrange_accel_adjoint(tr, w.r_s, args.theta, wt, check=False, ws=ws_adj,
                                                         out=acc_fu, total=total_fu, dpos=dpos, dmass=dmass),
                     max(1, min(args.steps, 3)), flush)
    fu_ms = max_over_ranks(fu_ms, ws, dev)
    fused = {"ms": fu_ms, "interactions_per_s": ws * interactions / (fu_ms * 1e-3),
             "separate_ms": pms["accel_fp32"] + pms["adjoint_fp32"],
             "speedup_vs_separate": (pms["accel_fp32"] + pms["adjoint_fp32"]) / fu_ms,
             "same_acc_bits": bool(torch.equal(acc_fu.view(torch.int32), acc.view(torch.int32))),
             "same_interactions": int(total_fu.item()) == interactions,
             "what": "og_shortrange_accel_adjoint: the adjoint walk that also writes the accelerations, "
                     "plus the push-down; L2 flushed"}
    del acc_fu

    # roofline of the dominant kernel.  "peak" is the unit-count FP32 peak
    # (SMs x 128 FMA lanes x 2 flops x the maximum SM clock); the pipe rates
    # measured above give the "_measured" fractions and the MUFU and FP64 ones.
    mp = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(mp.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    kern = {}
    for kname, kms, fl, fli in (("accel_fp32", pms["accel_fp32"], FWD_FLOPS, FWD_FLOPS_IMPL),
                                ("adjoint_fp32", pms["adjoint_fp32"], ADJ_FLOPS, ADJ_FLOPS_IMPL)):
        rate = interactions / (kms * 1e-3)
        tf = rate * fl / 1e12
        kern[kname] = {"ms": kms, "interactions_per_s": rate, "tflops_algorithmic": tf,
                       "tflops_implemented": rate * fli / 1e12, "frac_fp32": tf / alu_peak,
                       "frac_fp32_measured": tf / peaks["fp32_tflops"],
                       "mufu_per_s": rate * MUFU_PER_INTERACTION,
                       "frac_xu": rate * MUFU_PER_INTERACTION / peaks["mufu_per_s"]}
    r64 = inter64 / (f64_ms * 1e-3)
    kern["accel_fp64"] = {"ms": f64_ms, "interactions_per_s": r64, "tflops_algorithmic": r64 * FP64_FLOPS / 1e12,
                          "frac_fp64_measured": r64 * FP64_FLOPS / 1e12 / peaks["fp64_tflops"]}
    dom = max(("accel_fp32", "adjoint_fp32"), key=lambda k: kern[k]["ms"])
    dk = kern[dom]
    traffic = None if args.scale else walk_traffic("forward" if dom == "accel_fp32" else "adjoint", args.workload)
    roofline = {"bound": "alu", "achieved": dk["tflops_algorithmic"], "peak": alu_peak, "unit": "TFLOP/s",
                "frac": dk["tflops_algorithmic"] / alu_peak, "traffic": traffic, "kernel": dom,
                "flops_per_interaction": ADJ_FLOPS if dom == "adjoint_fp32" else FWD_FLOPS,
                "flops_per_interaction_implemented": ADJ_FLOPS_IMPL if dom == "adjoint_fp32" else FWD_FLOPS_IMPL,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 flops x {sm_max:.0f} MHz (max SM clock)",
                "frac_measured": dk["frac_fp32_measured"], "frac_xu": dk["frac_xu"],
                "measured_peaks": peaks, "kernels": kern}

    launches = og.LAUNCHES_PER_CALL
    per_step_launches = (launches["keys_sort"] + launches["tree_build"] + launches["accel"] +
                         launches["adjoint"])

    # the PM long-range complement on the same particles: a separate measurement,
    # not part of the step above (mesh of 1.25 box / r_s cells per side, so that
    # r_s is 1.25 mesh cells)
    pm_n = int(round(1.25 * w.box / w.r_s))
    plan = og.PMPlan(pm_n)
    ws_pm = og._workspace(plan.ws_bytes, dev)
    acc_pm = torch.empty((n, 3), dtype=torch.float32, device=dev)
    og.pm_accel(plan, pos, mass, w.box, w.r_s, ws=ws_pm, out=acc_pm)  # checked once
    pm_local = timed_ms(lambda: og.pm_accel(plan, pos, mass, w.box, w.r_s, check=False, ws=ws_pm, out=acc_pm),
                        max(1, min(args.steps, 10)), flush, warm=args.warmup)
    pm_ms = max_over_ranks(pm_local, ws, dev)
    plan.close()
    del ws_pm, acc_pm

    # one device-resident kick-drift-kick step (kick, drift, keys, tree, FP32
    # walk, PM mesh, kick) on copies of the inputs; reported beside the line,
    # never in place of it
    kdk = None
    try:
        vel0 = torch.zeros_like(pos)
        S = og.TreePMStepper(pos.clone(), vel0, mass, eps, w.box, w.r_s, args.theta, pm_n)
        kdk_local = timed_ms(lambda: S.step(1e-4, check=False), max(1, min(args.steps, 3)), flush, warm=1)
        S.poll()
        S.close()
        del S, vel0
    except Exception as e:  # the headline line must still be printed
        kdk_local, kdk = float("inf"), {"error": f"{type(e).__name__}: {e}"}
    # every rank takes part in the max, whether or not its leg failed
    kdk_ms = max_over_ranks(kdk_local, ws, dev)
    if kdk is None:
        kdk = ({"ms": kdk_ms, "particles_per_s": ws * n / (kdk_ms * 1e-3), "ngrid": pm_n,
                "what": "TreePMStepper.step: kick, drift, keys + sort, tree, FP32 walk, PM mesh, kick; "
                        "stream launches (no graph), L2 flushed"}
               if kdk_ms < float("inf") else {"error": "failed on another rank"})

    # SPH density and smoothing length on the same tree, reported beside the line
    sph = None
    try:
        n_ngb = 32.0
        og.sph_density(tree, n_ngb)  # warm-up, checked
        sph_local = timed_ms(lambda: og.sph_density(tree, n_ngb, check=False), 1, flush)
    except Exception as e:  # the headline line must still be printed
        sph_local, sph = float("inf"), {"error": f"{type(e).__name__}: {e}"}
    sph_ms = max_over_ranks(sph_local, ws, dev)
    if sph is None:
        sph = ({"ms": sph_ms, "particles_per_s": ws * n / (sph_ms * 1e-3), "n_ngb": n_ngb,
                "what": "og_sph_density: grouped tree gather, smoothing length by FP32 Newton steps and one FP64 step, density"}
               if sph_ms < float("inf") else {"error": "failed on another rank"})

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}"
                               + (f" (scaled down: {args.scale} per side)" if args.scale else ""),
                   "n": n, "theta": args.theta,
                   "step": "keys_sort + tree_build + accel_fp32 + adjoint_fp32 (inputs resident)",
                   "l2": "inputs larger than L2; also flushed by a 256 MiB write between timed steps",
                   "parallelism": f"replicas x{ws}",
                   "launch": "CUDA graph replay of the whole step" if graph is not None else "stream launches"},
        "clocks": clocks,
        "e2e": {"value": job_rate(interactions, ws, e2e_mean), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_mean, "steps": e2e_steps,
                "pipelined": "two device buffer sets: step k+1's upload and step k's download overlap the "
                             "neighbouring steps' kernels on two copy streams; stream launches",
                "clocks": clk_e2e.summary()},
        "gpu_launches": per_step_launches * args.steps,
        "roofline": roofline,
        "interactions_per_step": interactions,
        "particles_per_s": ws * n / (ms * 1e-3),
        "fwd_interactions_per_s": ws * interactions / (pms["accel_fp32"] * 1e-3),
        "fwd_particles_per_s": ws * n / (pms["accel_fp32"] * 1e-3),
        "adj_interactions_per_s": ws * interactions / (pms["adjoint_fp32"] * 1e-3),
        "fwd_adj_particles_per_s": ws * n / ((pms["accel_fp32"] + pms["adjoint_fp32"]) * 1e-3),
        "breakdown_ms": pms,
        "fused_fwd_adjoint": fused,
        "fp64": {"ms": f64_ms, "interactions_per_s": ws * inter64 / (f64_ms * 1e-3),
                 "same_interactions": inter64 == interactions,
                 "fp32_speedup": f64_ms / pms["accel_fp32"], "fp32_vs_fp64": fp32_vs_fp64},
        "wall_s": wall,
        "kdk_step": kdk,
        "sph_density": sph,
        "pm": {"ngrid": pm_n, "ms": pm_ms, "particles_per_s": ws * n / (pm_ms * 1e-3),
               "what": "og_pm_accel: CIC deposit, cuFFT R2C, Green's function, cuFFT C2R, "
                       "difference + interpolation; FP32 mesh; timed apart from the step, L2 flushed"},
    }
    del ws_adj, dpos, dmass, acc64
    torch.cuda.empty_cache()

    # other workloads, timed beside the line
    side = {}
    for name in [x for x in args.side.split(",") if x]:
        if name == args.workload or name not in WORKLOADS:
            continue
        try:
            side[name] = side_workload(og, L, name, dev, args.theta, 1 if name == "zoom8m" else 5, flush)
        except Exception as e:
            side[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    line["other_workloads"] = side
    if args.side:  # beside the other workloads (skipped with --side=)
        try:
            line["adjoint_autograd"] = autograd_leg(og, dev, args.theta, 3, flush)
        except Exception as e:
            line["adjoint_autograd"] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.time()
        T = oracle.Tree(w.pos, w.mass, 2.8 * w.eps)
        build_s = time.time() - t0
        v, pps, sample, tg, a_or = oracle_throughput(w, args.theta, T=T)
        sample = sample.replace("built once, 0.0 s", f"built once, {build_s:.1f} s")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                "particles_per_s": pps, **host_info()}
        # error against the FP64 oracle: the tree at the same theta on the
        # sampled targets, the direct sum on a time-bounded subset of them
        acc_or = {"vs_oracle_tree": rel_stats(acc_host[tg], a_or)}
        dt_, done, ad_l = 0.0, 0, []
        while done < len(tg) and (dt_ < 8.0 or done < 256):
            t1 = time.time()
            ad, _ = oracle.direct(w.pos, w.mass, 2.8 * w.eps, w.box, w.r_s, w.rcut, tg[done:done + 64])
            dt_ += time.time() - t1
            ad_l.append(ad)
            done += 64
        acc_or["vs_oracle_direct"] = rel_stats(acc_host[tg[:done]], np.concatenate(ad_l))
        acc_or["oracle_tree_vs_direct"] = rel_stats(a_or[:done], np.concatenate(ad_l))
        acc_or["c1"] = accuracy_c1(og, dev)
        acc_or["how"] = (f"per-particle |a_gpu - a_ref| / |a_ref| of the FP32 walk at theta = {args.theta}; "
                         "vs_oracle_tree on the CPU baseline's sampled targets, vs_oracle_direct on the first "
                         "of them (the direct sum's time bound), c1 on the 4096-particle uniform set")
        line["accuracy"] = acc_or
        T.close()
    if ws > 1:
        torch.distributed.barrier(device_ids=[local])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
