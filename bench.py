#!/usr/bin/env python3
"""Benchmark of the CLOSURE hot path on GB300.

One step = one pass of the whole hot path over one synthetic 2D-3D PURSE
(N = 16 keypoints, pinhole 600/600/320/240): centre statistics, 2^20 walks of
the rotation-boundary sampler and 2^20 walks of the translation-boundary
sampler (N_I = 100, N_P = 150, N_P* = 10, N_T = 15, FP32), then the two
minimum enclosing geodesic balls (200 GGD iterations each).

Printed JSON line: value = pose-constraint evaluations per second in the
algorithm's own count (Alg. 3/5 evaluate N_P perturbed poses and N_P* x N_T
ladder poses against all N constraints per walk iteration), whole job; the
evaluations the kernels actually executed (the ladder stops at the first
feasible rung and at the first violated constraint) are reported beside it and
price the roofline of the dominant walk kernel against the FP32 ALU peak;
e2e through the C ABI with host buffers; the FP64 oracle timed on the host
cores as cpu_baseline.  ``--impl reference`` times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MEGB solves/sec & pose-constraint evals/sec vs plain GPU path; % FP32 roofline"
UNIT = "evals/s"
N_KEYPOINTS = 16
N_WALKS = 1 << 20
N_ITER = 100
K_MEGB = 200
PURSE_SEED = 0
# algorithmic flops per (pose, constraint) evaluation of a 2D-3D constraint: the full transform,
# projection and test, 24 for in_purse (11 FFMA + 2 FMUL) and 28 for the margin of eq. 11
# (plus a square root, a division and two operations)
FLOPS_DIST, FLOPS_INPURSE = 28, 24
N_PERTURB, N_KEEP, N_STEPS = 150, 10, 15
SM_COUNT_NOMINAL = 152
# DRAM bytes (read + write) per launch of each walk kernel on this workload, from one ncu capture of the
# timed step's two walk launches: ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
# -k regex:walk_kernel -s 6 -c 2 python bench.py --steps 2 --warmup 3 --no-e2e --no-batch --no-cpu-baseline
# --no-plain --no-grad --no-c1 --no-tune (one pass).  The counters belong to the kernel built from the sources
# whose SHA-256 (walk.cu, dev.cuh, internal.h concatenated) begins with WALK_DRAM_SRC; any other source gives
# traffic null.
WALK_DRAM_BYTES = {"R": 438272 + 768, "t": 914944 + 0}
WALK_DRAM_SRC = "20892b8d1bfbb92d"
FP32_LANES_PER_SM = 128
# C1: 3D-3D PURSE (N = 8, seed 0) in FP64, |S0| = 2048 RANSAG seeds, N_W = 2 walks each (4096 samples of the
# dS_R sampler, N_I = 5, 3DMatch preset), both balls with K = 200; flops per 3D-3D evaluation: 26 for in_purse
# (R a + t - b, the squared norm and the test) and 28 for the margin of eq. 11
C1_N, C1_SEEDS, C1_NW, C1_ITERS, C1_K = 8, 2048, 2, 5, 200
FLOPS_DIST_3D, FLOPS_INPURSE_3D = 28, 26
# FP64 FMA results per clock per SM of this part (GB300: 1.25 TFLOP/s over 152 SMs at about 2 GHz)
FP64_FMA_PER_SM = 2


def walk_traffic(kern):
    """The captured DRAM bytes per launch of the walk kernel, or None if its sources changed since."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2403_09990_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("walk.cu", "dev.cuh", "internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return WALK_DRAM_BYTES[kern] if h.hexdigest()[:16] == WALK_DRAM_SRC else None


def workload_config():
    return {
        "workload": "2D-3D PURSE N=16 (pinhole 600/600/320/240, r_i~U[2,10] px, depth U[0.5,1.5] m); "
                    f"{N_WALKS} walks per sampler x {N_ITER} iterations (N_P=150, N_P*=10, N_T=15); "
                    "rotation + translation MEGB, 200 GGD iterations",
        "n_keypoints": N_KEYPOINTS, "walks_per_sampler": N_WALKS, "n_iter": N_ITER, "megb_iters": K_MEGB,
        "precision": "fp32 walk arithmetic, fp64 centre statistics and ball centres",
        "l2": "flushed between timed steps (512 MB write)", "data": "synthetic (seeded)",
    }


def make_purse(rank=0):
    from paper_2403_09990_gb300 import synthetic as syn
    return syn.purse_2d3d(N_KEYPOINTS, PURSE_SEED + rank)


def closure_params(sampler, n_iter=None, precision=0):
    import paper_2403_09990_gb300.purse as P
    return P.make_params(n_iter=N_ITER if n_iter is None else n_iter, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=2.0, gamma=0.5,
                         rot_perturb=0.2, trans_perturb=0.1, perturb_units=0, sampler=sampler, precision=precision)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle
def _oracle_chunk(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sampler, walk_ids, n_iter, rank = args
    from oracle import closure
    p = make_purse(rank)
    prm = closure.preset_2d3d(n_iter=n_iter)
    seeds = p.seed_pose()[None]
    t0 = time.perf_counter()
    if sampler == 0:
        R, t = closure.sample_rotation_boundary(p, seeds, prm, 1000, np.asarray(walk_ids))
    else:
        R, t = closure.sample_translation_boundary(p, seeds, prm, 1000, np.asarray(walk_ids))
    dt = time.perf_counter() - t0
    q, t = closure.as_samples(R, t)
    # the oracle evaluates every perturbation and the full ladder (Alg. 3/5 as written)
    evals = len(walk_ids) * n_iter * (prm.n_perturb + prm.n_keep * prm.n_steps) * p.n
    return evals, dt, q, t


def oracle_sample(walks_per_worker, workers, n_iter=None, rank=0):
    """The oracle on a bounded sample of the workload: both samplers, then both balls."""
    import multiprocessing as mp
    n_iter = N_ITER if n_iter is None else n_iter
    from oracle import megb as om
    ctx = mp.get_context("spawn")
    jobs = []
    for s in (0, 1):
        for k in range(workers):
            ids = list(range(k * walks_per_worker, (k + 1) * walks_per_worker))
            jobs.append((s, ids, n_iter, rank))
    with ctx.Pool(workers) as pool:
        pool.map(_warm, range(workers))
        t0 = time.perf_counter()
        out = pool.map(_oracle_chunk, jobs)
        qs = np.concatenate([o[2] for o, j in zip(out, jobs) if j[0] == 0])
        ts = np.concatenate([o[3] for o, j in zip(out, jobs) if j[0] == 1])
        om.megb_rotation(qs, K_MEGB)
        om.megb_translation(ts, K_MEGB)
        wall = time.perf_counter() - t0
    evals = sum(o[0] for o in out)
    return evals, wall, 2 * workers * walks_per_worker


def _warm(_):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle.closure  # noqa: F401
    return 0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- GPU arm
def combine_ranks(t_step, evals, dist, device):
    """Whole-job step time and executed evaluations of replicas: the largest per-rank step time (every rank
    ends its timed region before the slowest one) and the sum of the per-rank evaluations.  dist is the
    initialised torch.distributed module (None for one process)."""
    if dist is None:
        return t_step, float(evals)
    import torch
    tt = torch.tensor([t_step], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ee = torch.tensor([float(evals)], device=device, dtype=torch.float64)
    dist.all_reduce(ee)
    return float(tt.item()), float(ee.item())


def run_gpu(args, rank, world):
    import torch
    import paper_2403_09990_gb300.purse as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    P.lib(build_if_missing=True)
    p = make_purse(rank)
    stream = torch.cuda.current_stream()
    hR, hT = P.Purse(p), P.Purse(p)
    seeds = torch.as_tensor(p.seed_pose()[None], dtype=torch.float64, device=dev)
    qR = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tR = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    qT = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tT = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    pR, pT = closure_params(0), closure_params(1)
    launches_per_step = 2 + 2 + 3
    # autotuner: launch shapes measured on this workload (walks with 10 iterations: the shape depends on
    # the kind, N and the sample count, not on the iteration count) and used by the timed step
    tuning = None if args.no_tune else run_tune(hR, hT, seeds, qR, tR, qT, tT, res, stream)

    def step(seed, ev=None):
        if ev:
            ev[0].record(stream)
        P.purse_sample(hR.h, pR, seed, seeds, 1, N_WALKS, qR, tR, None, stream)
        if ev:
            ev[1].record(stream)
        P.purse_sample(hT.h, pT, seed, seeds, 1, N_WALKS, qT, tT, None, stream)
        if ev:
            ev[2].record(stream)
        P.megb_solve(hR.h, 0, K_MEGB, qR, N_WALKS, tT, N_WALKS, res, None, stream)
        if ev:
            ev[3].record(stream)

    for w in range(args.warmup):
        flush.fill_(w & 0xFF)
        step(100 + w)
    P.purse_sync(hR.h, stream)
    P.purse_sync(hT.h, stream)
    evals_dist = N_WALKS * N_ITER * N_PERTURB * p.n
    evals_alg = 2 * N_WALKS * N_ITER * (N_PERTURB + N_KEEP * N_STEPS) * p.n  # both samplers, per step
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    t_wall = time.perf_counter()
    rows = []
    for s in range(args.steps):
        flush.fill_(s & 0xFF)  # untimed: L2 flush between timed steps
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        step(1000 + s, ev)
        eR = P.purse_last_evals(hR.h, stream)
        eT = P.purse_last_evals(hT.h, stream)
        rows.append((ev, eR, eT))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    ck = clocks.stop()
    P.purse_sync(hR.h, stream)
    P.purse_sync(hT.h, stream)
    tot = walkR = walkT = ggd = 0.0
    evals = evR = evT = 0
    for ev, eR, eT in rows:
        a, b, c, d = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                      ev[0].elapsed_time(ev[3]))
        walkR += a
        walkT += b
        ggd += c
        tot += d
        evals += eR + eT
        evR += eR
        evT += eT
    t_step, evals_all = combine_ranks(tot / args.steps / 1e3, evals, dist, dev)
    value = evals_alg * world / t_step
    executed_per_s = evals_all / (t_step * args.steps)
    # roofline of the dominant kernel (the slower of the two walk kernels)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    kern = "t" if walkT >= walkR else "R"
    ev_k = evT if kern == "t" else evR
    ms_k = (walkT if kern == "t" else walkR) / args.steps
    dist_k = evals_dist * args.steps
    flops_k = (dist_k * FLOPS_DIST + (ev_k - dist_k) * FLOPS_INPURSE) / args.steps
    achieved = flops_k / (ms_k / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": dict(workload_config(), parallelism="replicas" if world > 1 else "single"),
        "megb_solves_per_s": world / t_step, "samples_per_s": 2 * N_WALKS * world / t_step,
        "evals_executed_per_s": executed_per_s,
        "value_counts": "Alg. 3/5 evaluations: (N_P + N_P* N_T) N per walk iteration, both samplers",
        "breakdown_ms": {"walk_dS_R": walkR / args.steps, "walk_dS_t": walkT / args.steps, "megb": ggd / args.steps},
        "evals_per_step": {"dS_R": evR / args.steps, "dS_t": evT / args.steps},
        "roofline": {"bound": "alu", "kernel": f"walk_kernel<float, 2D-3D, dS_{kern}>", "achieved": achieved,
                     "flops_per_eval": {"dist": FLOPS_DIST, "in_purse": FLOPS_INPURSE},
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": walk_traffic(kern), "traffic_unit": "bytes per launch",
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {clock_mhz:.0f} MHz (max SM clock)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck, "wall_s_timed": wall,
    }
    if tuning is not None:
        out["tuning"] = tuning
    out["megb_exact"] = run_exact(hR, qR, tT, res, dev)
    out["ransag"] = run_ransag(dev)
    if not args.no_c1:
        out["c1"] = run_c1(dev, sms, clock_mhz, with_oracle=rank == 0 and not args.no_cpu_baseline,
                           tune=not args.no_tune)
    if not args.no_plain:
        out["plain_gpu"] = run_plain(args, p, dev, seeds, value / world, t_step)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = run_e2e(args, p, dev)
    if not args.no_batch:
        out["batch"] = run_batch(args, dev)
    if not args.no_grad:
        out["grad"] = run_grad(args, dev)
    if rank == 0 and not args.no_cpu_baseline:
        ev_c, wall_c, walks_c = oracle_sample(args.cpu_walks, args.cpu_workers)
        out["cpu_baseline"] = {"value": ev_c / wall_c, "unit": UNIT, "cores": args.cpu_workers, "kind": "oracle",
                               "sample": f"{walks_c} walks ({args.cpu_walks} per worker, both samplers, N_I={N_ITER}) "
                                         f"+ both balls (200 GGD iterations); {wall_c:.1f} s"}
    hR.close()
    hT.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_ransag(dev):
    """Step I on the GPU, timed by the wall clock around the call (it synchronises): P3P RANSAG on the
    bench's 2D-3D PURSE (N = 16) and Arun/Horn RANSAG on a 3D-3D PURSE (N = 8), 2^20 trials each (up to
    2^20 seeds kept, so every trial runs)."""
    import torch
    import paper_2403_09990_gb300.purse as P
    from paper_2403_09990_gb300 import synthetic as syn
    trials = 1 << 20
    seeds = torch.empty((trials, 12), dtype=torch.float64, device=dev)
    out = {}
    for name, p in (("2d3d_p3p", syn.purse_2d3d(N_KEYPOINTS, PURSE_SEED)), ("3d3d_arun", syn.purse_3d3d(8, 0))):
        with P.Purse(p) as h:
            try:
                P.purse_ransag(h.h, 1, 1 << 16, trials, seeds)       # warm-up
            except P.PurseError:
                pass
            t0 = time.perf_counter()
            try:
                n = P.purse_ransag(h.h, 2, trials, trials, seeds)
            except P.PurseError:                                     # no trial inside the PURSE
                n = 0
            dt = time.perf_counter() - t0
        out[name] = {"trials": trials, "ms": dt * 1e3, "trials_per_s": trials / dt, "seeds": n}
    return out


def run_tune(hR, hT, seeds, qR, tR, qT, tT, res, stream):
    """purse_tune_walk for both walk kernels and purse_tune_megb for the two balls of the step: the
    chosen shape and its time beside the default shape's (CUDA events; the walks with 10 iterations)."""
    import paper_2403_09990_gb300.purse as P
    out = {}
    for key, h, smp, q, t in (("walk_dS_R", hR, 0, qR, tR), ("walk_dS_t", hT, 1, qT, tT)):
        r = P.purse_tune_walk(h.h, closure_params(smp, n_iter=10), 5, seeds, 1, N_WALKS, q, t, stream)
        out[key] = {"shape": "warps per block", "config": r["config"], "ms": r["ms"],
                    "default_config": r["default_config"], "default_ms": r["default_ms"], "n_iter": 10}
    r = P.purse_tune_megb(hR.h, 0, K_MEGB, qR, N_WALKS, tT, N_WALKS, res, stream)
    out["megb"] = {"shape": "samples per thread (blocks per ball)", "config": r["config"], "ms": r["ms"],
                   "default_config": r["default_config"], "default_ms": r["default_ms"]}
    return out


def run_c1(dev, sms, clock_mhz, with_oracle, tune=True):
    """Config C1 end to end in FP64 on the GPU: RANSAG to |S0| = 2048 seeds (wall clock around its
    synchronising call), 4096 dS_R walks of N_I = 5 and both balls with K = 200 (CUDA events), per solve;
    the walk kernel's executed evaluations (28 / 26 FLOP) against the FP64 FMA rate of the part; beside it
    the oracle on the same workload (one host core, FP64) with its balls.  With tune, the autotuner first
    picks the walk's warps per block and the balls' blocks for this workload (reported beside the
    defaults)."""
    import torch
    import paper_2403_09990_gb300.purse as P
    from paper_2403_09990_gb300 import synthetic as syn
    stream = torch.cuda.current_stream()
    p = syn.purse_3d3d(C1_N, 0)
    prm = P.make_params(n_iter=C1_ITERS, n_perturb=N_PERTURB, n_keep=N_KEEP, n_steps=N_STEPS, omega0=0.5, v0=0.0,
                        gamma=0.5, rot_perturb=0.0, trans_perturb=0.1, perturb_units=0, sampler=0, precision=1)
    S = C1_SEEDS * C1_NW
    seeds = torch.empty((C1_SEEDS, 12), dtype=torch.float64, device=dev)
    q = torch.empty((S, 4), dtype=torch.float64, device=dev)
    t = torch.empty((S, 3), dtype=torch.float64, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    rows = []
    tuning = None
    with P.Purse(p) as h:
        if tune:
            s0 = P.purse_ransag(h.h, 1, 1 << 20, C1_SEEDS, seeds)
            rw = P.purse_tune_walk(h.h, prm, 3, seeds, s0, S, q, t, stream)
            rb = P.purse_tune_megb(h.h, 1, C1_K, q, S, t, S, res, stream)
            tuning = {"walk": {"shape": "warps per block", "config": rw["config"], "ms": rw["ms"],
                               "default_config": rw["default_config"], "default_ms": rw["default_ms"]},
                      "megb": {"shape": "samples per thread (blocks per ball)", "config": rb["config"], "ms": rb["ms"],
                               "default_config": rb["default_config"], "default_ms": rb["default_ms"]}}
        for r in range(4):
            t0 = time.perf_counter()
            s0 = P.purse_ransag(h.h, 1, 1 << 20, C1_SEEDS, seeds)
            ransag_ms = (time.perf_counter() - t0) * 1e3
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            P.purse_sample(h.h, prm, 3, seeds, s0, S, q, t, None, stream)
            e[1].record(stream)
            P.megb_solve(h.h, 1, C1_K, q, S, t, S, res, None, stream)
            e[2].record(stream)
            ev = P.purse_last_evals(h.h, stream)
            P.purse_sync(h.h, stream)
            if r:
                rows.append((ransag_ms, e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), ev))
        x = res.cpu().numpy()
    ransag_ms = statistics.median(r[0] for r in rows)
    walk_ms = statistics.median(r[1] for r in rows)
    ball_ms = statistics.median(r[2] for r in rows)
    ev = rows[-1][3]
    dist = S * C1_ITERS * N_PERTURB * C1_N
    flops = dist * FLOPS_DIST_3D + (ev - dist) * FLOPS_INPURSE_3D
    peak = sms * FP64_FMA_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    achieved = flops / (walk_ms / 1e3) / 1e12
    solve_ms = ransag_ms + walk_ms + ball_ms
    alg = S * C1_ITERS * (N_PERTURB + N_KEEP * N_STEPS) * C1_N
    out = {"workload": "3D-3D PURSE N=8 (seed 0), FP64: RANSAG to 2048 seeds, 4096 dS_R walks (N_I=5, N_P=150, "
                       "N_P*=10, N_T=15), rotation + translation MEGB, 200 GGD iterations",
           "ms_per_solve": solve_ms, "solves_per_s": 1e3 / solve_ms,
           "breakdown_ms": {"ransag": ransag_ms, "walk": walk_ms, "megb": ball_ms},
           "evals_per_s": alg / (walk_ms / 1e3), "evals_executed_per_s": ev / (walk_ms / 1e3),
           "D_hat": float(x[7]), "d_hat": float(x[8]),
           "roofline": {"bound": "fp64 alu", "kernel": "walk_kernel<double, 3D-3D, dS_R>", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "flops_per_eval": {"dist": FLOPS_DIST_3D, "in_purse": FLOPS_INPURSE_3D},
                        "peak_source": f"{sms} SMs x {FP64_FMA_PER_SM} FP64 FMA x 2 x {clock_mhz:.0f} MHz"}}
    if tuning is not None:
        out["tuning"] = tuning
    if with_oracle:
        from oracle import closure, megb as om, ransag
        t0 = time.perf_counter()
        seeds_o, _ = ransag.ransag_3d3d(p, 1, 1 << 20, C1_SEEDS)
        t1 = time.perf_counter()
        R, tt = closure.sample_rotation_boundary(p, seeds_o, closure.preset_3d3d(n_iter=C1_ITERS), 3, np.arange(S))
        t2 = time.perf_counter()
        qo, to = closure.as_samples(R, tt)
        _, Do, _ = om.megb_rotation(qo, C1_K)
        _, do, _ = om.megb_translation(to, C1_K)
        t3 = time.perf_counter()
        out["cpu_baseline"] = {"ms_per_solve": (t3 - t0) * 1e3, "breakdown_ms": {"ransag": (t1 - t0) * 1e3,
                               "walk": (t2 - t1) * 1e3, "megb": (t3 - t2) * 1e3},
                               "evals_per_s": alg / (t2 - t1), "cores": 1, "kind": "oracle",
                               "sample": "the whole C1 solve", "D_hat": float(Do), "d_hat": float(do)}
        out["gpu_over_oracle"] = (t3 - t0) * 1e3 / solve_ms
    return out


def run_exact(h, qR, tT, res, dev):
    """Step III exactly (the miniball of the last step's samples: translations in R^3, rotations as
    quaternions in R^4 on the side of the descent centre) beside the geodesic-descent balls of the step;
    CUDA events around the call (it reads a flag from the device every eight passes)."""
    import torch
    import paper_2403_09990_gb300.purse as P
    stream = torch.cuda.current_stream()
    ggd = res.clone()
    out = torch.empty(9, dtype=torch.float64, device=dev)
    times = []
    for r in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.megb_solve_exact(h.h, 0, qR, N_WALKS, tT, N_WALKS, out, ggd[:4].contiguous(), stream)
        e1.record(stream)
        P.purse_sync(h.h, stream)
        if r:
            times.append(e0.elapsed_time(e1))
    g, x = ggd.cpu().numpy(), out.cpu().numpy()
    return {"ms": statistics.median(times), "D_exact": float(x[7]), "d_exact": float(x[8]),
            "D_descent": float(g[7]), "d_descent": float(g[8]),
            "descent_over_exact": {"D": float(g[7] / x[7]), "d": float(g[8] / x[8])},
            "samples": N_WALKS, "K_descent": K_MEGB}


def run_plain(args, p, dev, seeds, fused_value, fused_step_s):
    """The same step through the plain per-operation samplers (Alg. 3/5 in the paper's tensor form: one
    kernel per operation, intermediates in HBM, every constraint of every pose evaluated), then the same
    two balls; CUDA events around each step, L2 flushed in between."""
    import torch
    import paper_2403_09990_gb300.purse as P
    stream = torch.cuda.current_stream()
    h = P.Purse(p)
    qR = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tR = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    qT = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tT = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    pR, pT = closure_params(0), closure_params(1)
    times = []
    for s in range(1 + args.plain_steps):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.purse_sample_plain(h.h, pR, 1000 + s, seeds, 1, N_WALKS, qR, tR, None, stream)
        P.purse_sample_plain(h.h, pT, 1000 + s, seeds, 1, N_WALKS, qT, tT, None, stream)
        P.megb_solve(h.h, 0, K_MEGB, qR, N_WALKS, tT, N_WALKS, res, None, stream)
        e1.record(stream)
        P.purse_sync(h.h, stream)
        if s > 0:  # the first step warms up
            times.append(e0.elapsed_time(e1))
    h.close()
    ms = statistics.median(times)
    evals_alg = 2 * N_WALKS * N_ITER * (N_PERTURB + N_KEEP * N_STEPS) * p.n
    return {"ms_per_step": ms, "value": evals_alg / (ms / 1e3), "unit": UNIT, "steps": len(times),
            "megb_solves_per_s": 1e3 / ms, "fused_speedup": (ms / 1e3) / fused_step_s,
            "path": "purse_sample_plain per sampler (perturbation, eq. 11 dist, top_k_indices, ladder candidates, "
                    "in_purse, find_farthest: one kernel each per iteration, intermediates in HBM) + megb_solve"}


def run_sweep(args):
    """Precision / scale sweep of the single-PURSE path (2D-3D, presets of Section V with N_I = 5, ground-truth
    seeds, both balls with 200 GGD iterations): FP32 against FP64 walks and balls for N in {8, 32, 128, 256}
    and 2^16..2^20 samples per sampler, then FP32 alone up to 2^26 samples at N = 16, where the ball kernels
    stream the samples from HBM.  One JSON line per point."""
    import torch
    import paper_2403_09990_gb300.purse as P
    from paper_2403_09990_gb300 import synthetic as syn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    K = K_MEGB

    def solve(p, S, precision, reps):
        dt = torch.float32 if precision == 0 else torch.float64
        h = P.Purse(p)
        sd = torch.as_tensor(p.seed_pose()[None], dtype=torch.float64, device=dev)
        qR = torch.empty((S, 4), dtype=dt, device=dev)
        tR = torch.empty((S, 3), dtype=dt, device=dev)
        qT = torch.empty((S, 4), dtype=dt, device=dev)
        tT = torch.empty((S, 3), dtype=dt, device=dev)
        res = torch.empty(9, dtype=torch.float64, device=dev)
        pr = P.make_params(n_iter=5, precision=precision, sampler=0)
        pt = P.make_params(n_iter=5, precision=precision, sampler=1)
        times = []
        evals = 0
        for r in range(reps + 1):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            P.purse_sample(h.h, pr, 9, sd, 1, S, qR, tR, None, stream)
            P.purse_sample(h.h, pt, 9, sd, 1, S, qT, tT, None, stream)
            e[1].record(stream)
            P.megb_solve(h.h, precision, K, qR, S, tT, S, res, None, stream)
            e[2].record(stream)
            P.purse_sync(h.h, stream)
            if r > 0:  # the first pass warms up
                times.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
        h.close()
        walk_ms = statistics.median(t[0] for t in times)
        megb_ms = statistics.median(t[1] for t in times)
        return res.cpu().numpy(), walk_ms, megb_ms

    def angle(a, b):
        d = abs(float(np.dot(a, b)))
        return 2.0 * float(np.arccos(min(1.0, d)))

    for n in ((8, 32, 128, 256) if "precision" in args.sweep_parts else ()):
        p = syn.purse_2d3d(n, 0)
        for lg in (16, 18, 20):
            S = 1 << lg
            r32, w32, m32 = solve(p, S, 0, 2)
            r64, w64, m64 = solve(p, S, 1, 1)
            alg = 2 * S * 5 * (N_PERTURB + N_KEEP * N_STEPS) * n
            print(json.dumps({"sweep": "precision", "n_keypoints": n, "samples_per_sampler": S,
                              "fp32": {"walk_ms": w32, "megb_ms": m32, "evals_per_s": alg / (w32 / 1e3)},
                              "fp64": {"walk_ms": w64, "megb_ms": m64},
                              "err_vs_fp64": {"D_rel": abs(r32[7] - r64[7]) / r64[7],
                                              "d_rel": abs(r32[8] - r64[8]) / r64[8],
                                              "C_rad": angle(r32[:4], r64[:4]),
                                              "c_m": float(np.linalg.norm(r32[4:7] - r64[4:7]))}}), flush=True)
    kinds = (1, 0) if args.dist_kind is None else (args.dist_kind,)
    ns = (8, 16, 32, 64, 128, 256) if args.dist_n is None else (args.dist_n,)
    for kind in (kinds if "dist" in args.sweep_parts else ()):
        for n in ns:
            print(json.dumps(sweep_dist(P, syn, dev, stream, kind, n)), flush=True)
    if "next" in args.sweep_parts:
        for line in sweep_next(P, syn, dev, stream):
            print(json.dumps(line), flush=True)
    p = syn.purse_2d3d(N_KEYPOINTS, 0)
    for lg in (tuple(int(x) for x in args.scale_lg.split(",")) if "scale" in args.sweep_parts else ()):
        S = 1 << lg
        r32, w32, m32 = solve(p, S, 0, 1)
        ball_bytes = (16 + 12) * S * (K + 1)
        print(json.dumps({"sweep": "scale", "n_keypoints": N_KEYPOINTS, "samples_per_sampler": S,
                          "walk_ms": w32, "megb_ms": m32, "samples_per_s": 2 * S / ((w32 + m32) / 1e3),
                          "megb_gbs": ball_bytes / (m32 / 1e3) / 1e9,
                          "megb_bytes_note": "16 B per rotation sample + 12 B per translation sample, per GGD "
                                             "iteration and the final pass", "D": r32[7], "d": r32[8]}), flush=True)


def _host_timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


def sweep_next(P, syn, dev, stream):
    """The rows beyond the main workload, each with its oracle timed beside it (the cpu_baseline leg of each
    line: one host core, FP64, a bounded sample of the same input): P3P RANSAG (2D-3D Step I), the exact
    Step III miniball of boundary samples, the pose-regression PURSE (Example 3) and 2D-3D constraints in the
    norm of eq. 4; the last two through the fused walk kernels beside the per-operation samplers (and, for
    the noise matrices, the isotropic fused walk of the same size).  GPU parts: CUDA events (the RANSAG call synchronises, so it takes the wall clock)."""
    import torch
    from oracle import closure, megb as om, p3p as op3, ransag as ora
    lines = []

    def events(fn, reps):
        times = []
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if r:  # the first call warms up
                times.append(e0.elapsed_time(e1))
        return statistics.median(times)

    def cpu(value, unit, sample):
        return {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample}

    # ---- P3P RANSAG on the bench's 2D-3D PURSE
    p = syn.purse_2d3d(N_KEYPOINTS, PURSE_SEED)
    trials = 1 << 20
    seeds = torch.empty((trials, 12), dtype=torch.float64, device=dev)
    with P.Purse(p) as h:
        try:
            P.purse_ransag(h.h, 1, 1 << 16, trials, seeds)           # warm-up
        except P.PurseError:
            pass
        n, dt = _host_timed(lambda: P.purse_ransag(h.h, 2, trials, trials, seeds))
    ot = 1 << 13
    (os_, _), odt = _host_timed(lambda: op3.ransag_2d3d(p, 2, ot, ot))
    lines.append({"sweep": "next", "row": "p3p_ransag", "workload": f"2D-3D PURSE N={N_KEYPOINTS}, {trials} trials",
                  "gpu": {"ms": dt * 1e3, "trials_per_s": trials / dt, "seeds": n},
                  "cpu_baseline": cpu(ot / odt, "trials/s", f"{ot} trials ({len(os_)} seeds)"),
                  "gpu_over_oracle": (trials / dt) / (ot / odt)})

    # ---- exact miniball of 2^20 boundary samples per set (fused walks, N_I = 5)
    S = 1 << 20
    qR = torch.empty((S, 4), dtype=torch.float32, device=dev)
    tR = torch.empty((S, 3), dtype=torch.float32, device=dev)
    qT = torch.empty((S, 4), dtype=torch.float32, device=dev)
    tT = torch.empty((S, 3), dtype=torch.float32, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    ex = torch.empty(9, dtype=torch.float64, device=dev)
    sd = torch.as_tensor(p.seed_pose()[None], dtype=torch.float64, device=dev)
    with P.Purse(p) as h:
        iso_ms = events(lambda: (P.purse_sample(h.h, closure_params(0, 5), 9, sd, 1, S, qR, tR, None, stream),
                                 P.purse_sample(h.h, closure_params(1, 5), 9, sd, 1, S, qT, tT, None, stream)), 1)
        P.megb_solve(h.h, 0, K_MEGB, qR, S, tT, S, res, None, stream)
        ref = res[:4].contiguous()
        ems = events(lambda: P.megb_solve_exact(h.h, 0, qR, S, tT, S, ex, ref, stream), 2)
    m = 1 << 12
    qn, tn = qR[:m].double().cpu().numpy(), tT[:m].double().cpu().numpy()
    _, odt = _host_timed(lambda: (om.meb_exact_translation(tn), om.meb_exact_rotation(qn, qn[0])))
    lines.append({"sweep": "next", "row": "exact_meb", "workload": f"{S} rotation + {S} translation samples "
                  f"(2D-3D N={N_KEYPOINTS} boundary walks, N_I=5)",
                  "gpu": {"ms": ems, "samples_per_s": 2 * S / (ems / 1e3), "D": float(ex[7]), "d": float(ex[8])},
                  "cpu_baseline": cpu(2 * m / odt, "samples/s", f"the first {m} samples of each set (Welzl)"),
                  "gpu_over_oracle": (2 * S / (ems / 1e3)) / (2 * m / odt)})

    def plain_row(name, purse, prm, samplers, gpu_seeds, s0, seeds_np, walks, oracle_walks, note, fused=False):
        Sx = walks
        q = torch.empty((Sx, 4), dtype=torch.float32, device=dev)
        t = torch.empty((Sx, 3), dtype=torch.float32, device=dev)
        q2 = torch.empty((Sx, 4), dtype=torch.float32, device=dev)
        t2 = torch.empty((Sx, 3), dtype=torch.float32, device=dev)
        r = torch.empty(9, dtype=torch.float64, device=dev)
        with P.Purse(purse) as h:
            def run(sample):
                sample(h.h, prm(0), 11, gpu_seeds, s0, Sx, q, t, None, stream)
                if 1 in samplers:
                    sample(h.h, prm(1), 11, gpu_seeds, s0, Sx, q2, t2, None, stream)
                P.megb_solve(h.h, 0, K_MEGB, q, Sx, t2 if 1 in samplers else t, Sx, r, None, stream)
            ms = events(lambda: run(P.purse_sample_plain), 2)
            ms_fused = events(lambda: run(P.purse_sample), 2) if fused else None
            r_fused = r.cpu().numpy() if fused else None
        per_walk = prm(0).n_iter * (prm(0).n_perturb + prm(0).n_keep * prm(0).n_steps) * (
            2 * purse.n if purse.kind == syn.KIND_REG else purse.n)
        evals = len(samplers) * Sx * per_walk
        oprm = oracle_params(purse)
        ids = np.arange(oracle_walks)

        def oracle_run():
            R, tt = closure.sample_rotation_boundary(purse, seeds_np, oprm, 11, ids)
            qs, ts = closure.as_samples(R, tt)
            if 1 in samplers:
                R2, tt2 = closure.sample_translation_boundary(purse, seeds_np, oprm, 11, ids)
                ts = closure.as_samples(R2, tt2)[1]
            om.megb_rotation(qs, K_MEGB)
            om.megb_translation(ts, K_MEGB)
        _, odt = _host_timed(oracle_run)
        oev = len(samplers) * oracle_walks * per_walk
        plain = {"ms": ms, "evals_per_s": evals / (ms / 1e3), "path": "purse_sample_plain + megb_solve"}
        out = {"sweep": "next", "row": name, "workload": note, "gpu": plain,
               "cpu_baseline": cpu(oev / (odt), "evals/s", f"{oracle_walks} walks per sampler + both balls")}
        if fused:
            out["gpu"] = {"ms": ms_fused, "evals_per_s": evals / (ms_fused / 1e3), "path": "purse_sample + megb_solve",
                          "D": float(r_fused[7]), "d": float(r_fused[8])}
            out["gpu_plain"] = plain
        out["gpu_over_oracle"] = out["gpu"]["evals_per_s"] / (oev / odt)
        return out

    # ---- pose regression (10 hypotheses, LM preset: dS_R walks, both balls from them)
    pr = syn.purse_reg(10, 0)
    reg_seeds = torch.empty((2048, 12), dtype=torch.float64, device=dev)
    with P.Purse(pr) as h:
        s0 = P.purse_ransag(h.h, 3, 20000, 2048, reg_seeds)
    oseeds, _ = ora.convex_seeds(pr, 3, 20000, 2048)

    def reg_params(sampler):
        return P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=10, omega0=0.5, v0=0.0, gamma=0.5,
                             rot_perturb=0.0, trans_perturb=0.1, perturb_units=0, sampler=sampler, precision=0)
    lines.append(plain_row("purse_reg", pr, reg_params, (0,), reg_seeds, s0, oseeds, 1 << 18, 2048,
                           "pose regression, 10 hypotheses (Example 3), convex seeds, 2^18 dS_R walks (N_I=5, "
                           "N_P=150, N_P*=10, N_T=10), both balls", fused=True))

    # ---- 2D-3D with noise matrices (eq. 4), both samplers, beside the isotropic fused walk above
    pl = syn.purse_2d3d_ellipsoidal(N_KEYPOINTS, 0)
    lam_seeds = torch.as_tensor(pl.seed_pose()[None], dtype=torch.float64, device=dev)
    row = plain_row("lambda_norm_2d3d", pl, lambda smp: closure_params(smp, 5), (0, 1), lam_seeds, 1,
                    pl.seed_pose()[None], 1 << 20, 1024,
                    f"2D-3D PURSE N={N_KEYPOINTS} with 2x2 noise matrices (eigenvalues 0.5-2), ground-truth seed, "
                    "2^20 walks per sampler (N_I=5), both balls", fused=True)
    iso_evals = 2 * S * 5 * (N_PERTURB + N_KEEP * N_STEPS) * N_KEYPOINTS
    row["isotropic_fused_walks"] = {"ms": iso_ms, "evals_per_s": iso_evals / (iso_ms / 1e3),
                                    "note": "purse_sample on the identity-norm PURSE of the same seed, walks only"}
    lines.append(row)
    lines.append(sweep_batch_row(P, syn, dev, stream, "batch_lambda", events, cpu))
    lines.append(sweep_batch_row(P, syn, dev, stream, "batch_reg", events, cpu))
    return lines


def sweep_batch_row(P, syn, dev, stream, name, events, cpu, n_purses=1024, S=4096, n_single=16, oracle_walks=32):
    """One batch solve (graph replay, CUDA events) of n_purses PURSEs with noise matrices (3D-3D / 2D-3D
    by a fair coin, N ~ U{4..64}, eigenvalues 0.5-2) or of pose-regression PURSEs (N ~ U{3..20}
    hypotheses), S samples each, N_I = 5, both balls; beside it the single-PURSE path for the first
    n_single PURSEs (wall clock, create + both samplers + balls + D2H) and the oracle on oracle_walks
    walks per sampler of the first PURSE (one host core)."""
    import torch
    from oracle import closure, megb as om
    rng = np.random.default_rng(11)
    if name == "batch_lambda":
        purses = [syn.purse_3d3d_ellipsoidal(int(rng.integers(4, 65)), 1000 + p) if rng.random() < 0.5 else
                  syn.purse_2d3d_ellipsoidal(int(rng.integers(4, 65)), 1000 + p) for p in range(n_purses)]
        p3 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=0.5, v0=0.0, gamma=0.5,
                           rot_perturb=0.0, trans_perturb=0.1)
        p2 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=2.0, gamma=0.5,
                           rot_perturb=0.2, trans_perturb=0.1)
        b = P.purse_batch_create(purses)
        P.purse_batch_set_noise(b, purses)
        note = (f"{n_purses} PURSEs with noise matrices (eq. 4; 3D-3D / 2D-3D by a fair coin, N ~ U{{4..64}}, "
                f"eigenvalues 0.5-2), {S} samples each, N_I = 5, both balls ({K_MEGB} GGD iterations)")
    else:
        purses = [syn.purse_reg(int(rng.integers(3, 21)), 2000 + p) for p in range(n_purses)]
        p3 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=10, omega0=0.5, v0=0.02, gamma=0.5,
                           rot_perturb=0.2, trans_perturb=0.1)
        p2 = p3
        b = P.purse_batch_create_regression(purses)
        note = (f"{n_purses} pose-regression PURSEs (Example 3, N ~ U{{3..20}} hypotheses), {S} samples each, "
                f"both samplers, N_I = 5, both balls ({K_MEGB} GGD iterations)")
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device=dev)
    res = torch.empty((n_purses, 9), dtype=torch.float64, device=dev)
    try:
        ms = events(lambda: P.purse_batch_solve(b, p3, p2, 5, seeds, S, K_MEGB, res, stream), 2)
        P.purse_batch_sync(b, stream)
        finite = bool(torch.isfinite(res).all())
    finally:
        P.purse_batch_destroy(b)

    def samplers(pu):
        return (0, 1) if pu.kind != syn.KIND_3D3D else (0,)

    def per_walk(pu, prm):
        return prm.n_iter * (prm.n_perturb + prm.n_keep * prm.n_steps) * (2 * pu.n if pu.kind == syn.KIND_REG else pu.n)
    evals = sum(len(samplers(pu)) * S * per_walk(pu, p3 if pu.kind != syn.KIND_2D3D else p2) for pu in purses)
    # the single-PURSE path for the first PURSEs
    q = [torch.empty((S, 4), dtype=torch.float32, device=dev) for _ in range(2)]
    t = [torch.empty((S, 3), dtype=torch.float32, device=dev) for _ in range(2)]
    r1 = torch.empty(9, dtype=torch.float64, device=dev)

    def single():
        for p, pu in enumerate(purses[:n_single]):
            prm = p3 if pu.kind != syn.KIND_2D3D else p2
            with P.Purse(pu) as h:
                sd = torch.as_tensor(pu.seed_pose()[None], dtype=torch.float64, device=dev)
                for smp in samplers(pu):
                    prm.sampler = smp
                    P.purse_sample(h.h, prm, 5 + p, sd, 1, S, q[smp], t[smp], None, stream)
                prm.sampler = 0
                P.megb_solve(h.h, 0, K_MEGB, q[0], S, t[1] if len(samplers(pu)) == 2 else t[0], S, r1, None, stream)
                r1.cpu()
    single()
    _, sdt = _host_timed(single)
    # the oracle on a bounded sample of the first PURSE
    pu = purses[0]
    oprm = closure.preset_reg(v0=0.02, rot_perturb=0.2) if pu.kind == syn.KIND_REG else (
        closure.preset_3d3d() if pu.kind == syn.KIND_3D3D else closure.preset_2d3d())
    ids = np.arange(oracle_walks)

    def oracle_run():
        R, tt = closure.sample_rotation_boundary(pu, pu.seed_pose()[None], oprm, 5, ids)
        qs, ts = closure.as_samples(R, tt)
        if len(samplers(pu)) == 2:
            R2, tt2 = closure.sample_translation_boundary(pu, pu.seed_pose()[None], oprm, 5, ids)
            ts = closure.as_samples(R2, tt2)[1]
        om.megb_rotation(qs, K_MEGB)
        om.megb_translation(ts, K_MEGB)
    _, odt = _host_timed(oracle_run)
    oev = len(samplers(pu)) * oracle_walks * per_walk(pu, oprm)
    return {"sweep": "next", "row": name, "workload": note,
            "gpu": {"ms": ms, "purses_per_s": n_purses / (ms / 1e3), "evals_per_s": evals / (ms / 1e3),
                    "results_finite": finite, "path": "purse_batch_solve (one graph: statistics, persistent walk "
                    "launch, one block per ball)"},
            "per_instance": {"purses": n_single, "purses_per_s": n_single / sdt,
                             "path": "per PURSE: create + purse_sample per sampler + megb_solve + D2H, wall clock"},
            "speedup_vs_per_instance": (n_purses / (ms / 1e3)) / (n_single / sdt),
            "cpu_baseline": cpu(oev / odt, "evals/s", f"{oracle_walks} walks per sampler of the first PURSE + both "
                                "balls"),
            "gpu_over_oracle": (evals / (ms / 1e3)) / (oev / odt)}


def oracle_params(purse):
    from oracle import closure
    from paper_2403_09990_gb300 import synthetic as syn
    return closure.preset_reg() if purse.kind == syn.KIND_REG else closure.preset_2d3d()


def sweep_dist(P, syn, dev, stream, kind, n, n_poses=1 << 24):
    """eq. 11 distance of 2^24 materialised FP32 poses around the ground truth of one PURSE (rotations
    of about 0.02 rad, translations of a few noise radii) by the FP32 CUDA-core kernel, the tcgen05
    split-TF32 contraction and one TF32 pass; errors against the FP64 margins of the same poses
    (purse_eval in FP64); CUDA-event times with L2 flushed in between."""
    import torch
    p = syn.purse_3d3d(n, 0) if kind == 0 else syn.purse_2d3d(n, 0)
    rng = np.random.default_rng(n)
    m = 1 << 16
    phi = rng.normal(size=(m, 3)) * 0.02
    th = np.linalg.norm(phi, axis=1, keepdims=True)
    k = phi / th
    K = np.zeros((m, 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
    K = K - K.transpose(0, 2, 1)
    s_, c_ = np.sin(th)[..., None], np.cos(th)[..., None]
    R = (np.eye(3) + s_ * K + (1 - c_) * (K @ K)) @ p.R_gt
    t = p.t_gt + rng.normal(size=(m, 3)) * (3 * p.radii.mean() if kind == 0 else 0.01)
    base = np.concatenate([R.reshape(m, 9), t], axis=1).astype(np.float32)
    poses = torch.as_tensor(base, device=dev).repeat(n_poses // m, 1).contiguous()
    out = torch.empty(n_poses, dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    res = {"sweep": "dist", "kind": "3D-3D" if kind == 0 else "2D-3D", "n_keypoints": n, "poses": n_poses}
    with P.Purse(p) as h:
        m64 = torch.empty((m, n), dtype=torch.float64, device=dev)
        P.purse_eval(h.h, 1, poses[:m].double().contiguous(), m, m64, None, None, stream)
        ref = m64.min(dim=1).values
        scale = float(ref.abs().max())
        for mode, name in ((0, "fp32"), (1, "split_tf32"), (2, "tf32")):
            for _ in range(2):
                P.purse_dist(h.h, mode, poses, n_poses, out, stream)
            ts = []
            for r in range(5):
                flush.fill_(r)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.purse_dist(h.h, mode, poses, n_poses, out, stream)
                e1.record(stream)
                P.purse_sync(h.h, stream)
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            d = out[:m].double()
            fin = torch.isfinite(ref)
            err = float((d[fin] - ref[fin]).abs().max())
            res[name] = {"ms": ms, "poses_per_s": n_poses / (ms / 1e3), "evals_per_s": n_poses * n / (ms / 1e3),
                         "hbm_gbs": n_poses * 52 / (ms / 1e3) / 1e9, "max_abs_err": err,
                         "max_rel_err": err / scale}
    return res


def run_batch(args, dev):
    """Batched workload: 4096 PURSEs (fair-coin kind, N ~ U{4..64}), 4096 samples each, FP32, both balls
    with 200 GGD iterations; one CUDA graph (statistics, persistent walk launch, one block per ball)
    after the autotuner picked the walk launch shape."""
    import torch
    import paper_2403_09990_gb300.purse as P
    from paper_2403_09990_gb300 import synthetic as syn
    n_purses, S, K = args.batch_purses, args.batch_samples, K_MEGB
    purses = syn.purse_batch(n_purses, seed=7)
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device=dev)
    res = torch.empty((n_purses, 9), dtype=torch.float64, device=dev)
    p3 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=0.5, v0=0.0, gamma=0.5,
                       rot_perturb=0.0, trans_perturb=0.1)
    p2 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=1.0, v0=2.0, gamma=0.5,
                       rot_perturb=0.2, trans_perturb=0.1)
    b = P.purse_batch_create(purses)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    try:
        chunk, warps, _ = P.purse_batch_tune(b, p3, p2, 1, seeds, min(S, 1024), stream)
        for w in range(args.batch_warmup):
            P.purse_batch_solve(b, p3, p2, 10 + w, seeds, S, K, res, stream)
        P.purse_batch_sync(b, stream)
        tot, ev_total = 0.0, 0
        for st in range(args.batch_steps):
            flush.fill_(st & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.purse_batch_solve(b, p3, p2, 100 + st, seeds, S, K, res, stream)
            e1.record(stream)
            ev_total += P.purse_batch_sync(b, stream)
            tot += e0.elapsed_time(e1)
    finally:
        P.purse_batch_destroy(b)
    kinds = np.array([p.kind for p in purses])
    ns = np.array([p.n for p in purses])
    alg = float(((1 + kinds) * S * 5 * (150 + 10 * 15) * ns).sum())
    ms = tot / args.batch_steps
    per_instance = run_per_instance(args, purses[:args.per_instance_purses], p3, p2, S, K, dev)
    per_plain = run_per_instance(args, purses[:args.per_instance_purses], p3, p2, S, K, dev, plain=True)
    return {"workload": f"{n_purses} PURSEs (3D-3D / 2D-3D by a fair coin, N ~ U{{4..64}}), {S} samples each, "
                        f"presets of Section V (N_I = 5), both balls with {K} GGD iterations, FP32",
            "purses_per_s": n_purses / (ms / 1e3), "ms_per_solve": ms, "steps": args.batch_steps,
            "evals_per_s": alg / (ms / 1e3), "evals_executed_per_s": ev_total / args.batch_steps / (ms / 1e3),
            "launch": {"graph": "statistics + persistent walk kernel + one block per ball", "chunk": chunk,
                       "warps_per_block": warps},
            "per_instance": per_instance,
            "speedup_vs_per_instance": (n_purses / (ms / 1e3)) / per_instance["purses_per_s"],
            "per_instance_plain": per_plain,
            "speedup_vs_per_instance_plain": (n_purses / (ms / 1e3)) / per_plain["purses_per_s"]}


def run_per_instance(args, purses, p3, p2, S, K, dev, plain=False):
    """Per-instance GPU paths on the same GPU: the batch's first PURSEs solved one call sequence per PURSE
    (purse_create, a sampler call per sampler, megb_solve, result read back), as a caller without the batch
    API would; the sampler is the fused walk kernel (purse_sample) or, with plain=True, the plain
    per-operation samplers (purse_sample_plain, Alg. 3/5 in the paper's tensor form)."""
    import torch
    import paper_2403_09990_gb300.purse as P
    stream = torch.cuda.current_stream()
    q1 = torch.empty((S, 4), dtype=torch.float32, device=dev)
    t1 = torch.empty((S, 3), dtype=torch.float32, device=dev)
    q2 = torch.empty((S, 4), dtype=torch.float32, device=dev)
    t2 = torch.empty((S, 3), dtype=torch.float32, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    out = torch.empty(9, dtype=torch.float64)

    def one(pu, seed):
        with P.Purse(pu) as h:
            sd = torch.as_tensor(pu.seed_pose()[None], dtype=torch.float64, device=dev)
            prm = p3 if pu.kind == 0 else p2
            if plain:
                P.purse_sample_plain(h.h, P.purse_params.from_buffer_copy(prm), seed, sd, 1, S, q1, t1, None, stream)
            else:
                P.purse_sample(h.h, P.purse_params.from_buffer_copy(prm), seed, sd, 1, S, q1, t1, None, stream)
            if pu.kind == 1:
                p_t = P.purse_params.from_buffer_copy(prm)
                p_t.sampler = 1
                if plain:
                    P.purse_sample_plain(h.h, p_t, seed, sd, 1, S, q2, t2, None, stream)
                else:
                    P.purse_sample(h.h, p_t, seed, sd, 1, S, q2, t2, None, stream)
            P.megb_solve(h.h, 0, K, q1, S, t2 if pu.kind == 1 else t1, S, res, None, stream)
            out.copy_(res)
            P.purse_sync(h.h, stream)

    for pu in purses[:2]:
        one(pu, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, pu in enumerate(purses):
        one(pu, 100 + i)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"purses": len(purses), "purses_per_s": len(purses) / wall, "ms_per_purse": 1e3 * wall / len(purses),
            "path": f"per PURSE: purse_create + {'purse_sample_plain' if plain else 'purse_sample'} (dS_R; dS_t for "
                    "2D-3D) + megb_solve + result D2H, the batch's first PURSEs, wall clock"}


def run_grad(args, dev):
    """Differentiation workload: 1024 3D-3D PURSEs (N = 32, r_i ~ U[0.005, 0.02] m), 4096 samples per PURSE
    and sampler with boundary snap (dS_R walks for the rotation ball, dS_t walks with v0 = 0.02 m for the
    translation ball), both balls with 200 GGD iterations, then the adjoint of both radii with respect to
    every y_i and r_i (purse_batch_backward)."""
    import torch
    import paper_2403_09990_gb300.purse as P
    from paper_2403_09990_gb300 import synthetic as syn
    n_purses, S, K = args.grad_purses, 4096, K_MEGB
    purses = [syn.purse_3d3d(32, seed=5000 + i) for i in range(n_purses)]
    seeds = torch.as_tensor(syn.seed_array(purses), dtype=torch.float64, device=dev)
    res = torch.empty((n_purses, 9), dtype=torch.float64, device=dev)
    g = torch.zeros((n_purses, 9), dtype=torch.float64, device=dev)
    g[:, 7] = 1.0
    g[:, 8] = 1.0
    total = sum(pu.n for pu in purses)
    gy = torch.empty((total, 3), dtype=torch.float64, device=dev)
    gr = torch.empty(total, dtype=torch.float64, device=dev)
    p3 = P.make_params(n_iter=5, n_perturb=150, n_keep=10, n_steps=15, omega0=0.5, v0=0.02, gamma=0.5,
                       rot_perturb=0.025, trans_perturb=0.00125, perturb_units=1)
    p2 = P.make_params(n_iter=5)
    b = P.purse_batch_create(purses)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    try:
        P.purse_batch_set_grad(b, 1)
        P.purse_batch_tune(b, p3, p2, 1, seeds, 1024, stream)
        P.purse_batch_solve(b, p3, p2, 3, seeds, S, K, res, stream)
        P.purse_batch_backward(b, res, g, gy, gr, stream)
        P.purse_batch_sync(b, stream)
        fw = bw = 0.0
        for st in range(args.batch_steps):
            flush.fill_(st & 0xFF)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            P.purse_batch_solve(b, p3, p2, 200 + st, seeds, S, K, res, stream)
            e[1].record(stream)
            P.purse_batch_backward(b, res, g, gy, gr, stream)
            e[2].record(stream)
            P.purse_batch_sync(b, stream)
            fw += e[0].elapsed_time(e[1])
            bw += e[1].elapsed_time(e[2])
        nz = float((gr != 0).double().mean())
    finally:
        P.purse_batch_destroy(b)
    fw /= args.batch_steps
    bw /= args.batch_steps
    return {"workload": f"{n_purses} 3D-3D PURSEs, N=32, {S} samples per PURSE and sampler with boundary snap, "
                        f"both balls ({K} GGD iterations), adjoint of D-hat + d-hat w.r.t. every y_i and r_i, FP32 "
                        "walks, FP64 adjoint",
            "ms_forward": fw, "ms_backward": bw, "purses_per_s": n_purses / ((fw + bw) / 1e3),
            "backward_purses_per_s": n_purses / (bw / 1e3), "frac_radii_with_gradient": nz}


def run_e2e(args, p, dev):
    """Same step through the public API from host buffers: create the PURSE from host arrays, copy the
    seed pose in, sample both boundaries, solve both balls, read the result back."""
    import torch
    import paper_2403_09990_gb300.purse as P
    seeds_h = torch.as_tensor(p.seed_pose()[None], dtype=torch.float64).pin_memory()
    res_h = torch.empty(9, dtype=torch.float64).pin_memory()
    qR = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tR = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    qT = torch.empty((N_WALKS, 4), dtype=torch.float32, device=dev)
    tT = torch.empty((N_WALKS, 3), dtype=torch.float32, device=dev)
    seeds = torch.empty((1, 12), dtype=torch.float64, device=dev)
    res = torch.empty(9, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    pR, pT = closure_params(0), closure_params(1)
    total, evals = 0.0, 0
    n = p.n
    evals_alg = 2 * N_WALKS * N_ITER * (N_PERTURB + N_KEEP * N_STEPS) * n
    h2d = 8 * n * 8 + 8 * n * 4 + seeds_h.numel() * 8
    d2h = res_h.numel() * 8 + 2 * 8
    for s in range(args.warmup + args.steps):
        flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hR, hT = P.Purse(p), P.Purse(p)
        seeds.copy_(seeds_h, non_blocking=True)
        P.purse_sample(hR.h, pR, 2000 + s, seeds, 1, N_WALKS, qR, tR, None, stream)
        P.purse_sample(hT.h, pT, 2000 + s, seeds, 1, N_WALKS, qT, tT, None, stream)
        P.megb_solve(hR.h, 0, K_MEGB, qR, N_WALKS, tT, N_WALKS, res, None, stream)
        res_h.copy_(res, non_blocking=True)
        ev = P.purse_last_evals(hR.h, stream) + P.purse_last_evals(hT.h, stream)
        P.purse_sync(hR.h, stream)
        dt = time.perf_counter() - t0
        hR.close()
        hT.close()
        if s >= args.warmup:
            total += dt
            evals += ev
    return {"value": evals_alg * args.steps / total, "unit": UNIT, "evals_executed_per_s": evals / total, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": total / args.steps * 1e3,
            "path": "purse_create(host arrays) + pinned seed H2D + purse_sample x2 + megb_solve + result D2H"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    times, evals_all = [], 0
    walks = 0
    for s in range(args.warmup + args.steps):
        ev, wall, w = oracle_sample(args.ref_walks, args.cpu_workers)
        if s >= args.warmup:
            times.append(wall)
            evals_all += ev
            walks = w
    t = sum(times)
    value = evals_all / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(workload_config(), parallelism="host cores"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": args.cpu_workers, "kind": "oracle",
                            "sample": f"per step {walks} walks (both samplers, N_I={N_ITER}) + both balls"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    global N_WALKS, N_ITER
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-walks", type=int, default=192, help="oracle walks per worker per sampler (cpu_baseline)")
    ap.add_argument("--ref-walks", type=int, default=64, help="oracle walks per worker per sampler (reference arm)")
    ap.add_argument("--cpu-workers", type=int, default=min(16, cpu_cores()))
    ap.add_argument("--walks", type=int, default=N_WALKS, help="walks per sampler (profiling of a smaller case)")
    ap.add_argument("--iters", type=int, default=N_ITER, help="walk iterations (profiling of a smaller case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-PURSE measurement")
    ap.add_argument("--batch-purses", type=int, default=4096)
    ap.add_argument("--batch-samples", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-warmup", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-operation comparator")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (default launch shapes)")
    ap.add_argument("--no-c1", action="store_true", help="skip the FP64 3D-3D configuration (C1)")
    ap.add_argument("--no-grad", action="store_true", help="skip the batched differentiation measurement")
    ap.add_argument("--sweep", action="store_true", help="precision / scale sweep instead of the bench step")
    ap.add_argument("--sweep-parts", default="precision,scale,dist,next", help="which parts of the sweep to run")
    ap.add_argument("--dist-kind", type=int, default=None, help="dist sweep: one PURSE kind (0 3D-3D, 1 2D-3D)")
    ap.add_argument("--scale-lg", default="22,24,26", help="scale sweep: log2 of the samples per sampler")
    ap.add_argument("--dist-n", type=int, default=None, help="dist sweep: one keypoint count")
    ap.add_argument("--grad-purses", type=int, default=1024)
    ap.add_argument("--per-instance-purses", type=int, default=256,
                    help="PURSEs of the batch solved one by one for the per-instance comparison")
    args = ap.parse_args()
    N_WALKS, N_ITER = args.walks, args.iters
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sweep:
        run_sweep(args)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
