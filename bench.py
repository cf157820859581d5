#!/usr/bin/env python3
"""Benchmark of the MetaDE batched inner-DE generation step on GB300.

Headline workload (the full MetaDE configuration): eight MetaDE runs of 128
executors each (1024 concurrent inner DEs).  Per run the population size is
drawn from U{50..200}, the dimension from {20, 50, 100, 200} and the
objective from the six synthetic shifted-rotated functions (sphere,
Rosenbrock, Rastrigin, Griewank, Ackley, Schwefel 1.2).  One step = one
evolver generation of all eight runs (Alg. 3): rand/1/bin trials and
decoding, executor initialisation, 200 executor generations, best-fitness
reduction, evolver selection = 2.6e7 individual-generations.  The batched
path runs the rotation of every executor with D >= 129 as a BF16 tcgen05 GEMM
with FP32 accumulation (the width is autotuned) and the rest in FP32.

Metric: individual-generations per second (the paper's FEs per second) and
the evolver-generation time, for the batched mixed-precision path next to
the plain FP32 path (one executor per launch per generation, no graph, no
tuning).  The line also carries the FP64 final error of every run's best
individual, and the moderate workload (six runs x 100 executors x NP 100 x
D 20, 500 generations) with both selection-tie modes as a secondary key.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 oracle on
the host cores on a bounded sample of the same workload.  Other studies
(`--workload`): moderate (the D 20 workload alone), precision (D 1000 on the
tensor cores), batching (512 ragged executors), full (whole MetaDE runs),
equal_error (batched mixed precision vs plain FP32 over 31 seeds), mlp (the
MLP objective), evolvers (DE, PSO, CSO, NES), oracle (the FP64 oracle alone
on one core and on all host cores).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "inner-DE individual-gens/s & outer-gen time: batched+BF16 vs plain FP32"
UNIT = "individual-gens/s"
WORKLOAD = "full-8x128-ragged"
INNER_GENS = 200
MODERATE = "moderate-6x100x100xD20"
MODERATE_GENS = 500
CPU_SAMPLE_PER_RUN = 2  # executors per run of the full workload timed on the host (of 128)
ERROR_FLOOR = 1e-8      # final errors below this are reported as 0 (Sec. IV-A)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--inner-gens", type=int, default=INNER_GENS)
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "moderate", "precision", "batching", "full", "equal_error", "mlp",
                             "evolvers", "oracle"],
                    help="headline: the full workload, batched mixed precision vs plain FP32 (the JSON line "
                         "of the benchmark contract); moderate: 6 runs x 100 executors, D 20; precision: the "
                         "D=1000 precision study; batching: 512 ragged executors; full: whole MetaDE runs of "
                         "the full workload; equal_error: batched mixed precision vs plain FP32 over 31 seeds "
                         "at an equal FE budget; evolvers: whole MetaDE runs with each evolver (DE, PSO, CSO, "
                         "NES); oracle: the FP64 oracle alone on the host cores (one core and all cores) on "
                         "the tiny, moderate, batching and precision workloads")
    ap.add_argument("--outer-gens", type=int, default=3, help="evolver generations per run of equal_error")
    ap.add_argument("--eq-seeds", type=int, default=31, help="seeds of equal_error")
    ap.add_argument("--no-moderate", action="store_true", help="skip the moderate secondary key")
    ap.add_argument("--seeds", type=int, default=5, help="whole MetaDE runs of the full workload")
    ap.add_argument("--n-inst", type=int, default=64, help="executors of the precision study")
    ap.add_argument("--tc-min-dim", type=int, default=0,
                    help="width of the per-generation GEMM pipeline for the headline and batching studies "
                         "(0: metade_autotune picks it)")
    ap.add_argument("--tune-gens", type=int, default=0,
                    help="generations metade_autotune times per candidate (0: the generations of one step, so the "
                         "choice sees the late, near-tie-heavy generations too)")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small untimed case for an ncu capture and exit")
    return ap.parse_args(argv)


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: all_reduce(MAX) over the process group (the
    replicas' timed regions are bracketed by the same barriers)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def scale_sampled(prof, launches):
    """Profile of a run whose tensor-core kinds were sampled (one inner
    generation in PROFILE_STRIDE): each such kind's mean time per launch times
    `launches` (one launch per kind and inner generation of the run), with the
    count set to it; the other kinds as read."""
    out = dict(prof)
    for k in TC_KINDS:
        ms_k, n_k = prof.get(k, (0.0, 0))
        if n_k:
            out[k] = (ms_k * launches / n_k, launches)
    return out


def whole_job_rate(units_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank runs the whole workload)."""
    return world * units_per_step * steps / (max_ms / 1000.0)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# --------------------------------------------------------------- CPU oracle
def _oracle_job(args):
    """One executor run of the oracle (module-level so a spawn pool can pickle it)."""
    import oracle
    theta, np_, obj, shift, rot, gens, seed, stream = args
    oracle.build()
    oracle.pde_run(theta, np_, obj, shift, rot, gens, seed=seed, stream=stream, epoch=0)
    return np_ * gens


def oracle_tasks(wl, per_run: int, gens: int):
    """Executors of the first evolver generation: the oracle's own evolver
    draws and decodes theta exactly as the workload does."""
    import oracle
    tasks = []
    for g, p in enumerate(wl.problems):
        opop, _ = oracle.outer_init(wl.n_out, wl.seed, g)
        trial = oracle.outer_trial(opop, wl.seed, g, 0)
        for j in range(per_run):
            th = oracle.decode(trial[j])
            tasks.append((th, int(wl.inst_np[g * wl.n_out + j]), p.obj, p.shift, p.rot, gens, wl.seed, g))
    return tasks


def _oracle_box_job(args):
    """One executor run of the oracle in a given box (module-level for the spawn pool)."""
    import oracle
    theta, np_, obj, shift, rot, gens, seed, stream, lo, hi = args
    oracle.build()
    oracle.pde_run(theta, np_, obj, shift, rot, gens, seed=seed, stream=stream, epoch=0, lo=lo, hi=hi)
    return np_ * gens


def time_oracle(tasks, cores: int, job=_oracle_job):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(job, [t[:5] + (1,) + t[6:] for t in tasks[:cores]])  # workers up, library built, before timing
        t0 = time.perf_counter()
        units = sum(pool.map(job, tasks, chunksize=1))
        dt = time.perf_counter() - t0
    return units, dt


def cpu_baseline(wl, gens: int, per_run: int = CPU_SAMPLE_PER_RUN):
    cores = os.cpu_count() or 1
    tasks = oracle_tasks(wl, per_run, gens)
    units, dt = time_oracle(tasks, cores)
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d executors (%d per run, the first of the evolver's first generation) x %d generations "
                      "of the %s workload (%d individual-generations), FP64 C oracle, %d spawn processes, %.1f s "
                      "wall" % (len(tasks), per_run, gens, wl.name, units, cores, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    wl = synth.full(inner_gens=args.inner_gens)
    cores = os.cpu_count() or 1
    per_run = -(-cores // len(wl.problems))  # every core busy in each step
    tasks = oracle_tasks(wl, per_run, args.inner_gens)
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    times, units = [], 0
    with ctx.Pool(cores) as pool:
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            u = sum(pool.map(_oracle_job, tasks, chunksize=1))
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
                units += u
    total = sum(times)
    value = units / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "inner_gens": args.inner_gens,
                                             "sample_executors_per_step": len(tasks)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d executors (%d per run, NP of their run) x %d generations per step"
                                       % (len(tasks), per_run, args.inner_gens)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- our arm
# DRAM bytes (read + written) of one k_fused_small<20> launch of the moderate
# workload, from the ncu capture summarised in profiles/k_fused_small_moderate_d20.md:
# the launch loads the executors' state once and stores it once, so the figure
# does not depend on the number of fused generations.
SMALL_KERNEL_DRAM_BYTES = 5.224704e6


def alu_ops(theta, inst_np, dims):
    """Algorithmic lane operations of one generation of every executor:
    D^2 rotation FMAs + (2 dn + 8) D mutation/crossover/clip/shift operations
    + 100 per Philox4x32-10 call (10 rounds of 10 integer operations), with
    1 + ceil(m/4) calls per individual for the index draws and ceil(D/4) for
    binomial masks.  Transcendentals of the objectives are not counted."""
    import numpy as np
    th = np.asarray(theta)
    bl, br, dn, cs = th[:, 2].astype(int), th[:, 3].astype(int), th[:, 4].astype(int), th[:, 5].astype(int)
    a = ((bl == 1) | (br == 1)).astype(int)
    m = a + 2 * dn
    D = np.asarray(dims, dtype=np.float64)
    calls = 1 + np.ceil(m / 4.0) + np.where(cs == 1, np.ceil(D / 4.0), 0.0)
    per = D * D + (2 * dn + 8) * D + 100.0 * calls
    return float((per * np.asarray(inst_np, dtype=np.float64)).sum())


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def measure_moderate(args, dev, stream, rank, world, tie_fp64=0, steps=None, e2e=False, plain=False):
    """The moderate workload (6 runs x 100 executors x NP 100 x D 20, 500
    generations per evolver generation; the small-D kernel keeps every
    executor in shared memory): batched steps timed with CUDA events after an
    L2 flush, the roofline of k_fused_small<20> (ALU-bound: alu_ops lane
    operations per launch over its event time, against 152 SMs x 128 lanes x
    the maximum SM clock).  Optionally e2e through the graph call with host
    copies, and the plain FP32 arm (one step)."""
    import torch
    import torch.distributed as dist
    import paper_2502_10470_gb300 as M
    import synth
    gens = MODERATE_GENS
    steps = steps or args.steps
    wl = synth.moderate(inner_gens=gens)
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]

    def make(path):
        return M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed + rank, one_shot=1,
                       n_out=wl.n_out, path=path, device=dev, stream=stream.cuda_stream, tie_fp64=tie_fp64)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def step(batch, og):
        M.metade_outer_step(batch.ctx, batch.opop, batch.ofit, batch.trial, batch.theta, None, og, 0)
        M.metade_init(batch.ctx, batch.pop, batch.fit, 0)
        M.metade_inner_step(batch.ctx, batch.pop, batch.fit, batch.theta, 0, 0, gens, batch.best_f, batch.best_i)
        M.metade_outer_step(batch.ctx, batch.opop, batch.ofit, batch.trial, batch.theta, batch.best_f, og, 1)

    b = make(M.METADE_PATH_BATCHED)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 20)
    units = float(wl.inst_np.sum()) * gens
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    og = 0
    for _ in range(args.warmup):
        step(b, og)
        og += 1
    if M.metade_sync(b.ctx) != 0:
        raise RuntimeError("device status after warm-up")
    barrier()
    M.metade_profile(b.ctx, True)
    M.metade_profile_read(b.ctx)
    evs, thetas = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(b, og)
        e1.record(stream)
        evs.append((e0, e1))
        thetas.append(b.theta.clone())
        og += 1
    barrier()
    prof = M.metade_profile_read(b.ctx)
    M.metade_profile(b.ctx, False)
    total = sum(a.elapsed_time(c) for a, c in evs)
    total_max = max_over_ranks(total, world, dev)
    kern = prof["fused_small"][0] / max(1, prof["fused_small"][1])
    ops = sum(alu_ops(th.cpu().numpy(), wl.inst_np, b.dims) * gens for th in thetas) / steps
    sm_max = float(load_peaks().get("sm_max_mhz", 2070.0))
    peak_ops = 152 * 128 * sm_max * 1e6
    out = {"workload": wl.name, "tie_fp64": tie_fp64, "value": whole_job_rate(units, steps, world, total_max),
           "unit": UNIT, "ms_per_step": total_max / steps, "steps": steps,
           "roofline": {"bound": "alu", "kernel": "k_fused_small<20>", "achieved": ops / (kern / 1e3) / 1e9,
                        "peak": peak_ops / 1e9, "unit": "Gop/s", "frac": ops / (kern / 1e3) / peak_ops,
                        "kernel_ms": kern, "kernel_share": kern * steps / total,
                        "peak_source": "152 SMs x 128 lanes x %.0f MHz (max SM clock), of derived peak" % sm_max}}
    if e2e:
        out["e2e"] = measure_e2e(b, wl, gens, og, steps, dev, stream, world, units)
    if plain:
        p = make(M.METADE_PATH_PLAIN)
        M.metade_outer_init(p.ctx, p.opop, p.ofit)
        M.metade_outer_step(p.ctx, p.opop, p.ofit, p.trial, p.theta, None, 0, 0)
        M.metade_init(p.ctx, p.pop, p.fit, 0)
        M.metade_inner_step(p.ctx, p.pop, p.fit, p.theta, 0, 0, 1, None, None)  # warm-up
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = M.metade_launch_count(p.ctx)
        e0.record(stream)
        step(p, 1)
        e1.record(stream)
        barrier()
        pms = e0.elapsed_time(e1)
        out["plain_fp32"] = {"value": units / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms, "steps": 1,
                             "gpu_launches": M.metade_launch_count(p.ctx) - l0,
                             "path": "one cooperative launch per executor per generation, FP32, no graph"}
        p.close()
    out["plan"] = json.loads(M.metade_plan_info(b.ctx))
    b.close()
    return out


def measure_e2e(b, wl, gens, og, steps, dev, stream, world, units):
    """End to end through the public call a user makes, metade_outer_generation
    (one CUDA graph per evolver generation): every step copies the evolver
    state host -> device from pinned memory and reads the meta-fitness and the
    evolver fitness back device -> host, inside the timed region."""
    import torch
    import paper_2502_10470_gb300 as M
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    h_opop = b.opop.cpu().pin_memory()
    h_ofit = b.ofit.cpu().pin_memory()
    h_best = torch.empty_like(b.best_f, device="cpu").pin_memory()
    h_ofit_out = torch.empty_like(b.ofit, device="cpu").pin_memory()
    M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i, og,
                              gens, True)  # capture the graph before timing
    og += 1
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.opop.copy_(h_opop, non_blocking=True)
        b.ofit.copy_(h_ofit, non_blocking=True)
        M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i, og,
                                  gens, True)
        h_best.copy_(b.best_f, non_blocking=True)
        h_ofit_out.copy_(b.ofit, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        og += 1
    if M.metade_sync(b.ctx) != 0:
        raise RuntimeError("device status after the e2e steps")
    tot = max_over_ranks(sum(ms), world, dev)
    return {"value": whole_job_rate(units, steps, world, tot), "unit": UNIT,
            "h2d_bytes_per_step": (h_opop.numel() + h_ofit.numel()) * 4,
            "d2h_bytes_per_step": (h_best.numel() + h_ofit_out.numel()) * 4,
            "ms_per_step": tot / steps, "call": "metade_outer_generation (CUDA graph)"}


def final_errors(b, wl):
    """FP64 final error f(x_best) - f* (f* = 0) of every run's best
    individual after the last evolver generation (Sec. IV-A; values below
    1e-8 reported as 0), through metade_eval on caller-given points, with the
    stored fitness of the same individual next to it."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    bf = b.best_f.cpu().numpy()
    bi = b.best_i.cpu().numpy()
    ldx = int(np.max(b.dpad))
    pts, inst, stored = [], [], []
    pop = b.pop.cpu().numpy()
    for g in range(wl.n_groups):
        ks = np.arange(g * wl.n_out, (g + 1) * wl.n_out)
        k = int(ks[np.argmin(bf[ks])])
        dp = int(b.dpad[k])
        row = pop[b.pop_off[k] + int(bi[k]) * dp:b.pop_off[k] + (int(bi[k]) + 1) * dp]
        x = np.zeros(ldx, dtype=np.float32)
        x[:dp] = row
        pts.append(x)
        inst.append(k)
        stored.append(float(bf[k]))
    xd = torch.from_numpy(np.stack(pts)).to(b.device)
    idd = torch.tensor(inst, dtype=torch.int32, device=b.device)
    f64 = torch.zeros(len(inst), dtype=torch.float64, device=b.device)
    M.metade_eval(b.ctx, xd, len(inst), idd, ldx, M.METADE_FP64, f64)
    if M.metade_sync(b.ctx) != 0:
        raise RuntimeError("device status after metade_eval")
    f64 = f64.cpu().numpy()
    err = [0.0 if v < ERROR_FLOOR else float(v) for v in f64]
    rel = [abs(s - v) / abs(v) if v != 0 else abs(s) for s, v in zip(stored, f64)]
    return {"per_run": err, "median": float(np.median(err)), "stored_rel_err_vs_fp64_max": float(max(rel)),
            "problems": [{"dim": p.dim, "obj": synth_name(p.obj)} for p in wl.problems],
            "how": "metade_eval(FP64) at each run's best individual after the last timed evolver generation; "
                   "< 1e-8 reported as 0"}


def synth_name(obj):
    import synth
    return synth.OBJ_NAMES[obj]


def run_ours(args):
    """The headline line: the full workload, batched mixed precision."""
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    import synth
    wl = synth.full(inner_gens=args.inner_gens)
    gens = args.inner_gens
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, gens)  # before the first GPU call (spawn pool)

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2502_10470_gb300 as M
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]

    def make(path, prec):
        return M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed + rank, one_shot=1,
                       n_out=wl.n_out, path=path, prec=prec, device=dev, stream=stream.cuda_stream,
                       tc_min_dim=args.tc_min_dim if path == M.METADE_PATH_BATCHED else 0)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def step(batch, og):
        M.metade_outer_step(batch.ctx, batch.opop, batch.ofit, batch.trial, batch.theta, None, og, 0)
        M.metade_init(batch.ctx, batch.pop, batch.fit, 0)
        M.metade_inner_step(batch.ctx, batch.pop, batch.fit, batch.theta, 0, 0, gens, batch.best_f, batch.best_i)
        M.metade_outer_step(batch.ctx, batch.opop, batch.ofit, batch.trial, batch.theta, batch.best_f, og, 1)

    b = make(M.METADE_PATH_BATCHED, M.METADE_BF16)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    units = float(wl.inst_np.sum()) * gens
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    # autotune (tensor-core width, block shapes) on a real state: the first evolver generation's executors
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, args.tune_gens or gens)
    og = 0
    for _ in range(args.warmup):
        step(b, og)
        og += 1
    if M.metade_sync(b.ctx) != 0:
        raise RuntimeError("device status after warm-up")
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = M.metade_launch_count(b.ctx)
    M.metade_profile(b.ctx, PROFILE_STRIDE)
    M.metade_profile_read(b.ctx)
    evs, thetas = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(b, og)
        e1.record(stream)
        evs.append((e0, e1))
        thetas.append(b.theta.clone())
        og += 1
    barrier()
    launches = M.metade_launch_count(b.ctx) - launches0
    clocks = sampler.stop()
    prof = M.metade_profile_read(b.ctx)
    M.metade_profile(b.ctx, False)
    if M.metade_sync(b.ctx) != 0:
        raise RuntimeError("device status after timing")
    prof = scale_sampled(prof, gens * args.steps)
    total = sum(a.elapsed_time(c) for a, c in evs)
    total_max = max_over_ranks(total, world, dev)
    value = whole_job_rate(units, args.steps, world, total_max)
    plan = json.loads(M.metade_plan_info(b.ctx))
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
               for k, v in prof.items() if v[1] and k != "near_ties"}
    near_ties_per_step = prof["near_ties"][1] / args.steps  # selections decided by the near-tie path
    roof = rooflines(wl, b, plan, prof, thetas, gens, args.steps, total, clocks)
    fe = final_errors(b, wl)
    e2e = measure_e2e(b, wl, gens, og + 1, args.steps, dev, stream, world, units)
    b.close()

    plain = None
    if not args.no_plain:
        p = make(M.METADE_PATH_PLAIN, M.METADE_FP32)
        M.metade_outer_init(p.ctx, p.opop, p.ofit)
        M.metade_outer_step(p.ctx, p.opop, p.ofit, p.trial, p.theta, None, 0, 0)
        M.metade_init(p.ctx, p.pop, p.fit, 0)
        M.metade_inner_step(p.ctx, p.pop, p.fit, p.theta, 0, 0, 1, None, None)  # warm-up: one generation
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = M.metade_launch_count(p.ctx)
        e0.record(stream)
        step(p, 1)
        e1.record(stream)
        barrier()
        pms = e0.elapsed_time(e1)
        plain = {"value": units / (pms / 1000.0), "unit": UNIT, "ms_per_step": pms, "steps": 1,
                 "gpu_launches": M.metade_launch_count(p.ctx) - l0,
                 "path": "one cooperative launch per executor per generation, FP32, no graph, no tuning"}
        p.close()

    # the literal tie rule on this workload: the same evolver generation's executors, the first
    # TIE_GENS inner generations with FP64 tie re-evaluation against the default difference form
    tie64 = None
    if not args.no_moderate:
        tie64 = measure_tie_rule(wl, probs, dev, stream, rank, plan.get("tc_min_dim") or 129, gens)

    moderate = None
    if not args.no_moderate:
        ms = min(args.steps, 20)
        moderate = measure_moderate(args, dev, stream, rank, world, tie_fp64=0, steps=ms)
        lit = measure_moderate(args, dev, stream, rank, world, tie_fp64=1, steps=ms)
        moderate["tie_fp64"] = {"value": lit["value"], "ms_per_step": lit["ms_per_step"],
                                "kernel_ms": lit["roofline"]["kernel_ms"],
                                "ties": "FP64 re-evaluation of both vectors"}
        moderate.pop("plan", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "runs": wl.n_groups, "evolver_pop": wl.n_out,
                           "executors": wl.n_inst, "individuals": wl.individuals(),
                           "executor_pop": "U{50..200} per run", "dims": [p.dim for p in wl.problems],
                           "objectives": [synth_name(p.obj) for p in wl.problems],
                           "inner_gens": gens, "precision": "BF16 tcgen05 rotation GEMM (FP32 accumulate) for "
                           "D >= tc_min_dim, FP32 below; FP32 difference form for near ties",
                           "tc_min_dim": plan.get("tc_min_dim"),
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed (256 MB write) before every timed step", "plan": plan},
                "outer_gen_ms": total_max / args.steps,
                "e2e": e2e,
                "gpu_launches": launches,
                "roofline": roof[0],
                "roofline_by_kernel": roof[1],
                "kernels": kernels,
                "kernel_timing": "CUDA events on the launching stream inside the timed steps: around the "
                                 "tensor-core kernels of one inner generation in %d (mean per launch x the "
                                 "launches of the steps), around every size-bucket launch; a sampled "
                                 "generation also carries its events' gaps, so the tensor-core kinds sum to a "
                                 "little more than the step" % PROFILE_STRIDE,
                "near_ties_per_step": near_ties_per_step, "tie_fp64": tie64,
                "final_error": fe,
                "plain_fp32": plain,
                "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "moderate": moderate,
                "cpu_baseline": cpu,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# The headline's per-kernel CUDA events: around the tensor-core kernels of one inner generation in
# PROFILE_STRIDE (events between kernels add to the step they measure); the size buckets' fused launches
# on every call.
PROFILE_STRIDE = 4
TC_KINDS = ("tc_gemm", "tc_generation", "tc_prologue", "tc_trial", "tc_select", "tc_ties", "tc_sel")
TIE_GENS = 20  # inner generations the literal tie rule is timed over (its FP64 ties cost seconds per step)
# (kernel, tensor-core width) -> DRAM bytes per launch on the full workload, from an ncu capture of the
# current kernel (read 84.4 MB: the population once and the draw records; write 81.4 MB: trial and operand
# rows, part of them still in L2 when the kernel ends)
TRAFFIC_BYTES = {("k_tc_trial2", 33): 165.78e6}


def measure_tie_rule(wl, probs, dev, stream, rank, tc_min_dim, gens):
    """The same state (the evolver's first generation of executors, after
    initialisation) run for TIE_GENS inner generations twice: near ties by
    the FP32 difference form (the default) and by FP64 re-evaluation of both
    vectors (tie_fp64 = 1, the literal rule; the tensor-core executors then
    take the five-kernel pipeline with a CTA per tie).  CUDA-event time per
    inner generation and the near ties decided, for each."""
    import torch
    import paper_2502_10470_gb300 as M
    out = {"inner_gens": TIE_GENS, "of": gens, "tc_min_dim": tc_min_dim,
           "state": "initialised executors of the evolver's first generation"}
    for key, t64 in (("difference_form", 0), ("fp64", 1)):
        b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed + rank, one_shot=1,
                    n_out=wl.n_out, prec=M.METADE_BF16, device=dev, stream=stream.cuda_stream,
                    tc_min_dim=tc_min_dim, tie_fp64=t64)
        M.metade_outer_init(b.ctx, b.opop, b.ofit)
        M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)  # loads the kernels
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        torch.cuda.synchronize()
        M.metade_profile(b.ctx, True)
        M.metade_profile_read(b.ctx)
        M.metade_profile(b.ctx, False)  # the tie count runs regardless
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, TIE_GENS, None, None)
        e1.record(stream)
        torch.cuda.synchronize()
        if M.metade_sync(b.ctx) != 0:
            raise RuntimeError("device status (tie rule)")
        ties = M.metade_profile_read(b.ctx)["near_ties"][1]
        out[key] = {"ms_per_inner_gen": e0.elapsed_time(e1) / TIE_GENS, "near_ties_per_inner_gen": ties / TIE_GENS}
        b.close()
    out["fp64_over_difference"] = out["fp64"]["ms_per_inner_gen"] / out["difference_form"]["ms_per_inner_gen"]
    return out


def rooflines(wl, b, plan, prof, thetas, gens, steps, total_ms, clocks):
    """Roofline of each measured kernel kind of the step, and the dominant one
    (largest share of the step).

    - ALU-bound fused kernels (small-D, tile): alu_ops lane operations of
      their executors over their event time, against 152 SMs x 128 lanes x
      the maximum SM clock.
    - The tensor-core GEMM (k_rot_tc, or k_tc_sel, which holds the GEMM with
      the objective, selection and commit): 2 NP D^2 algorithmic flops per
      executor-generation over its event time, against the measured BF16 peak
      (sustained: it runs inside a long step).
    - The trial kernel (k_tc_trial2, or k_tc_trial): HBM-bound; algorithmic
      bytes per row and generation = read the target row (4 D_pad), write the
      FP32 trial row (4 D_pad) and the BF16 operand row (2 x its K extent:
      round_up(D_pad, 64) on the four-kernel path, the context's K on the
      five-kernel one); the random parent rows are re-reads, not counted.
    - The selection kernel of the five-kernel pipeline (k_tc_select):
      HBM-bound; both rows read, the accepted ones written (counted as all).
    The near-tie kernels are left out: their work depends on how many
    selections are near ties, which the host does not see."""
    import numpy as np
    peaks = load_peaks()
    sm_max = float((clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * sm_max * 1e6
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0)) * 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    dims = b.dims
    on_tc = np.zeros(b.n_inst, dtype=bool)
    tcmin = plan.get("tc_min_dim") or 129
    tcinfo = plan.get("tensor_core") or {}
    if tcinfo:
        on_tc = dims >= tcmin
    fused = tcinfo.get("kernel") == "k_tc_sel"
    small = (dims <= 32) & ~on_tc
    tile = ~small & ~on_tc
    dpads = (dims + 3) // 4 * 4
    th = [t.cpu().numpy() for t in thetas]
    out = {}

    def alu(kind, mask, name):
        if not prof[kind][1] or not mask.any():
            return
        ms = prof[kind][0]
        ops = sum(alu_ops(t[mask], wl.inst_np[mask], dims[mask]) * gens for t in th)
        out[name] = {"bound": "alu", "achieved": ops / (ms / 1e3) / 1e9, "peak": alu_peak / 1e9, "unit": "Gop/s",
                     "frac": ops / (ms / 1e3) / alu_peak, "ms_per_step": ms / steps,
                     "share": ms / total_ms,
                     "peak_source": "152 SMs x 128 lanes x %.0f MHz (max SM clock), of derived peak" % sm_max}

    alu("fused_small", small, "k_fused_small")
    alu("fused_tile", tile & (dpads <= 128), "k_fused_tile")
    alu("fused_tile_stream", tile & (dpads > 128), "k_fused_tile_stream")
    gemm_kind = "tc_sel" if fused else "tc_gemm"
    if on_tc.any() and prof[gemm_kind][1]:
        rows = wl.inst_np[on_tc].astype(np.float64)
        dd = dims[on_tc].astype(np.float64)
        flops = 2.0 * float((rows * dd * dd).sum())  # per generation
        ms = prof[gemm_kind][0] / prof[gemm_kind][1]
        name = "k_tc_sel" if fused else "k_rot_tc"
        out[name] = {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12, "peak": bf16_peak / 1e12,
                     "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / bf16_peak,
                     "ms_per_step": prof[gemm_kind][0] / steps, "share": prof[gemm_kind][0] / total_ms,
                     "launch_ms": ms, "flops_per_launch": flops,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured"}
    if on_tc.any():
        rows = wl.inst_np[on_tc].astype(np.float64)
        dp = dpads[on_tc].astype(np.float64)
        kcols = np.ceil(dp / 64) * 64 if fused else float(tcinfo.get("kp", 0))
        trial = ("tc_trial", "k_tc_trial2" if fused else "k_tc_trial", 4 * dp + 4 * dp + 2 * kcols)
        kinds = [trial] if fused else [trial, ("tc_select", "k_tc_select", 4 * dp + 4 * dp + 4 * dp + 12)]
        for kind, name, per_row in kinds:
            if not prof[kind][1]:
                continue
            byts = float((rows * per_row).sum())
            ms = prof[kind][0] / prof[kind][1]
            out[name] = {"bound": "hbm", "achieved": byts / (ms / 1e3) / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                         "frac": byts / (ms / 1e3) / hbm, "ms_per_step": prof[kind][0] / steps,
                         "share": prof[kind][0] / total_ms, "launch_ms": ms, "bytes_per_launch": byts,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    # kernels with no roofline entry, by time: reported so that the dominant one is visible
    for kind in ("tc_ties", "tc_prologue"):
        if prof[kind][1]:
            out.setdefault("k_tc_ties2" if kind == "tc_ties" and fused else
                           ("k_tc_ties" if kind == "tc_ties" else ("k_tc_rank" if fused else "k_tc_prologue")),
                           {"bound": None, "ms_per_step": prof[kind][0] / steps, "share": prof[kind][0] / total_ms})
    ranked = [kv for kv in out.items() if kv[1].get("bound")]
    dom = max(ranked, key=lambda kv: kv[1]["share"]) if ranked else (None, {})
    head = dict(dom[1])
    head["kernel"] = dom[0]
    # DRAM bytes per launch from one ncu capture of the same kernel on the same rows (this workload at
    # the width the autotuner picks for it), while the kernel is the one captured; otherwise unknown
    known = TRAFFIC_BYTES.get((dom[0], int(tcmin))) if wl.name == WORKLOAD else None
    head["traffic"] = known
    if known is not None:
        head["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                  "(bench.py --profile-case tc-d200, generation 40)")
    return head, out


def run_moderate(args):
    """The moderate workload alone (6 runs x 100 executors x NP 100 x D 20,
    500 generations per evolver generation), with e2e and the plain arm."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    out = measure_moderate(args, dev, stream, rank, world, tie_fp64=0, e2e=True, plain=not args.no_plain)
    out["metric"] = METRIC
    out["warmup"] = args.warmup
    print(json.dumps(out), flush=True)


def run_equal_error(args):
    """The metric's comparison at an equal FE budget on the full workload:
    whole MetaDE runs (--outer-gens evolver generations of 200 executor
    generations, one-shot evaluation) over --eq-seeds seeds, with the batched
    mixed-precision path (BF16 GEMM for D >= 129, FP32 below), the batched
    FP32 path and the plain FP32 path (one executor per launch per
    generation).  Per run and arm: the median over seeds of the run's best
    meta-fitness (the evolver's stored y*) and of the FP64 final error of the
    last evolver generation's best individual (metade_eval, < 1e-8 as 0), and
    the Wilcoxon rank-sum p-value against plain FP32 (Sec. IV-A's test at
    0.05).  Also the wall time of one whole run per arm."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    import synth
    from scipy.stats import ranksums
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.full()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    gens = wl.inner_gens
    arms = (("batched_bf16", M.METADE_PATH_BATCHED, M.METADE_BF16),
            ("batched_fp32", M.METADE_PATH_BATCHED, M.METADE_FP32),
            ("plain_fp32", M.METADE_PATH_PLAIN, M.METADE_FP32))
    res = {}
    for name, path, prec in arms:
        ystar, ferr, wall = [], [], []
        for seed in range(args.eq_seeds):
            b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=seed, one_shot=1, n_out=wl.n_out,
                        path=path, prec=prec, device=dev, stream=stream.cuda_stream, tc_min_dim=129)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ofit = b.run_metade(args.outer_gens, gens, use_graph=path == M.METADE_PATH_BATCHED)
            wall.append(time.perf_counter() - t0)
            ystar.append(ofit.min(axis=1).astype(np.float64))
            ferr.append(np.array(final_errors(b, wl)["per_run"]))
            b.close()
        res[name] = {"ystar": np.array(ystar), "ferr": np.array(ferr), "wall_s_per_run": float(np.median(wall))}
    out = {}
    trunc = lambda a: np.where(a < ERROR_FLOOR, 0.0, a)
    for name, _, _ in arms:
        r = res[name]
        out[name] = {"wall_s_per_metade_run": r["wall_s_per_run"],
                     "ystar_median_per_run": [float(v) for v in np.median(trunc(r["ystar"]), axis=0)],
                     "final_error_fp64_median_per_run": [float(v) for v in np.median(r["ferr"], axis=0)]}
        if name != "plain_fp32":
            pv = [float(ranksums(trunc(r["ystar"][:, g]), trunc(res["plain_fp32"]["ystar"][:, g]))[1])
                  for g in range(wl.n_groups)]
            pf = [float(ranksums(r["ferr"][:, g], res["plain_fp32"]["ferr"][:, g])[1]) for g in range(wl.n_groups)]
            out[name]["ranksum_p_vs_plain_ystar"] = pv
            out[name]["ranksum_p_vs_plain_final_error"] = pf
            out[name]["runs_different_at_0.05"] = int(sum(1 for v in pf if v < 0.05))
    line = {"metric": "equal-FE-budget comparison: median final error, batched mixed precision vs plain FP32",
            "workload": wl.name, "seeds": args.eq_seeds, "outer_gens": args.outer_gens,
            "inner_gens_per_outer_generation": gens,
            "fe_per_run": [int(wl.inst_np[g * wl.n_out]) * wl.n_out * gens * args.outer_gens
                           for g in range(wl.n_groups)],
            "problems": [{"dim": p.dim, "obj": synth_name(p.obj)} for p in wl.problems],
            "results": out}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- precision study
def run_precision(args):
    """64 executors, NP 512, D 1000 (Rastrigin / Rosenbrock): one generation
    in FP32 (CUDA cores), BF16, bf16x3 and FP8-e4m3 (tcgen05), from a shared
    state.
    Per precision: generation time and individual-gens/s, the tensor-core
    GEMM's own time and TFLOP/s (2 NP D^2 algorithmic flops per executor),
    the relative fitness error against FP64 at the same trials, and the
    selection-bit mismatch rate against FP64 decisions (f64(u) <= f64(x))
    when both sides of each comparison are evaluated in the precision."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.precision(n_inst=args.n_inst)
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]

    def make(prec):
        return M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, prec=prec,
                       device=dev, stream=stream.cuda_stream)

    ref = make(M.METADE_FP32)
    ref.set_theta(wl.theta)
    M.metade_init(ref.ctx, ref.pop, ref.fit, 0)
    pop0, fit0 = ref.pop.clone(), ref.fit.clone()
    n = ref.n_indiv
    f64x = torch.empty(n, dtype=torch.float64, device=dev)
    M.metade_eval_pop(ref.ctx, pop0, M.METADE_FP64, f64x)
    ident = np.tile(np.array([0.0, 1.0, 4, 4, 1, 1], dtype=np.float32), (wl.n_inst, 1))  # trial = target
    inf = torch.full_like(fit0, float("inf"))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    gemm_flops = 2.0 * float((wl.inst_np.astype(np.float64) * wl.dims().astype(np.float64) ** 2).sum())
    out = {}
    for name, prec in (("fp32", M.METADE_FP32), ("bf16", M.METADE_BF16), ("bf16x3", M.METADE_BF16X3),
                       ("fp8e4m3", M.METADE_FP8E4M3)):
        b = make(prec)
        b.set_theta(wl.theta)
        b.pop.copy_(pop0)
        b.fit.copy_(inf)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
        trial, ft = b.pop.clone(), b.fit.clone()
        b.set_theta(ident)
        b.pop.copy_(pop0)
        b.fit.copy_(inf)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
        fxp = b.fit.clone()
        f64u = torch.empty(n, dtype=torch.float64, device=dev)
        M.metade_eval_pop(ref.ctx, trial, M.METADE_FP64, f64u)
        if M.metade_sync(b.ctx) != 0 or M.metade_sync(ref.ctx) != 0:
            raise RuntimeError("device status")
        rel = ((ft.double() - f64u).abs() / f64u.abs()).cpu().numpy()
        relx = ((fxp.double() - f64x).abs() / f64x.abs()).cpu().numpy()
        mism = float(((ft.double() <= fxp.double()) != (f64u <= f64x)).float().mean().item())
        # near ties at the first generation: |f(u) - f(x)| <= band f(x), band = max(1e-6, 2^-21 sqrt(D))
        band = max(1e-6, 2.0 ** -21 * float(np.sqrt(wl.dims().max())))
        ties0 = float(((ft - fxp).abs() <= band * fxp).float().mean().item())
        b.set_theta(wl.theta)
        b.pop.copy_(pop0)
        b.fit.copy_(fit0)
        for w in range(args.warmup):
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, w, 1, None, None)
        torch.cuda.synchronize()
        M.metade_profile(b.ctx, True)
        M.metade_profile_read(b.ctx)
        ms = []
        for st in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, args.warmup + st, 1, None, None)
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        prof = M.metade_profile_read(b.ctx)
        M.metade_profile(b.ctx, False)
        gen_ms = float(np.mean([a.elapsed_time(c) for a, c in ms]))
        # from the initial state: the first 20 generations, then 180 more (one call each, L2 not flushed
        # between the generations of a call; the state, 131 MB of population, exceeds L2), then the
        # same 200 generations again with per-kernel events
        runs = {}
        for profiled in (False, True):
            b.pop.copy_(pop0)
            b.fit.copy_(fit0)
            flush.zero_()
            torch.cuda.synchronize()
            if profiled:
                M.metade_profile(b.ctx, True)
                M.metade_profile_read(b.ctx)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 20, None, None)
            ev[1].record(stream)
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 20, 180, None, None)
            ev[2].record(stream)
            torch.cuda.synchronize()
            runs[profiled] = (ev[0].elapsed_time(ev[1]) / 20, ev[0].elapsed_time(ev[2]) / 200,
                              M.metade_profile_read(b.ctx) if profiled else None)
            M.metade_profile(b.ctx, False)
        if M.metade_sync(b.ctx) != 0:
            raise RuntimeError("device status")
        r = {"ms_per_generation": gen_ms, "indiv_gens_per_s": n / (gen_ms / 1e3),
             "first20_ms_per_generation": runs[False][0], "gens200_ms_per_generation": runs[False][1],
             "gens200_kernel_ms_per_generation": {k: v[0] / 200 for k, v in runs[True][2].items()
                                                  if v[1] and k not in ("tc_generation", "near_ties")},
             "gens200_near_ties_per_generation": runs[True][2]["near_ties"][1] / 200,
             "near_ties_per_generation": prof["near_ties"][1] / max(1, args.steps),
             "fitness_rel_err_vs_fp64": {"median": float(np.median(rel)), "p99": float(np.quantile(rel, 0.99)),
                                         "max": float(rel.max())},
             "target_fitness_rel_err_max": float(relx.max()),
             "selection_mismatch_rate_vs_fp64": mism, "near_tie_rate_first_generation": ties0,
             "plan": json.loads(M.metade_plan_info(b.ctx))}
        # the GEMM: k_rot_tc of the five-kernel pipeline, or the four-kernel generation's GEMM kernel
        # (k_rot_tc selecting in its epilogue), whose time includes the selection and the commit
        gkind = "tc_gemm" if prof["tc_gemm"][1] else "tc_sel"
        if prof[gkind][1]:
            gms = prof[gkind][0] / prof[gkind][1]
            r["tc_gemm_kernel"] = "k_rot_tc" + (" (selection epilogue)" if gkind == "tc_sel" else "")
            r["tc_gemm_ms"] = gms
            r["tc_gemm_tflops_algorithmic"] = gemm_flops / (gms / 1e3) / 1e12
            r["tc_gemm_tflops_issued"] = (3 if name == "bf16x3" else 1) * gemm_flops / (gms / 1e3) / 1e12
        if prof["fused_general"][1]:
            r["fused_general_ms"] = prof["fused_general"][0] / prof["fused_general"][1]
        out[name] = r
        b.close()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf = out["bf16"]
    peak = float(peaks.get("bf16_tflops", 1900.0))
    line = {"metric": "precision study: individual-gens/s, GEMM TFLOP/s, fitness error and selection mismatch vs FP64",
            "workload": "precision-%dx512xD1000" % wl.n_inst, "steps": args.steps, "warmup": args.warmup,
            "gemm_gflop_per_generation": gemm_flops / 1e9, "results": out,
            "roofline": {"bound": "tensor", "kernel": bf.get("tc_gemm_kernel", "k_rot_tc") + " bf16",
                         "achieved": bf.get("tc_gemm_tflops_algorithmic"),
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": (bf.get("tc_gemm_tflops_algorithmic") or 0) / peak, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"},
            "roofline_fp8": {"bound": "tensor", "kernel": "k_rot_tc (fp8e4m3)",
                             "achieved": out["fp8e4m3"].get("tc_gemm_tflops_algorithmic"), "peak": 2.0 * peak,
                             "unit": "TFLOP/s",
                             "frac": (out["fp8e4m3"].get("tc_gemm_tflops_algorithmic") or 0) / (2.0 * peak),
                             "peak_source": "2 x the measured bf16 burst peak (nominal fp8/bf16 dense ratio 4.5/2.25)"},
            "l2": "flushed before every timed generation"}
    print(json.dumps(line), flush=True)
    ref.close()


# ------------------------------------------------------- batching study
def run_batching(args):
    """512 executors of uneven size (NP ~ U{20..400}, D ~ U{10,20,50,100},
    objective ~ U{0..5}, theta sampled per executor): one step = 100
    generations of every executor, batched path (one launch per size bucket)
    vs plain path (one executor per launch per generation)."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.batching()
    gens = wl.inner_gens
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    units = float(wl.inst_np.sum()) * gens
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, path, steps in (("batched", M.METADE_PATH_BATCHED, args.steps), ("plain", M.METADE_PATH_PLAIN, 1)):
        if name == "plain" and args.no_plain:
            continue
        b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, path=path, device=dev,
                    stream=stream.cuda_stream, tc_min_dim=args.tc_min_dim)
        b.set_theta(wl.theta)
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        if path == M.METADE_PATH_BATCHED:
            M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, args.tune_gens or gens)
        for w in range(1 if name == "plain" else args.warmup):
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, w * gens, gens, b.best_f, b.best_i)
        torch.cuda.synchronize()
        M.metade_profile(b.ctx, True)
        M.metade_profile_read(b.ctx)
        ms = []
        for st in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, (10 + st) * gens, gens, b.best_f, b.best_i)
            e1.record(stream)
            ms.append((e0, e1))
        torch.cuda.synchronize()
        if M.metade_sync(b.ctx) != 0:
            raise RuntimeError("device status")
        prof = M.metade_profile_read(b.ctx)
        t = float(np.mean([a.elapsed_time(c) for a, c in ms]))
        out[name] = {"ms_per_step": t, "indiv_gens_per_s": units / (t / 1e3), "steps": steps,
                     "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1] and k != "near_ties"},
                     "plan": json.loads(M.metade_plan_info(b.ctx))}
        b.close()
    line = {"metric": "batching study: individual-gens/s, batched vs plain FP32", "workload": wl.name,
            "executors": wl.n_inst, "individuals": wl.individuals(), "generations_per_step": gens,
            "results": out, "speedup_vs_plain": (out["batched"]["indiv_gens_per_s"] / out["plain"]["indiv_gens_per_s"])
            if "plain" in out else None, "l2": "flushed before every timed step"}
    print(json.dumps(line), flush=True)


def run_full(args):
    """The full workload: 8 MetaDE runs x 128 executors (1024 inner DEs), NP
    ~ U{50..200}, D in {20, 50, 100, 200}, one-shot, 200 inner generations
    per evolver generation (all D < 256, so every executor is on the FP32
    CUDA-core kernels).  Per evolver generation: the batched path
    (metade_outer_generation, CUDA graph, tuned plan) against the plain FP32
    path (one executor per launch per generation, no graph, no tuning), both
    timed with CUDA events after an L2 flush.  Then whole MetaDE runs (50
    evolver generations) of the batched path over --seeds seeds, with
    one-shot evaluation (every executor of a run starts from the same
    population and draw stream, Sec. III-C) and with a stream per executor:
    the final error of each run per mode, the wall time of a whole run, and a
    rank-sum p-value per run between the two modes."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.full()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    gens = wl.inner_gens
    units = float(wl.inst_np.sum()) * gens
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def make(path, seed, one_shot=1):
        return M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=seed, one_shot=one_shot,
                       n_out=wl.n_out, path=path, device=dev, stream=stream.cuda_stream)

    out = {}
    for name, path, steps, warm in (("batched", M.METADE_PATH_BATCHED, args.steps, args.warmup),
                                    ("plain", M.METADE_PATH_PLAIN, 1, 0)):
        b = make(path, 0)
        M.metade_outer_init(b.ctx, b.opop, b.ofit)
        og = 0
        if path == M.METADE_PATH_BATCHED:
            M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
            M.metade_init(b.ctx, b.pop, b.fit, 0)
            M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 5)
        use_graph = path == M.METADE_PATH_BATCHED
        for _ in range(warm):
            M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i,
                                      og, gens, use_graph)
            og += 1
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i,
                                      og, gens, use_graph)
            e1.record(stream)
            evs.append((e0, e1))
            og += 1
        torch.cuda.synchronize()
        if M.metade_sync(b.ctx) != M.METADE_OK:
            raise RuntimeError("device status")
        ms = float(np.mean([a.elapsed_time(c) for a, c in evs]))
        out[name] = {"ms_per_outer_generation": ms, "indiv_gens_per_s": units / (ms / 1e3), "steps": steps,
                     "plan": json.loads(M.metade_plan_info(b.ctx))}
        b.close()
    finals = {1: [], 0: []}
    run_s = []
    for one_shot in (1, 0):
        for seed in range(args.seeds):
            b = make(M.METADE_PATH_BATCHED, seed, one_shot)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ofit = b.run_metade(wl.outer_gens, gens)
            run_s.append(time.perf_counter() - t0)
            finals[one_shot].append(ofit.min(axis=1).astype(np.float64))
            b.close()
    from scipy.stats import ranksums
    f1, f0 = np.array(finals[1]), np.array(finals[0])  # [seeds][runs]
    pvals = [float(ranksums(f1[:, r], f0[:, r])[1]) if args.seeds > 1 else None for r in range(f1.shape[1])]
    line = {"metric": "full workload: individual-gens/s per evolver generation, batched vs plain FP32",
            "workload": wl.name, "executors": wl.n_inst, "individuals": wl.individuals(),
            "inner_gens_per_outer_generation": gens, "results": out,
            "speedup_vs_plain": out["batched"]["indiv_gens_per_s"] / out["plain"]["indiv_gens_per_s"],
            "whole_runs": {"seeds": args.seeds, "outer_gens": wl.outer_gens,
                           "wall_s_per_run_median": float(np.median(run_s)),
                           "final_error_median_per_run_one_shot": [float(v) for v in np.median(f1, axis=0)],
                           "final_error_median_per_run_stream_per_executor": [float(v) for v in np.median(f0, axis=0)],
                           "ranksum_p_per_run": pvals,
                           "problems": [{"dim": p.dim, "obj": p.obj} for p in wl.problems]},
            "l2": "flushed before every timed evolver generation"}
    print(json.dumps(line), flush=True)


def run_evolvers(args):
    """The supplement's comparison of evolvers on the full workload (8 MetaDE
    runs x 128 executors, one-shot, 200 inner generations per evolver
    generation, 50 evolver generations): for DE/rand/1/bin, PSO, CSO and NES
    (xNES), --seeds whole runs each through metade_outer_generation (CUDA
    graph).  Reports the time per evolver generation (CUDA events, graph
    replays after the first), the time of the evolver's own two kernels per
    generation, the final best meta-fitness per run (median over seeds) and a
    rank-sum p-value per run against DE."""
    import numpy as np
    import torch
    import paper_2502_10470_gb300 as M
    import synth
    from scipy.stats import ranksums
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.full()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    gens = wl.inner_gens
    names = {M.EVOLVER_DE: "de", M.EVOLVER_PSO: "pso", M.EVOLVER_CSO: "cso", M.EVOLVER_NES: "nes"}
    out, finals = {}, {}
    for ev, name in names.items():
        ms, evo_ms, fin = [], [], []
        for seed in range(args.seeds):
            b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=seed, one_shot=1, n_out=wl.n_out,
                        device=dev, stream=stream.cuda_stream, evolver=ev)
            M.metade_outer_init(b.ctx, b.opop, b.ofit)
            evs = []
            for og in range(wl.outer_gens):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f,
                                          b.best_i, og, gens, True)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            if M.metade_sync(b.ctx) != M.METADE_OK:
                raise RuntimeError("device status")
            ms.append(float(np.median([a.elapsed_time(c) for a, c in evs[1:]])))
            fin.append(b.ofit.cpu().numpy().reshape(wl.n_groups, wl.n_out).min(axis=1).astype(np.float64))
            # the evolver's own kernels: phase 0 and phase 1 after the run, timed alone
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            for _ in range(20):
                M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, wl.outer_gens, 0)
                M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.best_f, wl.outer_gens, 1)
            e[1].record(stream)
            torch.cuda.synchronize()
            evo_ms.append(e[0].elapsed_time(e[1]) / 20)
            b.close()
        finals[name] = np.array(fin)  # [seeds][runs]
        out[name] = {"ms_per_outer_generation_median": float(np.median(ms)),
                     "evolver_kernels_ms_per_generation": float(np.median(evo_ms)),
                     "final_best_median_per_run": [float(v) for v in np.median(finals[name], axis=0)]}
    for name in names.values():
        out[name]["ranksum_p_vs_de_per_run"] = (
            [float(ranksums(finals[name][:, r], finals["de"][:, r])[1]) for r in range(wl.n_groups)]
            if args.seeds > 1 and name != "de" else None)
    line = {"metric": "comparison of evolvers: time per evolver generation and final best meta-fitness",
            "workload": wl.name, "executors": wl.n_inst, "inner_gens_per_outer_generation": gens,
            "outer_gens": wl.outer_gens, "seeds": args.seeds, "results": out,
            "problems": [{"dim": p.dim, "obj": p.obj} for p in wl.problems]}
    print(json.dumps(line), flush=True)


def run_mlp(args):
    """The MLP workload (64 executors x NP 100, D = 1522): batched
    generations of the MLP-objective path, timed with CUDA events after an
    L2 flush.  Roofline: FP32 FMA throughput, 256 inputs x (16 h + 2 h)
    multiply-adds = 256 * 36 h flops per evaluation (tanh not counted)
    against 152 SMs x 128 lanes x 2 flops x the sampled maximum SM clock.
    Beside it, the FP64 oracle on the host cores on a bounded sample (one
    generation of as many executors as there are cores)."""
    import numpy as np
    import torch
    import synth
    wl = synth.mlp()
    gens = wl.inner_gens
    cores = os.cpu_count() or 1
    tiny_rot = np.zeros((1, 1), dtype=np.float32)  # the objective does not read R
    tasks = [(wl.theta[k], int(wl.inst_np[k]), synth.OBJ_MLP, wl.problems[int(wl.inst_prob[k])].shift, tiny_rot, 1,
              wl.seed, k, wl.lo, wl.hi) for k in range(min(cores, wl.n_inst))]
    cpu_units, cpu_dt = time_oracle(tasks, cores, _oracle_box_job)  # before the first GPU call
    import paper_2502_10470_gb300 as M
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]

    def timed(prec):
        """(CUDA-event ms per step, ms of the MLP generations, median best, plan, clocks) of one precision."""
        b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, lo=wl.lo, hi=wl.hi,
                    device=dev, stream=stream.cuda_stream, prec=prec)
        b.set_theta(wl.theta)
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        g0 = 0
        for _ in range(args.warmup):
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, g0, gens, b.best_f, b.best_i)
            g0 += gens
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        M.metade_profile(b.ctx, True)
        M.metade_profile_read(b.ctx)
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, g0, gens, b.best_f, b.best_i)
            e1.record(stream)
            evs.append((e0, e1))
            g0 += gens
        torch.cuda.synchronize()
        clk = sampler.stop()
        prof = M.metade_profile_read(b.ctx)
        if M.metade_sync(b.ctx) != M.METADE_OK:
            raise RuntimeError("device status")
        ms_ = float(np.mean([a.elapsed_time(c) for a, c in evs]))
        kms_ = prof["mlp_generations"][0] / max(1, prof["mlp_generations"][1])
        best_ = float(np.median(b.best_f.cpu().numpy()))
        plan_ = json.loads(M.metade_plan_info(b.ctx)).get("mlp")
        b.close()
        return ms_, kms_, best_, plan_, clk

    ms, kms, best_med, _, clocks = timed(M.METADE_FP32)
    ms16, kms16, best16, plan16, _ = timed(M.METADE_BF16)
    units = float(wl.inst_np.sum()) * gens
    h = (wl.problems[0].dim - 2) // 19
    flops = units * 256 * 36 * h
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float((clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    line = {"metric": "MLP workload: individual-gens/s (MLP-objective path)", "workload": wl.name,
            "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "generations_per_step": gens, "dtype": "f32", "data": "synthetic",
            "roofline": {"bound": "fp32", "kernel": "MLP generations (k_mlp_eval dominant)",
                         "achieved": flops / (kms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / (kms / 1e3) / 1e12 / peak, "traffic": None,
                         "peak_source": "152 SMs x 128 lanes x 2 flops x %.0f MHz (max SM clock)" % sm_max},
            "cpu_baseline": {"value": cpu_units / cpu_dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d executors x NP 100 x 1 generation of the MLP workload, FP64 C oracle, "
                                       "%d spawn processes, %.1f s wall" % (len(tasks), cores, cpu_dt)},
            "best_f_median": best_med, "clocks": clocks,
            "bf16_tensor_cores": {
                "kernel": plan16["kernels"][2] if plan16 else None, "ms_per_step": ms16,
                "value": units / (ms16 / 1e3), "speedup_vs_fp32": ms / ms16, "best_f_median": best16,
                "forward_tflops": flops / (kms16 / 1e3) / 1e12,
                "layer1_tensor": {"bound": "tensor", "achieved": units * 256 * 32 * h / (kms16 / 1e3) / 1e12,
                                  "peak": bf16_peak, "unit": "TFLOP/s",
                                  "frac": units * 256 * 32 * h / (kms16 / 1e3) / 1e12 / bf16_peak,
                                  "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured"},
                "note": "the first layer (2 x 256 x 16 x h flops per evaluation) on tcgen05 in BF16; tanh, the "
                        "second layer and the error on the CUDA cores in FP32, which bound the kernel"},
            "l2": "flushed before every timed step"}
    print(json.dumps(line), flush=True)


def _case_tile_d100():
    """The D = 100 executors of the batching study (133 executors, 27556
    individuals), 20 fused generations: one k_fused_tile launch."""
    import numpy as np
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.batching()
    keep = [k for k in range(wl.n_inst) if wl.problems[k].dim == 100]
    probs = [(wl.problems[k].dim, wl.problems[k].obj, wl.problems[k].shift, wl.problems[k].rot) for k in keep]
    b = M.Batch(probs, wl.inst_np[keep], np.arange(len(keep)), seed=0, one_shot=0)
    b.set_theta(wl.theta[keep])
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 20, None, None)
    if M.metade_sync(b.ctx) != M.METADE_OK:
        raise SystemExit("device status not OK")
    b.close()


def _case_tc_d1000():
    """The precision study's 64 x 512 x D1000 state: initialisation (one
    k_rot_tc evaluation launch) and 40 BF16 generations (k_tc_rank,
    k_tc_trial, k_rot_tc selecting, k_tc_ties_wide once each per
    generation; the near ties grow from about 300 to several hundred), then
    one bf16x3 generation of the five-kernel pipeline."""
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.precision()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    for prec, gens in ((M.METADE_BF16, 40), (M.METADE_BF16X3, 1)):
        b = M.Batch(probs, wl.inst_np, wl.inst_prob, seed=0, one_shot=0, prec=prec)
        b.set_theta(wl.theta)
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, gens, None, None)
        if M.metade_sync(b.ctx) != M.METADE_OK:
            raise SystemExit("device status not OK")
        b.close()


def _case_mlp_d1522():
    """The MLP workload (64 executors x NP 100, D = 1522): initialisation and
    two generations, so 8 launches of the MLP path (k_mlp_eval twice)."""
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.mlp()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, lo=wl.lo, hi=wl.hi)
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 2, None, None)
    if M.metade_sync(b.ctx) != M.METADE_OK:
        raise SystemExit("device status not OK")
    b.close()


def _case_mlp_tc_d1522():
    """The MLP workload in a BF16 context: initialisation and two
    generations, so three k_mlp_tc launches (the initial evaluation and one
    per generation)."""
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.mlp()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, lo=wl.lo, hi=wl.hi,
                prec=M.METADE_BF16)
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 2, None, None)
    if M.metade_sync(b.ctx) != M.METADE_OK:
        raise SystemExit("device status not OK")
    b.close()


def _case_simt_d1000():
    """The precision study's 64 x 512 x D1000 state in FP32: initialisation
    and one generation, two k_rot_simt launches."""
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.precision()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, seed=0, one_shot=0, prec=M.METADE_FP32)
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
    if M.metade_sync(b.ctx) != M.METADE_OK:
        raise SystemExit("device status not OK")
    b.close()


def _case_tc_d200():
    """The full workload (8 runs x 128 executors) in BF16 with the
    tensor-core width 33 that the autotuner picks for it, so the D = 100 and
    D = 200 runs (seven of eight, 896 executors, rows ordered widest problem
    first) take the four-kernel generation: initialisation and 40
    generations (k_tc_rank, k_tc_trial2, k_tc_sel and k_tc_ties2 once each
    per generation; the size-bucket kernel of the D = 20 run beside them)."""
    import paper_2502_10470_gb300 as M
    import synth
    wl = synth.full()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=1, n_out=wl.n_out,
                prec=M.METADE_BF16, tc_min_dim=33)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 40, b.best_f, b.best_i)
    if M.metade_sync(b.ctx) != M.METADE_OK:
        raise SystemExit("device status not OK")
    b.close()


def _oracle_run_job(args):
    """One whole MetaDE run of the oracle (module-level for the spawn pool)."""
    import oracle
    n_out, np_, obj, shift, rot, inner, outer, seed = args
    oracle.build()
    oracle.metade_run(n_out, np_, obj, shift, rot, inner, outer, seed=seed)
    return n_out * np_ * inner * outer


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_oracle_timing(args):
    """The FP64 oracle alone on the host cores, one core and all cores (a
    spawn pool, one executor or run per task), on four workloads: the tiny
    workload as whole MetaDE runs (20 inner x 5 outer generations; all cores:
    one run per core, run seeds 0..cores-1), the moderate workload for 5
    inner generations, the batching workload for 1 and the precision workload
    (D 1000) for 1.  Each executor's inner DE also initialises and evaluates
    its population once, which the generations counted do not include.  No
    GPU is used.  One JSON line, rank 0 only."""
    import numpy as np
    import synth
    rank, _, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1

    def inner_tasks(wl, ks, gens):
        return [(wl.theta[k], int(wl.inst_np[k]), wl.problems[int(wl.inst_prob[k])].obj,
                 wl.problems[int(wl.inst_prob[k])].shift, wl.problems[int(wl.inst_prob[k])].rot, gens, wl.seed,
                 int(k), wl.lo, wl.hi) for k in ks]

    cases = []
    t = synth.tiny()
    p = t.problems[0]
    run = lambda s: (t.n_out, int(t.inst_np[0]), p.obj, p.shift, p.rot, t.inner_gens, t.outer_gens, s)
    cases.append(("tiny: whole MetaDE runs, evolver 8 x NP 16 x D 10, 20 x 5 generations", _oracle_run_job,
                  [run(0)], [run(s) for s in range(cores)]))
    m = synth.moderate(inner_gens=5)
    tasks = oracle_tasks(m, m.n_out, 5)
    one = [tasks[g * m.n_out] for g in range(len(m.problems))]  # one executor per run
    cases.append(("moderate: 600 executors x NP 100 x D 20, 5 generations (one core: 6 executors)",
                  _oracle_job, one, tasks))
    bt = synth.batching()
    rng = np.random.default_rng(0)
    cases.append(("batching: 512 ragged executors, NP 20..400, D 10..100, 1 generation (one core: 32 executors)",
                  _oracle_box_job, inner_tasks(bt, sorted(rng.choice(bt.n_inst, 32, replace=False)), 1),
                  inner_tasks(bt, range(bt.n_inst), 1)))
    pr = synth.precision()
    cases.append(("precision: 64 executors x NP 512 x D 1000, 1 generation (one core: 1 executor)",
                  _oracle_box_job, inner_tasks(pr, [0], 1), inner_tasks(pr, range(pr.n_inst), 1)))
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = {}
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [tasks[0][:5] + (1,) + tasks[0][6:]] * cores)  # workers up, library built
        for name, job, single, full in cases:
            u1, n1, t0 = 0, 0, time.perf_counter()
            while True:  # this process, one core; repeated to at least 0.5 s
                u1 += sum(job(a) for a in single)
                n1 += len(single)
                d1 = time.perf_counter() - t0
                if d1 >= 0.5:
                    break
            # all cores: the task list, repeated so that the pool runs about 2 s
            once = len(full) * (d1 / n1) / cores
            reps = max(1, min(64, int(2.0 / max(once, 1e-3))))
            if job is _oracle_run_job:  # whole runs: a new run seed per repetition
                full = [a[:-1] + (a[-1] + cores * r,) for r in range(reps) for a in full]
            else:
                full = full * reps
            t0 = time.perf_counter()
            un = sum(pool.map(job, full, chunksize=1))
            dn = time.perf_counter() - t0
            out[name] = {"one_core": {"value": u1 / d1, "units": u1, "s": round(d1, 3), "repeats": n1 // len(single)},
                         "all_cores": {"value": un / dn, "units": un, "s": round(dn, 3), "cores": cores,
                                       "repeats": reps}}
    print(json.dumps({"metric": "FP64 oracle on the host cores", "unit": UNIT, "kind": "oracle", "cores": cores,
                      "cpu_model": cpu_model(), "data": "synthetic", "cases": out}), flush=True)


PROFILE_CASES = {"tile-d100": _case_tile_d100, "tc-d1000": _case_tc_d1000, "mlp-d1522": _case_mlp_d1522,
                 "simt-d1000": _case_simt_d1000, "tc-d200": _case_tc_d200,
                 "mlp-tc-d1522": _case_mlp_tc_d1522}


def main(argv=None):
    args = parse_args(argv)
    if args.profile_case:
        PROFILE_CASES[args.profile_case]()
        print("profile case %s done" % args.profile_case)
        return
    if args.workload == "moderate":
        run_moderate(args)
        return
    if args.workload == "equal_error":
        run_equal_error(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "batching":
        run_batching(args)
        return
    if args.workload == "full":
        run_full(args)
        return
    if args.workload == "mlp":
        run_mlp(args)
        return
    if args.workload == "evolvers":
        run_evolvers(args)
        return
    if args.workload == "oracle":
        run_oracle_timing(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
