#!/usr/bin/env python3
"""Benchmark of the HP-MOCD generation engine (edge-evals/s).

One step = one whole NSGA-II generation of Alg. 1 (crossover, mutation,
evaluation of both objectives, environmental selection) for all N_p children,
on the LFR-style graph of the paper's scalability setup (n = 40,000, average
degree 20, maximum 50, tau1 = 2, tau2 = 1, communities 20-100, mu = 0.3),
N_p = 100, E_S = 4, C_P = 0.8, M_P = 0.2. The metric is N_p * m edge-evals per
generation divided by the device time of the generation; the K timed steps are
generations 1..K of a fresh run, after a separate warm-up run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
    python bench.py --workload batch64|serve|quality   (batched jobs, serving,
                                                        mixing sweep with NMI)

Prints one JSON line. Under torchrun each rank runs an independent replica
(a separate detection job with its own seed): weak scaling, no collective on
the data path.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "edge-evals/s (N_p*|E|*G/time)"
UNIT = "edge-evals/s"
FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", default="lfr-40k")
    ap.add_argument("--mu", type=float, default=0.3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--timing-every", type=int, default=1,
                    help="every k-th step of the stage-timing pass (after the timed steps, over the same "
                         "generations) runs the generation graph with per-stage events")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=80, help="serving trace length (--workload serve)")
    ap.add_argument("--hbm-budget-gb", type=int, default=64, help="server device-memory budget")
    ap.add_argument("--max-running", type=int, default=4, help="server concurrency limit")
    ap.add_argument("--depth", type=int, default=8, help="server: generations issued ahead per running job")
    ap.add_argument("--policy", type=int, default=0, help="server admission: 0 FIFO, 1 shortest work first")
    ap.add_argument("--preroll-s", type=float, default=0.5,
                    help="seconds of extra untimed generations before timing (clock settling)")
    ap.add_argument("--large", default="lfr-1m",
                    help="workload of the HBM-bound leg (a whole G-generation run with per-stage events); "
                         "'none' skips it")
    ap.add_argument("--large-generations", type=int, default=100)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# Multi-process plumbing (host logic, covered by a gloo test on CPU)
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_step(total_ms: float, units: float, world: int, device=None):
    """(max time over ranks, sum of units over ranks)."""
    if world == 1:
        return total_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# Workload and roofline bookkeeping
# ---------------------------------------------------------------------------

def build_workload(args):
    import synth
    spec = dict(synth.WORKLOADS[args.workload])
    if spec["kind"] == "lfr":
        rp, ci, _ = synth.workload(args.workload, seed=0, mu=args.mu)
        desc = (f"{args.workload}: LFR-style n={spec['n']}, avg deg {spec['avg_deg']}, max {spec['max_deg']}, "
                f"tau1 {spec['tau1']}, tau2 {spec['tau2']}, communities {spec['cmin']}-{spec['cmax']}, mu={args.mu}")
    else:
        rp, ci, _ = synth.workload(args.workload, seed=0)
        desc = f"{args.workload}: planted partition {spec['n_comm']}x{spec['size']}"
    return rp, ci, desc


def algorithmic_bytes(n: int, m: int, np_: int, p_mut: float, es: int = 4) -> dict:
    """Per-launch bytes of each kernel under the per-individual model of the
    method (every individual's label vector read and written as its own
    array, the CSR and the neighbour labels gathered per individual; int32
    labels and CSR): evaluation 16m + 8n, crossover 4 E_S n + 4n, mutation
    4n + 4n + M_P (16m + 8n) bytes per individual, times N_p."""
    return {
        "crossover": np_ * (4 * es * n + 4 * n),
        "mutation": np_ * (8 * n + p_mut * (16 * m + 8 * n)),
        "evaluate": np_ * (16 * m + 8 * n),
        "select": 0,
    }


def access_bytes(n: int, m: int, np_: int, p_mut: float) -> dict:
    """Per-launch bytes of the node-major kernels as built (rows of W int32
    labels per node, the CSR streamed once per population, each undirected
    edge read once by the evaluation), with no reuse beyond what a kernel
    stages explicitly."""
    W = (np_ + 3) & ~3
    csr = 4 * (n + 1) + 4 * 2 * m
    oriented = 4 * (n + 1) + 4 * m + 4 * n  # the evaluation's oriented CSR and the node order
    return {
        # P half + Q rows in, next P + children rows out
        "crossover": 16 * W * n,
        # own row in, Q row out, each selected pair's neighbour labels, CSR, and the degree-histogram
        # additions of every child's final label (read-modify-write of a 4-byte cell)
        "mutation": 8 * W * n + 4 * p_mut * np_ * 2 * m + csr + 8 * np_ * n,
        # own rows, one neighbour row per undirected edge (the oriented CSR lists each edge once),
        # that CSR, and the sweep of the [n][W] degree histogram that forms sum_c D_c^2
        "evaluate": 4 * W * n + 4 * W * m + oriented + 4 * W * n,
        "select": 0,
    }


def kernel_roofline(kernel: str, ms: float, n: int, m: int, np_: int, p_mut: float, peak: float,
                    peak_kind: str, workload: str) -> dict:
    """HBM roofline of one kernel from its mean CUDA-event duration: the
    per-individual bytes of the method (``achieved``/``frac``) and the
    node-major access bytes (``*_access``) side by side, and the ncu DRAM
    traffic per launch when a committed summary was taken on this source."""
    alg = algorithmic_bytes(n, m, np_, p_mut)[kernel]
    acc = access_bytes(n, m, np_, p_mut)[kernel]
    a = alg / (ms / 1e3) / 1e9
    b = acc / (ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
            "peak_source": peak_kind, "traffic": recorded_traffic(kernel, workload),
            "bytes_model": "per-individual (16m + 8n evaluation; 4 E_S n + 4n crossover; "
                           "8n + M_P (16m + 8n) mutation; x N_p)",
            "algorithmic_bytes_per_launch": alg, "launch_ms": ms,
            "access_bytes_per_launch": acc, "achieved_access": b, "frac_access": b / peak}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {"crossover": "k_variation.cu", "mutation": "k_variation.cu",
                  "evaluate": "k_eval.cu", "select": "k_select.cu"}


def source_digest(kernel: str) -> str:
    path = os.path.join(ROOT, "paper_2506_01752_gb300", "csrc", KERNEL_SOURCES[kernel])
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of that kernel."""
    pat = re.compile(rf"traffic_bytes_per_launch\[{kernel}@{re.escape(workload)}\]:\s*([0-9.eE+]+)\s+"
                     r"source_sha256_16:\s*([0-9a-f]+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                mt = pat.search(line)
                if mt and mt.group(2) == source_digest(kernel):
                    return float(mt.group(1))
    return None


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

def _gpu_index() -> int:
    """nvidia-smi index of this process's (first visible) GPU."""
    return int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or 0)


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def cpu_description() -> dict:
    """The host CPU the oracle runs on: model name (lscpu, else /proc/cpuinfo,
    else the platform string) and the number of online cores."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def cpu_oracle_sample(rp, ci, seed: int, budget_s: float = 12.0, max_gens: int = 6):
    """The oracle as it stands, single-threaded, for whole generations of the
    same workload until the budget is spent."""
    import oracle
    oracle.build()
    params = oracle.Params(seed=seed)
    st = oracle.population_init(rp, ci, params)
    m = int(rp[-1] // 2)
    gens, t0 = 0, time.perf_counter()
    while gens < max_gens:
        st = oracle.run(rp, ci, params, st, 1)
        gens += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": params.pop_size * m * gens / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{gens} whole generations (N_p={params.pop_size}) of the same workload, "
                      f"single-threaded C oracle, {dt:.1f} s", **cpu_description()}


def cpu_oracle_sample_all_cores(rp, ci, seed: int, budget_s: float = 6.0, max_gens: int = 20):
    """The oracle's threaded form (each generation's children split over all
    host cores; the same sequential code per child, so the same result) for
    whole generations of the same workload until the budget is spent."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    params = oracle.Params(seed=seed)
    st = oracle.population_init(rp, ci, params)
    m = int(rp[-1] // 2)
    gens, t0 = 0, time.perf_counter()
    while gens < max_gens:
        st = oracle.run_parallel(rp, ci, params, st, 1, threads)
        gens += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": params.pop_size * m * gens / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{gens} whole generations (N_p={params.pop_size}) of the same workload, children of "
                      f"each generation over {threads} host threads, {dt:.1f} s", **cpu_description()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    rp, ci, desc = build_workload(args)
    oracle.build()
    params = oracle.Params(seed=args.seed)
    st = oracle.population_init(rp, ci, params)
    m = int(rp[-1] // 2)
    chunk = 10  # children per step: a bounded sample of one generation
    gen = 1

    def step(k):
        i0 = (k * chunk) % params.pop_size
        oracle.make_offspring_range(rp, ci, params, gen, st, i0, i0 + chunk)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = time.perf_counter() - t0
    value = chunk * m * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": desc, "n": int(rp.size - 1), "m": m, "pop_size": params.pop_size,
                   "step": f"{chunk} of the {params.pop_size} children of one generation "
                           "(crossover, mutation, evaluation) by the CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x {chunk} children, single-threaded C oracle",
                         **cpu_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def large_leg(args, dev, stream, peak, peak_kind):
    """HBM-bound leg: a whole run of the large workload (generations
    1..G of a fresh population, per-stage CUDA events on every generation,
    L2 flushed between generations), where the label matrix and the degree
    histogram no longer fit in L2. Reports the mean stage times and the HBM
    roofline of the evaluation and mutation kernels over the run."""
    import torch
    import paper_2506_01752_gb300 as mocd
    import synth

    spec = synth.WORKLOADS[args.large]
    rp, ci, _ = synth.workload(args.large, seed=0)
    n, m = int(rp.size - 1), int(rp[-1] // 2)
    params = mocd.Params(seed=args.seed)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ctx = mocd.graph_upload(rp, ci, stream)
    try:
        mocd.population_init(ctx, params)
        mocd.set_timing(ctx, True)
        mocd.generation(ctx, 3)  # warm-up, then a fresh run
        mocd.population_init(ctx, params)
        mocd.synchronize(ctx)
        sampler = ClockSampler(_gpu_index())
        sampler.start()
        step_ms, stages = [], {s: [] for s in mocd.STAGES}
        for _ in range(args.large_generations):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0.record(stream)
            mocd.generation(ctx, 1)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            for s_, v in mocd.kernel_times(ctx).items():
                stages[s_].append(v)
        clocks = sampler.stop()
    finally:
        mocd.destroy(ctx)
    mean = {s_: statistics.fmean(v) for s_, v in stages.items()}
    G = args.large_generations
    return {
        "workload": f"{args.large}: LFR-style n={n}, m={m}, avg deg {spec['avg_deg']}, max {spec['max_deg']}, "
                    f"communities {spec['cmin']}-{spec['cmax']}, mu={spec['mu']}",
        "generations": f"1-{G} of a fresh run, per-stage events on every generation, L2 flushed between",
        "value": params.pop_size * m * G / (sum(step_ms) / 1e3), "unit": UNIT,
        "ms_per_step": sum(step_ms) / G,
        "stage_ms": {k: round(v, 4) for k, v in mean.items()},
        "evaluate": kernel_roofline("evaluate", mean["evaluate"], n, m, params.pop_size, params.p_mutation,
                                    peak, peak_kind, args.large),
        "mutation": kernel_roofline("mutation", mean["mutation"], n, m, params.pop_size, params.p_mutation,
                                    peak, peak_kind, args.large),
        "clocks": clocks,
    }


def run_mine(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2506_01752_gb300 as mocd
    mocd.build.build()
    rp, ci, desc = build_workload(args)
    n = int(rp.size - 1)
    m = int(rp[-1] // 2)
    params = mocd.Params(seed=args.seed + rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = mocd.graph_upload(rp, ci, stream)
    mocd.population_init(ctx, params)
    kernels_per_generation = mocd.generation_kernels(ctx)
    mocd.set_timing(ctx, True)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if world == 1 else local
    sampler = ClockSampler(index)
    sampler.start()
    # Warm-up: W generations (both generation graphs, with and without stage
    # events, get captured here), then a short pre-roll so that clocks settle.
    for w in range(args.warmup):
        mocd.set_timing(ctx, w % 2 == 0)
        mocd.generation(ctx, 1)
    mocd.set_timing(ctx, False)
    t_end = time.perf_counter() + args.preroll_s
    pre = 0
    while time.perf_counter() < t_end:
        mocd.generation(ctx, 20)
        mocd.synchronize(ctx)
        pre += 20
    mocd.synchronize(ctx)
    # The timed steps are generations 1..K of a fresh run (the configuration's
    # G-generation job), not a population that the warm-up has already
    # converged: re-initialising puts the run back to generation 0.
    mocd.population_init(ctx, params)
    mocd.synchronize(ctx)
    barrier(world)
    torch.cuda.synchronize()

    # The K timed steps run the plain generation graph. The per-stage
    # durations come from a second pass over the same generations 1..K of a
    # fresh run, whose steps run the graph with CUDA events between the
    # stages (every --timing-every-th step); those events cost a step about
    # 20 us, so they stay out of the timed steps. Both graphs hold the same
    # kernels.
    step_ms = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps, outside the events
        ev0.record(stream)
        mocd.generation(ctx, 1)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()

    stages = {s: [] for s in mocd.STAGES}
    every = max(1, args.timing_every)
    mocd.population_init(ctx, params)
    for k in range(args.steps):
        timed = k % every == 0
        mocd.set_timing(ctx, timed)
        with torch.cuda.stream(stream):
            flush.zero_()
        mocd.generation(ctx, 1)
        mocd.synchronize(ctx)
        if timed:
            for s_, v in mocd.kernel_times(ctx).items():
                stages[s_].append(v)
    mocd.set_timing(ctx, False)

    total_ms, units = reduce_step(sum(step_ms), float(params.pop_size * m * args.steps), world,
                                  device=dev if world > 1 else None)
    value = units / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    mean_stage = {s: statistics.fmean(v) for s, v in stages.items()}
    kernels = {k: mean_stage[k] for k in ("crossover", "mutation", "evaluate", "select")}
    dominant = max(kernels, key=kernels.get)
    peak, peak_kind = measured_peaks()
    roofline = kernel_roofline(dominant, kernels[dominant], n, m, params.pop_size, params.p_mutation, peak,
                               peak_kind, args.workload)
    roofline["stage_ms"] = {k: round(v, 5) for k, v in mean_stage.items()}
    roofline["stage_events_every"] = every
    # The objective (evaluation) kernel, against the same HBM roofline.
    roofline_objective = kernel_roofline("evaluate", kernels["evaluate"], n, m, params.pop_size,
                                         params.p_mutation, peak, peak_kind, args.workload)

    e2e = None
    if not args.no_e2e:
        # The same metric through the public C ABI from host buffers: upload
        # the CSR, initialise, run `steps` generations, read the front back.
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = mocd.graph_upload(rp, ci, stream)
        mocd.population_init(h, params)
        mocd.generation(h, args.steps)
        fr = mocd.pareto_front(h)
        t1 = time.perf_counter()
        mocd.destroy(h)
        h2d = rp.nbytes + ci.nbytes
        d2h = fr.labels.nbytes + fr.f1.nbytes + fr.f2.nbytes + fr.intra.nbytes + fr.sumsq.nbytes
        e2e_t, e2e_units = reduce_step((t1 - t0) * 1e3, float(params.pop_size * m * args.steps), world,
                                       device=dev if world > 1 else None)
        e2e = {"value": e2e_units / (e2e_t / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "job": f"graph upload + init + {args.steps} generations + front download, host buffers",
               "job_ms": round(e2e_t, 3)}

    mocd.destroy(ctx)
    large = None
    if world == 1 and args.large != "none":
        large = large_leg(args, dev, stream, peak, peak_kind)
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(rp, ci, args.seed)
        cpu_all = cpu_oracle_sample_all_cores(rp, ci, args.seed)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "n": n, "m": m, "pop_size": params.pop_size, "n_parents": params.n_parents,
                       "p_crossover": params.p_crossover, "p_mutation": params.p_mutation,
                       "step": "one generation of Alg. 1 (crossover, mutation, evaluation, selection)",
                       "l2": f"flushed between timed steps ({FLUSH_BYTES >> 20} MB write, outside the events)",
                       "parallelism": f"{world} independent replica(s)",
                       "warmup_generations": args.warmup + pre,
                       "timed_generations": f"1-{args.steps} of a fresh run (population re-initialised after the warm-up)"},
            "roofline": roofline,
            "roofline_objective": roofline_objective,
            "roofline_hbm": large,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e,
            "gpu_launches": kernels_per_generation * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


FORMS = {0: "per-member kernel chains", 1: "per-member chains, one merged selection launch",
         2: "one launch per stage for all members (mutation kernels per member)"}


def run_batch(args):
    """64 uneven jobs (synth.batch_instances): one batched CUDA-graph launch
    per generation of all of them, against the plain path that runs one
    instance's generation graph after another on the same GPU. A step is one
    generation of every job; both arms time the same K generations per job
    with CUDA events and the same L2 flush between steps."""
    import torch
    import paper_2506_01752_gb300 as mocd
    import synth

    torch.cuda.set_device(0)
    mocd.build.build()
    insts = synth.batch_instances(64, seed=0)
    units = float(sum(100 * int(rp[-1] // 2) for rp, _, _, _ in insts))
    stream = torch.cuda.Stream()
    ctxs = [mocd.graph_upload(rp, ci) for rp, ci, _, _ in insts]
    params = [mocd.Params(seed=k) for k in range(len(ctxs))]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def init_all():
        for c, p in zip(ctxs, params):
            mocd.population_init(c, p)

    init_all()
    b = mocd.batch_create(ctxs, stream)
    shape = mocd.batch_autotune(b, 2)
    _, form = mocd.batch_form(b)
    mocd.batch_destroy(b)
    init_all()
    b = mocd.batch_create(ctxs, stream)
    mocd.batch_configure(b, shape, form)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed(step):
        out = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            ev0.record(stream)
            step()
            ev1.record(stream)
            ev1.synchronize()
            out.append(ev0.elapsed_time(ev1))
        return out

    mocd.batch_generation(b, args.warmup)
    mocd.batch_synchronize(b)
    sampler = ClockSampler(_gpu_index())
    sampler.start()
    batch_ms = timed(lambda: mocd.batch_generation(b, 1))
    mocd.batch_synchronize(b)
    mocd.batch_destroy(b)
    # The other forms at the same shape, for comparison (the same generations
    # of fresh populations).
    other_ms = {}
    for other in (0, 1, 2):
        if other == form:
            continue
        init_all()
        b = mocd.batch_create(ctxs, stream)
        mocd.batch_configure(b, shape, other)
        mocd.batch_generation(b, args.warmup)
        mocd.batch_synchronize(b)
        other_ms[other] = statistics.fmean(timed(lambda: mocd.batch_generation(b, 1)))
        mocd.batch_synchronize(b)
        mocd.batch_destroy(b)

    # Plain path: each instance's own generation graph, one instance at a time.
    init_all()
    for c in ctxs:
        mocd.generation(c, args.warmup)
        mocd.synchronize(c)
    per_job = np.zeros(len(ctxs))

    def plain_step():
        for k, c in enumerate(ctxs):
            mocd.generation(c, 1)
            mocd.synchronize(c)

    plain_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, c in enumerate(ctxs):
            mocd.generation(c, 1)
            mocd.synchronize(c)
            per_job[k] += (time.perf_counter() - t0) * 1e3
        plain_ms.append((time.perf_counter() - t0) * 1e3)
    clocks = sampler.stop()
    for c in ctxs:
        mocd.destroy(c)

    bt = statistics.fmean(batch_ms)
    pt = statistics.fmean(plain_ms)
    # Job completion latency for G = steps generations, all jobs submitted at
    # once: batched, every job ends with the last batch step; plain, job k
    # ends after the jobs before it (per_job[k] = its cumulative time).
    batch_lat = np.full(len(ctxs), sum(batch_ms))
    line = {
        "metric": METRIC + " [batched jobs]", "value": units / (bt / 1e3), "unit": UNIT,
        "value_plain": units / (pt / 1e3), "speedup_vs_plain": pt / bt,
        "form": FORMS[form],
        "ms_per_step_other_forms": {FORMS[k]: v for k, v in other_ms.items()},
        "ms_per_step": bt, "ms_per_step_plain": pt, "steps": args.steps, "warmup": args.warmup,
        "job_latency_ms": {"batched_p50": float(np.percentile(batch_lat, 50)),
                           "batched_p99": float(np.percentile(batch_lat, 99)),
                           "plain_p50": float(np.percentile(per_job, 50)),
                           "plain_p99": float(np.percentile(per_job, 99))},
        "config": {"workload": "64 jobs: n log-uniform 1e3-5e4, avg degree U[10,30], mu U[0.2,0.5], "
                               "half planted partition, half LFR-style; N_p=100 each",
                   "total_n": int(sum(rp.size - 1 for rp, _, _, _ in insts)),
                   "total_m": int(sum(rp[-1] // 2 for rp, _, _, _ in insts)),
                   "autotuned_nodes_per_warp": shape,
                   "plain": "per-instance generation graph, instances one after another",
                   "l2": f"flushed between timed steps ({FLUSH_BYTES >> 20} MB write)"},
        "n_gpus": 1, "higher_is_better": True, "dtype": "int32", "data": "synthetic", "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson stream of detection requests (20/s, G = 100, graphs from
    synth.serving_pool), served by the continuous-batching server and, for
    comparison, by plain serial processing of the same trace (upload, init,
    100 generations, front download, one request after another)."""
    import torch
    import paper_2506_01752_gb300 as mocd
    import synth

    torch.cuda.set_device(0)
    mocd.build.build()
    pool = synth.serving_pool(12, seed=0)
    rng = np.random.default_rng(1)
    n_req, rate, G = args.requests, 20.0, 100
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    picks = rng.integers(0, len(pool), n_req)
    seeds = rng.integers(0, 1 << 31, n_req)
    units = float(sum(100 * G * int(pool[k][0][-1] // 2) for k in picks))

    def lat_stats(lat, makespan):
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(np.mean(lat)), "makespan_s": makespan,
                "edge_evals_per_s": units / makespan}

    # warm up the library and the device
    rp, ci, _ = pool[0]
    h = mocd.graph_upload(rp, ci)
    mocd.population_init(h, mocd.Params())
    mocd.generation(h, 5)
    mocd.pareto_front(h)
    mocd.destroy(h)

    sampler = ClockSampler(_gpu_index())
    sampler.start()
    # Continuous-batching server (background scheduler + admission workers).
    srv = mocd.Server(args.hbm_budget_gb << 30, max_running=args.max_running, depth=args.depth)
    srv.start(admission_threads=2, policy=args.policy)
    t0 = time.perf_counter()
    ids, done_at, submitted = [], {}, 0
    while len(done_at) < n_req:
        now = time.perf_counter() - t0
        while submitted < n_req and arrivals[submitted] <= now:
            k = picks[submitted]
            ids.append(srv.submit(pool[k][0], pool[k][1], mocd.Params(seed=int(seeds[submitted])), G))
            submitted += 1
        srv.step()
        now = time.perf_counter() - t0
        for i, jid in enumerate(ids):
            if i not in done_at and srv.state(jid)[0] >= mocd.Server.DONE:
                done_at[i] = now
        time.sleep(0.0005)
    srv_make = max(done_at.values())
    srv_lat = np.array([done_at[i] - arrivals[i] for i in range(n_req)])
    failed = sum(1 for j in ids if srv.state(j)[0] == mocd.Server.FAILED)
    srv.close()

    # Plain serial processing of the same trace.
    t0 = time.perf_counter()
    plain_lat = []
    for i in range(n_req):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        k = picks[i]
        h = mocd.graph_upload(pool[k][0], pool[k][1])
        mocd.population_init(h, mocd.Params(seed=int(seeds[i])))
        mocd.generation(h, G)
        mocd.pareto_front(h)
        mocd.destroy(h)
        plain_lat.append(time.perf_counter() - t0 - arrivals[i])
    plain_make = time.perf_counter() - t0
    clocks = sampler.stop()

    line = {
        "metric": "detection request latency p50/p99 (s) and edge-evals/s [serving]",
        "server": lat_stats(srv_lat, srv_make), "plain_serial": lat_stats(np.array(plain_lat), plain_make),
        "failed": failed, "requests": n_req, "rate_per_s": rate, "generations": G,
        "config": {"workload": "Poisson 20/s; LFR-style graphs, n log-spaced 1e3-1e6 (12-graph pool), "
                               "mu U[0.1,0.6]; N_p=100, G=100",
                   "hbm_budget_gb": args.hbm_budget_gb, "max_running": args.max_running, "depth": args.depth,
                   "admission": "highest response ratio next" if args.policy else "first come first served",
                   "admission_threads": 2,
                   "pool": [d for _, _, d in pool]},
        "n_gpus": 1, "dtype": "int32", "data": "synthetic", "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_quality(args):
    """The paper's mixing sweep at the benchmark size: for mu = 0.1 .. 0.7 and
    each initialisation, one whole detection run (population init, G = 100
    generations, Pareto front and Alg. 3's recommended member) on the LFR-style
    n = 40,000 graph; run time on the device (CUDA events around init ..
    front) and wall-clock from graph upload to the returned front, then the
    recommended member scored against the planted communities."""
    import torch
    import paper_2506_01752_gb300 as mocd
    import synth
    from synth import quality

    torch.cuda.set_device(0)
    mocd.build.build()
    stream = torch.cuda.Stream()
    G = 100
    rows = []
    sampler = ClockSampler(_gpu_index())
    sampler.start()
    for mu in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7):
        rp, ci, truth = synth.workload("lfr-40k", seed=args.seed, mu=mu)
        m = int(rp[-1] // 2)
        for init_mode in (0, 1):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = mocd.graph_upload(rp, ci, stream)
            try:
                ev0.record(stream)
                mocd.population_init(h, mocd.Params(seed=args.seed, init_mode=init_mode))
                mocd.generation(h, G)
                ev1.record(stream)
                fr = mocd.pareto_front(h)
                wall = time.perf_counter() - t0
            finally:
                mocd.destroy(h)
            ev1.synchronize()
            lab = fr.labels[fr.best]
            rows.append({
                "mu": mu, "init_mode": init_mode, "n": int(rp.size - 1), "m": m,
                "device_ms": round(ev0.elapsed_time(ev1), 3), "wall_s": round(wall, 4),
                "front": int(fr.f1.size), "modularity": round(1.0 - fr.f1[fr.best] - fr.f2[fr.best], 6),
                "communities": int(np.unique(lab).size), "truth_communities": int(np.unique(truth).size),
                "nmi": round(quality.nmi(lab, truth), 4), "ami": round(quality.ami(lab, truth), 4),
                "f1": round(quality.pairwise_f1(lab, truth), 4),
            })
    clocks = sampler.stop()
    line = {
        "metric": "whole-run quality and run time (G = 100)", "unit": "NMI / ms", "clocks": clocks,
        "workload": "lfr-40k mixing sweep", "rows": rows, "n_gpus": 1, "dtype": "int32",
        "data": "synthetic", "config": {"workload": "lfr-40k", "N_p": 100, "G": G, "E_S": 4,
                                        "C_P": 0.8, "M_P": 0.2, "seed": args.seed},
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "quality":
        return run_quality(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
