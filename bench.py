#!/usr/bin/env python3
"""Throughput benchmark of the QIEO generation loop on GB300.

One step = one full solve of the named workload: reset to generation 0 (a0), then every
generation's CIP + QIP + Evaluation + DetermineElite (a1-a4, one fused kernel each) and the
final CIP (a5). The metric is gene-updates/s = Np * Ng * generations / time, summed over
all ranks (each rank solves its own independent instance: weak scaling, no collective on
the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1]
  python bench.py --workload c4           # 256 uneven instances, batched (solves/s)
  python bench.py --workload c5           # served Poisson stream (solves/s, p50/p99)
  python bench.py --impl reference ...    # the CPU oracle timed on the host cores

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import platform
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_30862_gb300 import workload as WL  # noqa: E402

METRIC = "gene-updates/s (Np*Ng*gens) & % roofline"
UNIT = "gene-updates/s"
SM_COUNT = 152
STATE_BYTES_PER_GENE = 4          # int16 angle index read + written once per generation
# Generations whose single-launch times represent the two phases of a run of the
# HBM-resident instance: every qubit still drawn (the population spread) and every qubit
# saturated on the elite's side (fixed-allele passes).
SPREAD_WINDOW = (45, 55)
SATURATED_WINDOW = (185, 195)
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WL.WORKLOADS) + ["c4", "c5"])
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--rate", type=float, default=0.0,
                    help="c5 arrivals per second (0: 0.8 x the measured batched capacity)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--per-generation", action="store_true",
                    help="c4: one batched launch per generation (QIEO_FLAG_PER_GENERATION on the "
                         "members) instead of one persistent launch per run")
    ap.add_argument("--state-i8", action="store_true",
                    help="c1-c3: store the angle indices as bytes (QIEO_FLAG_STATE_I8)")
    ap.add_argument("--streamed", action="store_true",
                    help="c1-c3: never keep the state resident in shared memory (QIEO_FLAG_STREAMED)")
    ap.add_argument("--no-fixed-words", action="store_true",
                    help="c1-c3: keep no fixed-vector words, so every generation runs the dense "
                         "pass (QIEO_FLAG_NO_FIXED_WORDS)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-phases", action="store_true",
                    help="c1-c3: skip the per-generation timing run and the integer ceiling")
    ap.add_argument("--phases", action="store_true",
                    help="per-step breakdown (CIP, QIP, Evaluation, DetermineElite) of the "
                         "unfused form, and device vs host DetermineElite, on --workload")
    ap.add_argument("--sweep", action="store_true",
                    help="time per generation over the paper's (Np, Ng) grid")
    ap.add_argument("--sweep-max-gb", type=float, default=120.0,
                    help="--sweep: skip pairs whose instance needs more device memory")
    ap.add_argument("--ref-budget-s", type=float, default=150.0,
                    help="--impl reference: seconds of oracle work over warm-up + timed steps")
    ap.add_argument("--oracle-scan", action="store_true",
                    help="the oracle's rate on --workload at 1 thread (serial build) and at 1, 8, "
                         "16 and all threads (OpenMP build), on the host cores")
    return ap.parse_args()


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest of one float over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def workload_config(name: str, state_i8: bool = False) -> dict:
    c = WL.WORKLOADS[name]
    return {
        "workload": "%s: 0/1 knapsack Ng=%d items (w uniform [1,10], v=w+5, W=floor(sum w/2)), "
                    "Np=%d chromosomes, %d generations, dtheta=0.01pi, start pi/4, %s angle "
                    "state, Philox seed %d" % (name, c["ng"], c["np"], c["gens"],
                                               "int8" if state_i8 else "int16", c["seed"]),
        "ng": c["ng"], "np": c["np"], "generations": c["gens"], "rotation_rule": "R1",
    }


def load_peaks() -> tuple[dict, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def profile_traffic(kernel: str, workload: str):
    """DRAM traffic per generation (read + write bytes; per launch for the kernels launched
    once per generation) from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_generation:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


def kernel_source_hash() -> str:
    import hashlib
    hs = hashlib.sha256()
    for name in ("qieo_device.cuh", "qieo_kernels.cuh", "qieo_api.cu"):
        with open(os.path.join(ROOT, "paper_2609_30862_gb300", "csrc", name), "rb") as fh:
            hs.update(fh.read())
    return hs.hexdigest()[:16]


# ------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.count(",") >= 8]
        sm, mx, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p >= 0.5 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


def gpu_id_for_smi(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return vis.split(",")[dev] if vis else str(dev)


# ------------------------------------------------------------------------- CPU oracle

def oracle_sample(name: str, target_s: float = 10.0):
    """The OpenMP build of the oracle, as it stands, on all host cores, over the first
    generations of the named workload. Returns (gene-updates/s, cores, sample text)."""
    from oracle import oracle as O
    c = WL.WORKLOADS[name]
    prob = WL.knapsack(c["ng"], c["item_seed"])
    cores = os.cpu_count() or 1
    O.build()
    O.set_threads(cores)
    t0 = time.perf_counter()
    O.run(prob, c["np"], 1, seed=c["seed"], inst=c["inst"], kind="omp", threads=cores)
    t1 = time.perf_counter() - t0
    gens = int(max(1, min(c["gens"], round(target_s / max(t1, 1e-6)))))
    t0 = time.perf_counter()
    O.run(prob, c["np"], gens, seed=c["seed"], inst=c["inst"], kind="omp", threads=cores)
    dt = time.perf_counter() - t0
    rate = c["np"] * c["ng"] * gens / dt
    sample = "first %d of %d generations of %s (Np=%d, Ng=%d), OpenMP build, %d threads" % (
        gens, c["gens"], name, c["np"], c["ng"], cores)
    return rate, cores, sample, gens, dt


def run_oracle_scan(a):
    """The oracle, as it stands, on the host cores: its serial build and its OpenMP build
    (parallel over chromosomes, the same results) at 1, 8, 16 and all threads, each over
    the first generations of the workload that fill about 8 seconds. One JSON line."""
    from oracle import oracle as O
    name = a.workload if a.workload in WL.WORKLOADS else "c2"
    c = WL.WORKLOADS[name]
    prob = WL.knapsack(c["ng"], c["item_seed"])
    O.build()
    cores = os.cpu_count() or 1
    runs = [("serial", 1)] + [("omp", n) for n in sorted({1, 8, 16, cores}) if n <= cores]
    out = []
    for kind, n in runs:
        if kind == "omp":
            O.set_threads(n)
        t0 = time.perf_counter()
        O.run(prob, c["np"], 1, seed=c["seed"], inst=c["inst"], kind=kind, threads=n)
        t1 = time.perf_counter() - t0
        gens = int(max(1, min(c["gens"], round(8.0 / max(t1, 1e-6)))))
        t0 = time.perf_counter()
        O.run(prob, c["np"], gens, seed=c["seed"], inst=c["inst"], kind=kind, threads=n)
        dt = time.perf_counter() - t0
        out.append({"build": kind, "threads": n, "generations": gens, "seconds": round(dt, 3),
                    "gene_updates_per_s": c["np"] * c["ng"] * gens / dt})
    print(json.dumps({"oracle_scan": name, "np": c["np"], "ng": c["ng"], "host_cores": cores,
                      "cpu": platform.processor() or platform.machine(), "runs": out}), flush=True)


def run_reference(a):
    """--impl reference: the CPU oracle (OpenMP build, all host cores) timed per step on a
    bounded sample of the same workload. Rank 0 only."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    if a.workload in ("c4", "c5"):
        run_reference_solves(a)
        return
    from oracle import oracle as O
    c = WL.WORKLOADS[a.workload]
    prob = WL.knapsack(c["ng"], c["item_seed"])
    cores = os.cpu_count() or 1
    O.build()
    budget_s = a.ref_budget_s
    t0 = time.perf_counter()
    O.run(prob, c["np"], 1, seed=c["seed"], inst=c["inst"], kind="omp", threads=cores)
    t1 = time.perf_counter() - t0
    per_step = budget_s / max(1, a.steps + a.warmup)
    gens = int(max(1, min(c["gens"], per_step / max(t1, 1e-6))))
    for _ in range(a.warmup):
        O.run(prob, c["np"], gens, seed=c["seed"], inst=c["inst"], kind="omp", threads=cores)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        O.run(prob, c["np"], gens, seed=c["seed"], inst=c["inst"], kind="omp", threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = c["np"] * c["ng"] * gens * a.steps / total
    sample = "first %d of %d generations of %s per step (Np=%d, Ng=%d), OpenMP build, %d threads" % (
        gens, c["gens"], a.workload, c["np"], c["ng"], cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(a.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_solves(a):
    """Reference arm of the batched (c4) and served (c5) workloads: the oracle solving the
    manifest's instances (300 generations each) in order, a bounded number per step, on all
    host cores. The metric is solves/s."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    O.build()
    G = 300
    specs = WL.batch_manifest(256 if a.workload == "c4" else a.requests, first_seed=1)
    budget_s = a.ref_budget_s / max(1, a.steps + a.warmup)
    pos, times, counts = 0, [], []
    for k in range(a.warmup + a.steps):
        t0, done = time.perf_counter(), 0
        while time.perf_counter() - t0 < budget_s or done == 0:
            sp = specs[pos % len(specs)]
            pos += 1
            O.run(WL.knapsack(sp.ng, sp.seed), sp.np_, G, seed=sp.seed, inst=sp.seed,
                  kind="omp", threads=cores)
            done += 1
        if k >= a.warmup:
            times.append(time.perf_counter() - t0)
            counts.append(done)
    total = sum(times)
    value = sum(counts) / total
    sample = "%d manifest instances x %d generations per step on average, OpenMP build, %d threads" % (
        round(sum(counts) / len(counts)), G, cores)
    line = {
        "impl": "reference", "metric": "solves/s", "value": value, "unit": "solves/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "%s: manifest instances (Ng log-uniform [50, 20000], Np uniform "
                               "{32,64,128,256,512}), 300 generations" % a.workload},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- GPU path

def run_gpu(a):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2609_30862_gb300 import qieo as Q
    Q.load()
    c = WL.WORKLOADS[a.workload]
    prob = WL.knapsack(c["ng"], c["item_seed"])
    np_, ng, G = c["np"], c["ng"], c["gens"]
    genes_per_step = np_ * ng * G
    stream = torch.cuda.Stream()
    flags = ((Q.QIEO_FLAG_STATE_I8 if a.state_i8 else 0) | (Q.QIEO_FLAG_STREAMED if a.streamed else 0) |
             (Q.QIEO_FLAG_NO_FIXED_WORDS if a.no_fixed_words else 0))
    inst = Q.Instance(prob, np_, seed=c["seed"], inst=c["inst"] + rank,
                      stream=stream.cuda_stream, flags=flags)
    shape = inst.shape()
    state_bytes = np_ * ((ng + 7) // 8) * (8 if a.state_i8 else 16)
    flush = state_bytes < 2 * L2_BYTES
    flush_buf = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda") if flush else None

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            if flush:
                flush_buf.fill_(1)
            inst.reset()
            inst.run(G)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        sampler = ClockSampler(gpu_id_for_smi(torch, local)) if rank == 0 else None
        if sampler:
            sampler.start()
        barrier()
        wall0 = time.perf_counter()
        for i in range(a.steps):
            if flush:
                flush_buf.fill_(i & 0xFF)
            evs[i][0].record(stream)
            inst.reset()
            evs[i][1].record(stream)
            inst.run(G)
            evs[i][2].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
        clocks = sampler.stop() if sampler else None
    step_ms = [e0.elapsed_time(e2) for e0, _, e2 in evs]
    run_ms = [e1.elapsed_time(e2) for _, e1, e2 in evs]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dist)
    run_total_ms = max_over_ranks(float(sum(run_ms)), dist)
    value = world * genes_per_step * a.steps / (total_ms / 1e3)

    # Roofline of the fused generation kernel. A run is G launches of generation_kernel +
    # one final CIP launch, timed with events on its stream; the per-generation duration is
    # that time / G (an upper bound on one launch: it includes the CIP pass and the gaps).
    # Per gene-update the kernel moves 4 B of state (int16 read + written) and does the
    # drawn pass's integer work (a quarter Philox4x32-10 call, CIP, the compare, the allele
    # bit, the item sums); its two ceilings are the measured HBM copy bandwidth and the
    # measured integer ceiling (qieo_measure_integer_ceiling, the same per-gene arithmetic
    # with nothing streamed), and the bound is the slower of the two.
    launch_s = run_total_ms / 1e3 / (a.steps * G)
    peaks, peak_src = load_peaks()
    genes_per_launch = np_ * ng
    hbm_peak = float(peaks["hbm_gbs"])
    state_bpg = 2 if a.state_i8 else STATE_BYTES_PER_GENE   # byte state: 1 B read + 1 B written
    t_hbm = state_bpg * genes_per_launch / (hbm_peak * 1e9)
    ceiling = None if a.no_phases else Q.qieo_measure_integer_ceiling(5)
    int_peak = ceiling.drawn_genes_per_s if ceiling is not None else None
    t_int = genes_per_launch / int_peak if int_peak else 0.0
    l2_resident = state_bytes < L2_BYTES
    hbm_achieved = state_bpg * genes_per_launch / launch_s / 1e9
    if t_hbm >= t_int:
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_achieved / hbm_peak, "peak_source": "%s hbm_gbs" % peak_src}
    else:
        achieved = genes_per_launch / launch_s / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": int_peak / 1e9,
                "unit": "Ggene-updates/s", "frac": achieved / (int_peak / 1e9),
                "peak_source": "measured: qieo_measure_integer_ceiling (the drawn pass's per-gene "
                               "integer work, state in registers, %d blocks, best of %d)" % (
                                   ceiling.grid_ctas, ceiling.reps)}
    roof["frac_hbm_4B_formula"] = hbm_achieved / hbm_peak
    roof["fixed_words"] = bool(shape.fixed_words)
    if shape.fixed_words:
        roof["note"] = ("fixed-vector words: generations in which most vectors are fixed skip their "
                        "draws and state traffic exactly (identical results), so the 4 B and full-draw "
                        "per gene-update formula behind frac can exceed 1; phases.work_adjusted is "
                        "the roofline of the work each generation needed")
    roof["hbm_peak_gbs"] = hbm_peak
    if int_peak:
        roof["int_ceiling_gene_updates_per_s"] = int_peak
        roof["philox_only_gene_updates_per_s"] = ceiling.philox_genes_per_s
        roof["t_hbm_us"] = t_hbm * 1e6
        roof["t_int_us"] = t_int * 1e6
    roof["state_in_l2"] = l2_resident
    kname = ("resident_run_kernel" if shape.resident else "run_kernel" if shape.persistent
             else "generation_kernel")
    roof["traffic"] = None if a.state_i8 else profile_traffic(kname, a.workload)
    roof["traffic_per"] = ("generation (one launch per generation)" if not shape.persistent
                           else "generation (the run's launch divided by its generations)")
    if roof["traffic"]:
        roof["frac_dram_measured"] = roof["traffic"] / launch_s / 1e9 / hbm_peak
    roof["kernel"] = ("resident_run_kernel (one cooperative launch per run, state in shared memory)"
                      if shape.resident else
                      "run_kernel (one cooperative launch per run)" if shape.persistent
                      else "generation_kernel (one launch per generation)")
    roof["us_per_generation"] = launch_s * 1e6
    if not a.no_phases and (shape.resident or not shape.persistent):
        roof["phases"] = generation_phases(Q, prob, c, np_, G, rank, flags, stream, torch,
                                           hbm_peak, int_peak)

    # end to end through the C ABI with host buffers: create (uploads the items), run,
    # read the best record back, destroy -- every step
    e2e_times = []
    with torch.cuda.stream(stream):
        for i in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
            barrier()
            t0 = time.perf_counter()
            h = Q.Instance(prob, np_, seed=c["seed"], inst=c["inst"] + rank,
                           stream=stream.cuda_stream, flags=flags)
            h.run(G)
            bits, bf, bg, bc = h.best()
            h.close()
            torch.cuda.synchronize()
            if i > 0:
                e2e_times.append(time.perf_counter() - t0)
    e2e_value = (world * genes_per_step * len(e2e_times) / max_over_ranks(sum(e2e_times), dist)
                 if e2e_times else None)
    svec = (ng + 7) // 8
    h2d = svec * 8 * 4 * (1 if shape.narrow else 2) + 4 * (2 * 25 + 1)
    d2h = ((svec + 15) // 16) * 16 + 24

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(workload_config(a.workload, a.state_i8),
                       l2="flushed between steps (512 MB write)" if flush
                       else "state larger than L2 (no flush)",
                       parallelism="one independent instance per GPU",
                       launch_shape="%d lanes x %d warps per row tile, %d tiles per row, "
                                    "%d persistent blocks, %s, %s" % (
                           shape.lanes_per_row, shape.warps_per_row, shape.tiles,
                           shape.grid_ctas,
                           # the library queues segments when a block's share is >= 64 rows
                           ("segments of decreasing size (<= %d tile-rows) from a queue"
                            % shape.rows_per_cta) if shape.rows_per_cta >= 64
                           else "equal static shares of <= %d tile-rows" % shape.rows_per_cta,
                           "one cooperative launch per run with the state resident in shared memory"
                           if shape.resident else "one cooperative launch per run" if shape.persistent
                           else "one launch per generation")),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": "qieo_create_instance from host arrays + qieo_run + qieo_get_best + "
                        "qieo_destroy_instance per step"},
        # per step: the reset's init launch, then either one cooperative launch + the
        # end-of-run launch, or G generation launches + the final CIP + the end-of-run launch
        "gpu_launches": a.steps * (1 + (2 if shape.persistent else G + 2)),
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, cores, sample, gens, dt = oracle_sample(a.workload)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    inst.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return np


def generation_phases(Q, prob, c, np_, G, rank, flags, stream, torch, hbm_peak, int_peak):
    """Device time of every generation of one run (QIEO_FLAG_TIME_GENERATIONS: an event
    before each launch, so each time is that launch alone), summarised per window of 25
    generations and for the two phase windows. Run after the timed region."""
    import numpy as np
    ng = c["ng"]
    with torch.cuda.stream(stream):
        inst = Q.Instance(prob, np_, seed=c["seed"], inst=c["inst"] + rank, stream=stream.cuda_stream,
                          flags=flags | Q.QIEO_FLAG_TIME_GENERATIONS)
        inst.run(G)                        # warm-up run
        inst.reset()
        inst.run(G)
        ms = inst.generation_times(G)
        drawn = inst.drawn_vectors(0, G) if inst.shape().fixed_words else None
        inst.close()
    genes = np_ * ng

    def window(lo, hi):
        lo, hi = min(lo, len(ms)), min(hi, len(ms))
        if hi <= lo:
            return None
        us = 1e3 * float(np.mean(ms[lo:hi]))
        rate = genes / (us * 1e-6)
        out = {"generations": "%d-%d" % (lo, hi - 1), "us_per_generation": us,
               "gene_updates_per_s": rate,
               "frac_hbm_4B_formula": STATE_BYTES_PER_GENE * rate / 1e9 / hbm_peak}
        if int_peak:
            out["frac_int_ceiling"] = rate / int_peak
        return out

    step = 25
    out = {"spread": window(*SPREAD_WINDOW), "saturated": window(*SATURATED_WINDOW),
           "per_25": [round(1e3 * float(np.mean(ms[i:i + step])), 2) for i in range(0, len(ms), step)],
           "sum_of_launches_us": 1e3 * float(np.sum(ms)),
           "what": "device clock at each generation's start (resident form) or CUDA events before "
                   "every generation launch of one run (launches serialised)"}
    if drawn is not None and int_peak:
        out["work_adjusted"] = work_adjusted(ms, drawn, np_ * ((ng + 7) // 8), hbm_peak, int_peak)
    return out


# Bytes a vector that did not draw needs in a sparse generation: its fixed-vector bit and its
# previous alleles read, its alleles written.
STABLE_BYTES = 1.0 / 8.0 + 1.0 + 1.0


def work_adjusted(ms, drawn, nvec, hbm_peak, int_peak):
    """The roofline of the work each generation actually needed. A vector that drew (the
    qieo_get_drawn_vectors count) needs its 8 draws at the measured integer ceiling and its
    32 B of state (read and written); one that did not needs its fixed-vector bit and its
    previous alleles read and its alleles written (STABLE_BYTES = 1/8 + 1 + 1 B). Per
    generation the bound is the slower of the two; the fraction is the sum of the bounds
    over the sum of the measured times."""
    import numpy as np
    d = np.asarray(drawn, dtype=np.float64)
    t_int = 8.0 * d / int_peak
    t_hbm = (32.0 * d + STABLE_BYTES * (nvec - d)) / (hbm_peak * 1e9)
    bound = np.maximum(t_int, t_hbm)
    meas = np.asarray(ms, dtype=np.float64) * 1e-3
    return {"frac": float(bound.sum() / meas.sum()),
            "bound_us": 1e6 * float(bound.sum()), "measured_us": 1e6 * float(meas.sum()),
            "drawn_fraction": float(d.sum() / (nvec * len(d))),
            "drawn_per_25": [round(float(d[i:i + 25].mean()) / nvec, 4) for i in range(0, len(d), 25)],
            "frac_per_25": [round(float(bound[i:i + 25].sum() / meas[i:i + 25].sum()), 3)
                            for i in range(0, len(d), 25)],
            "what": "per generation: max(8 draws per vector that drew at the measured integer "
                    "ceiling, (32 B per vector that drew + 2.125 B per one that did not) at the "
                    "measured HBM bandwidth), summed, over the measured generation times"}


def batch_oracle_sample(specs, G: int, target_s: float = 10.0):
    """The oracle (OpenMP build, all host cores) solving manifest instances in order until
    about target_s of CPU work. Returns (solves/s, cores, sample text)."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    O.build()
    O.set_threads(cores)
    done, t0 = 0, time.perf_counter()
    for sp in specs:
        prob = WL.knapsack(sp.ng, sp.seed)
        O.run(prob, sp.np_, G, seed=sp.seed, inst=sp.seed, kind="omp", threads=cores)
        done += 1
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, cores, "first %d manifest instances x %d generations, OpenMP build, %d threads" % (
        done, G, cores)


def member_result(inst):
    """A member's result after a run, for comparing two arms: its best record and alleles,
    its generation counter and a digest of its final angle indices and fitness."""
    import hashlib
    bits, bf, bg, bc = inst.best()
    k, t = inst.state()
    h = hashlib.sha256(k.tobytes())
    h.update(inst.fitness().tobytes())
    return (bf, bg, bc, t, bits.tobytes(), h.hexdigest())


def run_batched(a):
    """c4: 256 independent instances (Ng log-uniform in [50, 20000], Np uniform in
    {32..512}, seeds 1..256), 300 generations each. One step = reset + 300 generations of
    all 256 in one batched launch per generation; compared with one launch sequence per
    instance. Under torchrun every rank solves its own 256 (seeds offset by 256 x rank)."""
    import torch
    from paper_2609_30862_gb300 import qieo as Q
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    Q.load()
    G, n = 300, 256
    specs = WL.batch_manifest(n, first_seed=1 + n * rank)
    probs = [WL.knapsack(sp.ng, sp.seed) for sp in specs]
    stream = torch.cuda.Stream()

    member_flags = Q.QIEO_FLAG_PER_GENERATION if a.per_generation else 0

    def make(tune: bool):
        out, t = [], 0.0
        for sp, prob in zip(specs, probs):
            inst = Q.Instance(prob, sp.np_, seed=sp.seed, inst=sp.seed, stream=stream.cuda_stream,
                              flags=member_flags)
            if tune:
                t0 = time.perf_counter()
                inst.autotune(4)
                t += time.perf_counter() - t0
            out.append(inst)
        return out, t

    insts, tune_s = make(not a.no_autotune)
    genes_per_gen = sum(sp.np_ * sp.ng for sp in specs)
    genes = genes_per_gen * G
    state_bytes = sum(sp.np_ * ((sp.ng + 7) // 8) * 16 for sp in specs)
    flush = state_bytes < 2 * L2_BYTES
    flush_buf = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda") if flush else None
    batch = Q.Batch(insts)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            for i in insts:
                i.reset()
            batch.run(G)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(a.steps)]
        sampler = ClockSampler(gpu_id_for_smi(torch, local)) if rank == 0 else None
        if sampler:
            sampler.start()
        barrier()
        for k in range(a.steps):
            if flush:
                flush_buf.fill_(k & 0xFF)
            evs[k][0].record(stream)
            for i in insts:
                i.reset()
            evs[k][1].record(stream)
            batch.run(G)
            evs[k][2].record(stream)
        barrier()
        clocks = sampler.stop() if sampler else None
        tb = max_over_ranks(sum(e0.elapsed_time(e2) for e0, _, e2 in evs) / 1e3, dist)
        run_s = max_over_ranks(sum(e1.elapsed_time(e2) for _, e1, e2 in evs) / 1e3, dist)

        # one launch sequence per instance, same members and results
        single_steps = max(1, a.steps // 5)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        batched_out = [member_result(i) for i in insts]
        barrier()
        ev[0].record(stream)
        for _ in range(single_steps):
            for i in insts:
                i.reset()
                i.run(G)
        ev[1].record(stream)
        barrier()
        ts = max_over_ranks(ev[0].elapsed_time(ev[1]) / 1e3, dist)
        single_out = [member_result(i) for i in insts]
        same = sum(1 for x, y in zip(batched_out, single_out) if x == y)
        ok = same == len(insts)
    batch.close()
    for i in insts:
        i.close()

    # end to end through the C ABI with host buffers: create the 256 instances (items
    # uploaded), run them as one batch, read every best record back, destroy -- every step
    e2e_times = []
    with torch.cuda.stream(stream):
        for k in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
            barrier()
            t0 = time.perf_counter()
            hs, _ = make(False)
            hb = Q.Batch(hs)
            hb.run(G)
            for h in hs:
                h.best()
            hb.close()
            for h in hs:
                h.close()
            torch.cuda.synchronize()
            if k > 0:
                e2e_times.append(time.perf_counter() - t0)
    e2e_value = (world * n * len(e2e_times) / max_over_ranks(sum(e2e_times), dist)
                 if e2e_times else None)
    h2d = sum(((sp.ng + 7) // 8) * 8 * 4 * 3 + 4 * 51 for sp in specs)
    d2h = sum(((sp.ng + 7) // 8 + 15) // 16 * 16 + 24 for sp in specs)

    # Roofline of the batched kernels: per generation the algorithmic work is every member's
    # genes -- 4 B of state each, read and written, and the drawn pass's integer work --
    # timed as the run / G; the bound is the slower of the two measured ceilings (HBM copy
    # bandwidth, the integer ceiling of the same per-gene arithmetic).
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    launch_s = run_s / (a.steps * G)
    ceiling = Q.qieo_measure_integer_ceiling(5)
    int_peak = ceiling.drawn_genes_per_s
    t_hbm = STATE_BYTES_PER_GENE * genes_per_gen / (hbm_peak * 1e9)
    t_int = genes_per_gen / int_peak
    achieved = STATE_BYTES_PER_GENE * genes_per_gen / launch_s / 1e9
    if t_hbm >= t_int:
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": "%s hbm_gbs" % peak_src}
    else:
        ach = genes_per_gen / launch_s / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": int_peak / 1e9, "unit": "Ggene-updates/s",
                "frac": ach / (int_peak / 1e9),
                "peak_source": "measured: qieo_measure_integer_ceiling (the drawn pass's per-gene "
                               "integer work, state in registers, %d blocks, best of %d)" % (
                                   ceiling.grid_ctas, ceiling.reps)}
    roof.update({"frac_hbm_4B_formula": achieved / hbm_peak, "hbm_peak_gbs": hbm_peak,
                 "int_ceiling_gene_updates_per_s": int_peak, "t_hbm_us": t_hbm * 1e6,
                 "t_int_us": t_int * 1e6,
                 "state_in_l2": state_bytes < L2_BYTES,
                 "traffic": profile_traffic("batch_generation_kernel" if a.per_generation
                                            else "batch_run_kernel", "c4"),
                 "kernel": ("batch_generation_kernel (one launch per generation for all members)"
                            if a.per_generation else
                            "batch_run_kernel (one persistent launch per run for all members)"),
                 "us_per_generation": launch_s * 1e6,
                 "traffic_per": "generation (the persistent launch divided by its generations)"})
    if roof["traffic"]:
        roof["frac_dram_measured"] = roof["traffic"] / launch_s / 1e9 / hbm_peak
    value = world * n * a.steps / tb
    line = {
        "metric": "solves/s (256 instances x 300 generations)", "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tb / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "c4: 256 instances, Ng log-uniform [50, 20000], Np uniform {32,64,128,256,512}, "
                               "300 generations, seeds 1..256",
                   "parallelism": ("one batched launch per generation" if a.per_generation
                                   else "one persistent batched launch per run")
                               + ("; 256 instances per rank" if world > 1 else ""),
                   "state_bytes": state_bytes,
                   "l2": "flushed between steps (512 MB write)" if flush else "state larger than L2 (no flush)"},
        "gene_updates_per_s": world * genes * a.steps / tb,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "256 x qieo_create_instance from host arrays + qieo_create_batch + qieo_batch_run + "
                        "256 x qieo_get_best + destroy, per step"},
        # per step: n resets, then G + 1 batched launches, or the first generation's launch, one
        # persistent launch for the others and the final CIP
        "gpu_launches": a.steps * (n + (G + 1 if a.per_generation else 3)),
        "clocks": clocks,
        "one_launch_per_instance": {"value": world * n * single_steps / ts, "unit": "solves/s",
                                    "gene_updates_per_s": world * genes * single_steps / ts},
        "speedup_vs_one_launch_per_instance": (n * a.steps / tb) / (n * single_steps / ts),
        "autotune_s": tune_s, "records_ok": ok,
        "results_identical": {"checked": n, "equal": same,
                              "what": "per member: best record, best alleles, generation counter and a "
                                      "SHA-256 of the final angle indices and fitness, batched arm vs "
                                      "one launch sequence per instance"},
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, cores, sample = batch_oracle_sample(specs, G)
        line["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_served(a):
    """c5: a Poisson stream of solve requests (sizes as in c4, seeds r+1, 300 generations)
    through the continuous-batching server, against serial per-request launches (one
    instance at a time in arrival order). Reports solves/s and p50/p99 latency."""
    import numpy as np
    import torch
    from paper_2609_30862_gb300 import qieo as Q
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(0)
    Q.load()
    G, n = 300, a.requests
    specs = WL.batch_manifest(n, first_seed=1)
    probs = [WL.knapsack(sp.ng, sp.seed) for sp in specs]
    rate = a.rate
    if rate <= 0:   # capacity of the batched form on a 256-request sample
        insts = [Q.Instance(probs[i], specs[i].np_, seed=specs[i].seed, inst=specs[i].seed)
                 for i in range(min(256, n))]
        b = Q.Batch(insts)
        b.run(G)
        torch.cuda.synchronize()
        for i in insts:
            i.reset()
        t0 = time.perf_counter()
        b.run(G)
        for i in insts:
            i.synchronize()
        cap = len(insts) / (time.perf_counter() - t0)
        b.close()
        for i in insts:
            i.close()
        rate = 0.8 * cap
    arrivals = WL.poisson_arrivals(n, rate)

    def latency_stats(lat, span):
        lat = np.asarray(lat)
        return {"solves_per_s": len(lat) / span, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean())}

    # continuous batching
    srv = Q.Server(gens_per_step=25)
    ids = []
    sampler = ClockSampler(gpu_id_for_smi(torch, 0))
    sampler.start()
    t_start = time.perf_counter()
    for i, sp in enumerate(specs):
        delay = arrivals[i] - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(probs[i], sp.np_, G, seed=sp.seed, inst=sp.seed))
    polled = [srv.poll(rid, wait_ms=600000) for rid in ids]
    results = [r for r, _ in polled]
    clocks = sampler.stop()
    assert all(r.state == Q.QIEO_SOLVE_DONE for r in results)
    lat = [r.done_s - r.submit_s for r in results]
    span = max(r.done_s for r in results) - min(r.submit_s for r in results)
    served = latency_stats(lat, span)
    stats = srv.stats()
    srv.close()

    # serial per-request launches: one instance at a time, in arrival order
    m = min(n, max(200, n // 10))
    lat_s, solo = [], []
    t_start = time.perf_counter()
    for i in range(m):
        now = time.perf_counter() - t_start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        with Q.Instance(probs[i], specs[i].np_, seed=specs[i].seed, inst=specs[i].seed) as inst:
            inst.run(G)
            solo.append(inst.best())
        lat_s.append(time.perf_counter() - t_start - arrivals[i])
    serial = latency_stats(lat_s, time.perf_counter() - t_start)
    # identical results: every request the serial arm ran, served vs alone
    same = sum(1 for i in range(m)
               if (results[i].fitness, results[i].generation, results[i].chromosome) == tuple(solo[i][1:])
               and np.array_equal(polled[i][1], solo[i][0]))

    genes = sum(sp.np_ * sp.ng for sp in specs) * G
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    achieved = STATE_BYTES_PER_GENE * genes / span / 1e9
    h2d = sum(((sp.ng + 7) // 8) * 8 * 4 * 3 + 4 * 51 + 8 * sp.ng for sp in specs) // n
    d2h = sum(sp.ng + 64 for sp in specs) // n
    line = {
        "metric": "served solves/s and p50/p99 latency (Poisson arrivals, 300 generations)",
        "value": served["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "c5: %d requests, sizes as c4, Poisson arrivals at %.1f/s" % (n, rate),
                   "parallelism": "continuous batching, 25 generations per step",
                   "l2": "arrival-driven: no flush (the resident set changes every step)"},
        "served": served,
        "serial_per_request": dict(serial, requests=m),
        "results_identical": {"checked": m, "equal": same,
                              "what": "best record and alleles of each request the serial arm ran, "
                                      "served (in the mix) vs solved alone"},
        "records_ok": same == m,
        "arrival_rate_per_s": rate,
        # the whole stream goes through the public API (submit from host arrays, poll the
        # result back), so value is itself end to end; the bytes are per request
        "e2e": {"value": served["solves_per_s"], "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "what": "qieo_server_submit (host arrays) ... qieo_server_poll (best record and "
                        "alleles), wall clock over the stream; bytes are per request"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": "%s hbm_gbs" % peak_src,
                     "traffic": None, "kernel": "batch_generation_kernel (server steps)",
                     "note": "4 B per served gene-update over the stream's span, idle gaps between "
                             "arrivals included"},
        "gpu_launches": stats["kernel_launches"],
        "server_stats": stats,
        "clocks": clocks,
    }
    if not a.no_cpu_baseline:
        rate_cpu, cores, sample = batch_oracle_sample(specs, G)
        line["cpu_baseline"] = {"value": rate_cpu, "unit": "solves/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line), flush=True)


def run_phases(a):
    """Per-step time breakdown of a generation (the paper's Table VI analysis on this GPU):
    the unfused form runs CIP, QIP, Evaluation and DetermineElite as four timed launches;
    the fused kernel and the host-DetermineElite variant run the same solve for comparison.
    All three produce identical results."""
    import torch
    from paper_2609_30862_gb300 import qieo as Q
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(0)
    Q.load()
    c = WL.WORKLOADS[a.workload]
    prob = WL.knapsack(c["ng"], c["item_seed"])
    np_, G = c["np"], c["gens"]
    stream = torch.cuda.Stream()

    def timed_run(inst, reps):
        best = None
        with torch.cuda.stream(stream):
            for r in range(reps + 1):
                inst.reset()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                inst.run(G)
                e1.record(stream)
                e1.synchronize()
                if r:
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
        return 1e3 * best / G, inst.best()

    mk = lambda **kw: Q.Instance(prob, np_, seed=c["seed"], inst=c["inst"], stream=stream.cuda_stream, **kw)
    with mk() as I:
        fused_us, fused_best = timed_run(I, max(1, a.steps))
    with mk(flags=Q.QIEO_FLAG_UNFUSED) as I:
        unfused_us, unfused_best = timed_run(I, max(1, a.steps))
    with mk(flags=Q.QIEO_FLAG_UNFUSED | Q.QIEO_FLAG_TIME_KERNELS) as I:
        with torch.cuda.stream(stream):
            I.run(G)
            I.synchronize()
        ms, gens = I.phase_times()
    with mk(elite_on_host=1) as I:
        host_us, host_best = timed_run(I, 1)
    with mk(elite_on_host=1, flags=Q.QIEO_FLAG_TIME_KERNELS) as I:
        with torch.cuda.stream(stream):
            I.run(G)
            I.synchronize()
        hms, hgens = I.phase_times()
    per = {k: 1e3 * v / gens for k, v in ms.items()}
    tot = sum(per.values())
    assert fused_best[1:] == unfused_best[1:] == host_best[1:]
    line = {
        "metric": "time per generation by step (CIP, QIP, Evaluation, DetermineElite)",
        "value": fused_us, "unit": "us/generation", "n_gpus": 1, "steps": max(1, a.steps),
        "warmup": 1, "higher_is_better": False, "dtype": "u32", "data": "synthetic",
        "config": workload_config(a.workload),
        "fused_us_per_generation": fused_us,
        "unfused_us_per_generation": unfused_us,
        "fusion_speedup": unfused_us / fused_us,
        "unfused_step_us_per_generation": per,
        "unfused_step_fraction": {k: v / tot for k, v in per.items()},
        "determine_elite": {
            "device_us_per_generation": per["determine_elite"],
            "host_us_per_generation": 1e3 * hms["determine_elite"] / hgens,
            "host_over_device": (hms["determine_elite"] / hgens) / (ms["determine_elite"] / gens),
            "host_variant_run_us_per_generation": host_us,
            "what_host": "copy of fitness[np] to the host + host argmax + the launch recording the "
                         "elite, after the generation kernel finished",
        },
        "gpu_launches": max(1, a.steps) * (G + 2),
    }
    print(json.dumps(line), flush=True)


SWEEP_NP = [32 << i for i in range(14)]                     # 32 .. 262,144
SWEEP_NG = [500, 1000, 2500, 5000, 10000, 25000, 50000, 100000, 200000]


def run_sweep(a):
    """Time per generation over the paper's (Np, Ng) grid (Np = 32 .. 262,144 in powers of
    two, Ng = 500 .. 200,000 in 1-2.5-5 steps), rules R1 and R2, for every pair whose
    instance fits --sweep-max-gb of device memory. Each pair is timed over its first
    generations from the start state (the population still spread: the costly phase), at
    least 3 generations and about 2e9 gene-updates."""
    import torch
    from paper_2609_30862_gb300 import qieo as Q
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(0)
    Q.load()
    stream = torch.cuda.Stream()
    peaks, peak_src = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    rows = []
    t_start = time.perf_counter()
    for rule in (0, 1):
        for np_ in SWEEP_NP:
            for ng in SWEEP_NG:
                svec = (ng + 7) // 8
                need = np_ * svec * 16 + 2 * np_ * ((svec + 15) // 16 * 16) + 64 * svec + 64 * np_
                if need > a.sweep_max_gb * 1e9:
                    continue
                if rule == 1 and (np_ * ng > 1 << 30):
                    continue        # R2 on the smaller half of the grid only
                G = int(max(3, min(200, round(2e9 / (np_ * ng)))))
                prob = WL.knapsack(ng, 1)
                with Q.Instance(prob, np_, seed=1, rule=rule, stream=stream.cuda_stream) as inst:
                    with torch.cuda.stream(stream):
                        inst.run(G)
                        inst.reset()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        inst.run(G)
                        e1.record(stream)
                        e1.synchronize()
                    us = 1e3 * e0.elapsed_time(e1) / G
                    rows.append({"np": np_, "ng": ng, "rule": "R2" if rule else "R1", "gens": G,
                                 "us_per_gen": round(us, 3),
                                 "gene_updates_per_s": np_ * ng / (us * 1e-6),
                                 "hbm_frac": STATE_BYTES_PER_GENE * np_ * ng / (us * 1e-6) / 1e9 / hbm,
                                 "state_gb": round(np_ * svec * 16 / 1e9, 3)})
                torch.cuda.empty_cache()
    best = max(rows, key=lambda r: r["gene_updates_per_s"])
    line = {
        "metric": "time per generation over the (Np, Ng) grid", "value": best["gene_updates_per_s"],
        "unit": "gene-updates/s (best pair)", "n_gpus": 1, "higher_is_better": True,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "Np in 32..262144 (x2), Ng in %s, item seed 1, first generations "
                               "from the start state" % SWEEP_NG, "max_gb": a.sweep_max_gb},
        "peak_hbm_gbs": hbm, "peak_source": peak_src, "pairs": rows,
        "wall_s": time.perf_counter() - t_start,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.oracle_scan:
        return run_oracle_scan(a)
    if a.impl != "reference" and a.sweep:
        run_sweep(a)
        return
    if a.impl != "reference" and a.phases:
        run_phases(a)
        return
    if a.impl != "reference" and a.workload == "c5":
        run_served(a)
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "c4":
        run_batched(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
