#!/usr/bin/env python
"""Benchmark of the voxel soft-robot co-design hot path on GB300.

One bench step = one full co-design generation of the MLP-encoded population: positional
encoding + MLP spatial query of 1024 genomes on an 8x8x8 grid, largest component, topology,
10,000 time steps of every robot, FP64 fitness, then elite selection / crossover / mutation of
the 1024 x 20,998 weight matrix, all on the GPU.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload on the host
cores.  Under torchrun (N > 1) every rank runs its own population shard (weak scaling, no
collective on the data path); time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2405_00698_gb300 import workloads as W  # noqa: E402

METRIC = "spring-updates/s"
WORKLOAD = dict(workload="mlp-encoded population: 1024 genomes, 8x8x8 grid, 10,000 steps per "
                "generation, 1 generation per step", robots=1024, grid=[8, 8, 8], sim_steps=10000,
                genome=W.GENOME_LEN)
P_ROBOTS, GRID, SIM_STEPS = 1024, (8, 8, 8), 10000
SMEM_PEAK_NOTE = "152 SMs x 128 B/clk x 2.07 GHz (unit counts and maximum SM clock)"
SMEM_PEAK_GBS = 152 * 128 * 2.07


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--robots", type=int, default=P_ROBOTS, help=argparse.SUPPRESS)
    ap.add_argument("--sim-steps", type=int, default=SIM_STEPS, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing (barrier and max-over-ranks only)
# ------------------------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def dist_max(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), max=float(parts[2]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# the GPU arm
# ------------------------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    from paper_2405_00698_gb300 import build as B
    from paper_2405_00698_gb300 import voxsim as vs
    if rank == 0 or world == 1:
        B.build()
    dist_barrier(world)
    P, N = args.robots, args.sim_steps
    phys = W.CONFIG
    evo = W.Evolution()
    genomes_h, Bmat_h = W.workload_mlp(P, seed=1 + 1000 * rank)
    dims = np.tile(np.asarray(GRID, np.int32), (P, 1))
    stream = torch.cuda.current_stream()
    sim = vs.Simulator(phys, device=local, stream=stream)
    g_a = torch.from_numpy(genomes_h).cuda()
    g_b = torch.empty_like(g_a)
    Bmat = torch.from_numpy(Bmat_h).cuda()
    fit = torch.empty(P, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    state = {"gen": 0, "g_in": g_a, "g_out": g_b}

    def generation():
        sim.set_population(dims, state["g_in"], vs.MODE_MLP, B=Bmat)
        sim.step(N)
        sim.fitness(fit)
        sim.evo_generation(fit, state["g_in"], state["g_out"], evo, state["gen"])
        state["gen"] += 1
        state["g_in"], state["g_out"] = state["g_out"], state["g_in"]

    for _ in range(args.warmup):
        generation()
    torch.cuda.synchronize()
    sim.timing()
    # timed region: device-resident inputs, L2 flushed between steps (outside the events)
    clocks = ClockSampler(local)
    clocks.start()
    dist_barrier(world)
    torch.cuda.synchronize()
    total_ms, updates, kernel_ms, launches, masses = 0.0, 0, 0.0, 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g_in_this = state["g_in"]
        generation()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        # spring count of the population this step simulated (read after the timed span)
        k_ms, n_launch = sim.timing()
        kernel_ms += k_ms
        launches += n_launch
        M, S = sim.counts()
        updates += int(S.astype(np.int64).sum()) * N
        masses += int(M.astype(np.int64).sum()) * N
        del g_in_this
    torch.cuda.synchronize()
    dist_barrier(world)
    clk = clocks.stop()
    total_ms = dist_max(total_ms, world, "cuda")
    updates_all = int(dist_max(float(updates), world, "cuda")) * world if world > 1 else updates

    # end to end through the public API: pinned host genomes in, fitness out, every step
    pinned = torch.from_numpy(genomes_h).pin_memory()
    fit_h = torch.empty(P, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_updates = 0.0, 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        state["g_in"].copy_(pinned, non_blocking=True)
        generation()
        fit_h.copy_(fit, non_blocking=True)
        stream.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        M, S = sim.counts()
        e2e_updates += int(S.astype(np.int64).sum()) * N
        sim.timing()
    e2e_ms = dist_max(e2e_ms, world, "cuda")

    peaks, peak_src = measured_peaks()
    # dominant kernel: the resident step kernel; algorithmic shared-memory bytes per step
    # 48 B per spring update (two position reads, two atomic force updates) + 36 B per mass
    alg_bytes = 48.0 * updates + 36.0 * masses
    achieved_gbs = alg_bytes / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else 0.0
    rec = {
        "metric": METRIC,
        "value": updates_all / (total_ms * 1e-3),
        "unit": "spring-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded MLP genomes, U(-1/sqrt(fan_in), 1/sqrt(fan_in)); B ~ N(0, 2^2))",
        "config": dict(WORKLOAD, l2="flushed between timed steps (256 MB write)",
                       parallelism=f"population shards x{world}" if world > 1 else "single GPU"),
        "e2e": {"value": e2e_updates * world / (e2e_ms * 1e-3), "unit": "spring-updates/s",
                "h2d_bytes_per_step": int(genomes_h.nbytes),
                "d2h_bytes_per_step": int(P * 8)},
        "gpu_launches": launches,
        "roofline": {"bound": "smem", "kernel": "k_step_resident_atomic",
                     "achieved": achieved_gbs, "peak": SMEM_PEAK_GBS, "unit": "GB/s",
                     "frac": achieved_gbs / SMEM_PEAK_GBS, "traffic": None,
                     "peak_source": SMEM_PEAK_NOTE,
                     "kernel_ms_per_step": kernel_ms / args.steps},
        "clocks": clk,
        "peaks_source": peak_src,
    }
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(genomes_h, Bmat_h, N, budget_s=12.0)
    if rank == 0:
        print(json.dumps(rec))
    sim.close()


# ------------------------------------------------------------------------------------------
# the CPU oracle (baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_generation(genomes, Bmat, N, nthreads=0):
    """The oracle's pass over a sample: MLP decode, simulation, fitness, one evolution
    generation.  Returns (spring updates, threads used)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    P = genomes.shape[0]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        dec = list(ex.map(lambda g: O.mlp_query(GRID, Bmat, g), genomes))
    mats = [d[0].reshape(GRID[::-1]) for d in dec]
    w = np.concatenate([d[1] for d in dec])
    pop = W.make_population([GRID] * P, mats)
    kappa = np.asarray(W.CONFIG.k_mat)[pop.mats]
    phi = np.asarray(W.CONFIG.phase_mat)[pop.mats]
    res = O.run_population(pop, W.CONFIG, N, w=w, kappa=kappa, phi=phi, nthreads=nthreads)
    evo = W.Evolution()
    O.evo_generation(res["fitness"], genomes, evo.elites(P), evo.seed, 0, evo.mut_threshold(), evo.sigma)
    return int(res["S"].astype(np.int64).sum()) * N, int(res["threads"])


def cpu_baseline(genomes, Bmat, N, budget_s=12.0):
    n = 16
    t0 = time.perf_counter()
    upd, th = oracle_generation(genomes[:n], Bmat, N)
    dt = time.perf_counter() - t0
    return {"value": upd / dt, "unit": "spring-updates/s", "cores": th, "kind": "oracle",
            "sample": f"{n} of the 1024 genomes, full {N}-step generation (decode, simulate, "
                      f"fitness, evolve), OpenMP over robots; {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    N = args.sim_steps
    genomes, Bmat = W.workload_mlp(args.robots, seed=1)
    n = 16
    for _ in range(args.warmup and 1):
        oracle_generation(genomes[:4], Bmat, 100)
    tot_t, tot_u, th = 0.0, 0, 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        u, th = oracle_generation(genomes[n * k:n * (k + 1)], Bmat, N)
        tot_t += time.perf_counter() - t0
        tot_u += u
    v = tot_u / tot_t
    sample = f"{n} genomes per step (different each step) of the 1024, full {N}-step generation"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "spring-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": WORKLOAD,
        "cpu_baseline": {"value": v, "unit": "spring-updates/s", "cores": th, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "spring-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
