#!/usr/bin/env python
"""Benchmark of the voxel soft-robot co-design hot path on GB300.

One bench step = the MLP-encoded population's whole run: 10 co-design generations from the
seeded population, each one positional encoding + MLP spatial query of 1024 genomes on an 8x8x8
grid, largest component, topology, 10,000 time steps of every robot, FP64 fitness, then elite
selection / crossover / mutation of the 1024 x 20,998 weight matrix, all on the GPU.  Every step
starts from the same seeded genomes, so the timed work does not depend on --steps or --warmup.
Prints one JSON line (rank 0).

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
WORKLOAD = dict(workload="mlp-encoded population: 1024 genomes, 8x8x8 grid, 10 generations of "
                "10,000 steps from the seeded population per step", robots=1024, grid=[8, 8, 8],
                sim_steps=10000, genome=W.GENOME_LEN)
P_ROBOTS, GRID, SIM_STEPS, GENERATIONS = 1024, (8, 8, 8), 10000, 10
SMEM_PEAK_NOTE = "152 SMs x 128 B/clk x 2.07 GHz (unit counts and maximum SM clock)"
SMEM_PEAK_GBS = 152 * 128 * 2.07
SMEM_PEAK_MEASURED_NOTE = ("measured: sim_measure_smem_bandwidth, two 1024-thread blocks per SM streaming "
                           "conflict-free 16-byte shared loads for 5 ms, best of 3 (peak_nominal: "
                           + SMEM_PEAK_NOTE + ")")
# DRAM bytes of one k_step_lattice launch per robot (ncu dram__bytes_read.sum + write of the
# 152-robot, 1000-step capture in profiles/k_step_lattice__mlp152_8cube_1000steps.md): the state
# stays in shared memory, so traffic grows with the robots, not with the steps.
# DRAM bytes of one generation's k_step_lattice_seg launch of the default workload (ncu: 1.29 GB
# read + 198.1 MB written for 1024 robots, 10 segments of 1000 steps), per robot: every
# (segment, robot) unit reloads its robot's parameters and state
LATTICE_DRAM_BYTES_PER_ROBOT = (1.29e9 + 198.1e6) / 1024
LATTICE_TRAFFIC_NOTE = ("ncu dram bytes (read + write) of the generation-0 k_step_lattice_seg launch of this "
                        "workload (1024 robots, 10,000 steps as 10 segments), scaled by robots; the "
                        "one-launch figure the roofline's kernel is timed against, default workload only")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--robots", type=int, default=P_ROBOTS, help=argparse.SUPPRESS)
    ap.add_argument("--sim-steps", type=int, default=SIM_STEPS, help=argparse.SUPPRESS)
    ap.add_argument("--generations", type=int, default=GENERATIONS, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattice", choices=["auto", "corner", "compact", "packed"], default="auto",
                    help="variant of the lattice-gather kernel")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uneven-population, adjoint and large-robot measurements")
    ap.add_argument("--no-autotune", action="store_true",
                    help="uneven population: keep the default per-class routing (reproducible under a profiler)")
    ap.add_argument("--case", choices=["streamed", "streamed_adjoint", "paper_preset", "adjoint", "uneven"], default=None,
                    help="run one extra measurement alone (for profiling; --robots sets its robots)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing: barrier and the max / sum over ranks (paper_2405_00698_gb300.shards)
# ------------------------------------------------------------------------------------------

from paper_2405_00698_gb300 import shards  # noqa: E402


def dist_env():
    return shards.env()


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def dist_max(x: float, world: int, device=None) -> float:
    return shards.max_over_ranks(x, device) if world > 1 else x


def dist_barrier(world):
    if world > 1:
        shards.barrier()


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

def measured_smem_peak(sim):
    """Shared-memory bandwidth of this GPU from the library's probe (best of three runs of about
    5 ms each), else the nominal figure from unit counts and the maximum clock."""
    try:
        return max(sim.measure_smem_bandwidth() for _ in range(3)), SMEM_PEAK_MEASURED_NOTE
    except Exception as exc:                    # noqa: BLE001 - reported in the line
        return SMEM_PEAK_GBS, f"{SMEM_PEAK_NOTE} (probe failed: {exc})"


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
    P, N, NG = args.robots, args.sim_steps, args.generations
    phys = W.CONFIG
    evo = W.Evolution()
    # one population of P robots per rank, sharded: every rank holds the whole genome matrix
    # (replicated evolution) and simulates rows [first, first + P)
    P_all, first = P * world, P * rank
    genomes_h, Bmat_h = W.workload_mlp(P_all, seed=1)
    dims = np.tile(np.asarray(GRID, np.int32), (P, 1))
    stream = torch.cuda.current_stream()
    lattice = {"auto": vs.LATTICE_AUTO, "corner": vs.LATTICE_CORNER, "compact": vs.LATTICE_COMPACT,
               "packed": vs.LATTICE_PACKED}[args.lattice]
    sim = vs.Simulator(phys, device=local, stream=stream, lattice=lattice)
    seed_d = torch.from_numpy(genomes_h).cuda()          # the seeded population, device-resident
    g_a = torch.empty_like(seed_d)
    g_b = torch.empty_like(seed_d)
    Bmat = torch.from_numpy(Bmat_h).cuda()
    fit = torch.empty(P, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def run_config(stats=None):
        """The whole workload once: NG generations (decode, 10,000 steps, fitness, evolution)
        from the seeded population, so every step does identical work whatever --steps and
        --warmup are.  stats (untimed only) collects per-generation spring and mass counts."""
        g_in, g_out = g_a, g_b
        g_in.copy_(seed_d)
        for gen in range(NG):
            sim.set_population(dims, g_in[first:first + P], vs.MODE_MLP, B=Bmat)
            sim.step(N)
            sim.fitness(fit)
            fit_all = shards.gather_population_fitness(fit, world)     # the exchange step
            sim.evo_generation(fit_all, g_in, g_out, evo, gen)
            if stats is not None:
                M, S = sim.counts()
                stats.append((int(S.astype(np.int64).sum()), int(M.astype(np.int64).sum())))
            g_in, g_out = g_out, g_in
        return g_in

    # warm-up; the first pass also counts the springs and masses of every generation (the
    # evolution is deterministic, so every later pass simulates the same populations)
    stats = []
    final_ref = run_config(stats).clone()
    for _ in range(max(args.warmup - 1, 0)):
        run_config()
    torch.cuda.synchronize()
    sim.timing()
    springs_per_step = sum(sp for sp, _ in stats) * N
    masses_per_step = sum(ms for _, ms in stats) * N
    # timed region: device-resident inputs, L2 flushed between steps (outside the events)
    clocks = ClockSampler(local)
    clocks.start()
    dist_barrier(world)
    torch.cuda.synchronize()
    total_ms, kernel_ms, launches = 0.0, 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        final = run_config()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        k_ms, n_launch = sim.timing()
        kernel_ms += k_ms
        launches += n_launch
    torch.cuda.synchronize()
    dist_barrier(world)
    clk = clocks.stop()
    # the timed passes evolved exactly the warm-up's populations
    assert torch.equal(final, final_ref), "the timed workload differs from the warm-up's"
    updates, masses = springs_per_step * args.steps, masses_per_step * args.steps
    value, updates_all, secs = shards.job_throughput(float(updates), total_ms * 1e-3, "cuda")
    # the paper's unit is ambiguous (springs, masses or both per step): springs + masses too
    sm_value, _, _ = shards.job_throughput(float(updates + masses), total_ms * 1e-3, "cuda")
    total_ms = secs * 1e3

    # end to end through the C ABI with host buffers: each step the seeded genomes (and B) go in
    # through sim_set_population from pinned host memory (the library's copy is also the first
    # generation's evolution input, genomes_in NULL) and every generation's fitness comes back
    # through sim_fitness into pinned host memory
    pinned = torch.from_numpy(genomes_h).pin_memory()
    pinned_B = torch.from_numpy(Bmat_h).pin_memory()
    fit_h = torch.empty(P, dtype=torch.float64).pin_memory()

    def run_config_e2e():
        g_in, g_out = None, g_a
        if world > 1:        # the replicated evolution needs every rank's copy of all genomes
            g_b.copy_(pinned, non_blocking=True)
            g_in, g_out = g_b, g_a
        for gen in range(NG):
            if gen == 0 and world == 1:
                sim.set_population(dims, pinned, vs.MODE_MLP, B=pinned_B)
            else:
                sim.set_population(dims, g_in[first:first + P], vs.MODE_MLP, B=Bmat)
            sim.step(N)
            sim.fitness(fit)                      # device: the evolution's input
            sim.fitness(fit_h)                    # host: the caller's read of the result
            fit_all = shards.gather_population_fitness(fit, world)
            sim.evo_generation(fit_all, g_in, g_out, evo, gen)
            g_in, g_out = g_out, (g_b if g_out is g_a else g_a)
        return g_in

    run_config_e2e()                              # warm-up of the host-buffer path
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        final = run_config_e2e()
        stream.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        sim.timing()
    assert torch.equal(final, final_ref), "the end-to-end pass evolved other populations"
    del final_ref
    e2e_value, _, _ = shards.job_throughput(float(springs_per_step * args.steps), e2e_ms * 1e-3, "cuda")

    peaks, peak_src = measured_peaks()
    smem_peak, smem_src = measured_smem_peak(sim)
    peaks["smem_gbs"] = smem_peak
    # dominant kernel: the resident step kernel; algorithmic shared-memory bytes per step
    # 48 B per spring update (the far end's position read, the force-plane write and its read by
    # the far end) + 36 B per mass
    alg_bytes = 48.0 * updates + 36.0 * masses
    achieved_gbs = alg_bytes / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else 0.0
    rec = {
        "metric": METRIC,
        "value": value,
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
        "config": dict(WORKLOAD, generations=NG, l2="flushed between timed steps (256 MB write)",
                       parallelism=(f"one population of {P_all} robots in {world} shards: fitness "
                                    "all-gather per generation, replicated evolution")
                       if world > 1 else "single GPU"),
        "e2e": {"value": e2e_value, "unit": "spring-updates/s",
                "h2d_bytes_per_step": int(genomes_h.nbytes + (Bmat_h.nbytes if world == 1 else 0)),
                "d2h_bytes_per_step": int(P * 8 * NG),
                "path": "C ABI host buffers: sim_set_population(SIM_MEM_HOST) of the seeded genomes, "
                        "sim_fitness(SIM_MEM_HOST) every generation"},
        "springs_per_generation": [sp for sp, _ in stats],
        "gpu_launches": launches,
        "spring_plus_mass_updates_per_s": sm_value,
        "roofline": {"bound": "smem",
                     "kernel": "k_step_lattice_seg (the per-corner step from a queue of 1000-step segments; "
                               "k_step_lattice_packed_seg, the mass-packed groups from the same kind of queue, "
                               "once the robots fill less than 55 % of their slots: generations 8 and 9)",
                     "achieved": achieved_gbs, "peak": smem_peak, "unit": "GB/s",
                     "frac": achieved_gbs / smem_peak, "traffic": (LATTICE_DRAM_BYTES_PER_ROBOT * P if (P, N) == (P_ROBOTS, SIM_STEPS) else None),
                     "traffic_source": LATTICE_TRAFFIC_NOTE,
                     "peak_source": smem_src, "peak_nominal": SMEM_PEAK_GBS,
                     "kernel_ms_per_step": kernel_ms / args.steps},
        "clocks": clk,
        "peaks_source": peak_src,
    }
    if rank == 0 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(genomes_h, Bmat_h, N, budget_s=12.0)
    if not args.no_extras and world == 1:
        sim.close()
        rec["batched_vs_plain"] = measure_uneven(vs, stream, args, peaks)
        rec["adjoint"] = measure_adjoint(vs, stream, args)
        rec["adjoint_records"] = measure_adjoint(vs, stream, args, records=True)
        rec["lamarckian"] = measure_lamarckian(vs, stream, args)
        rec["streamed"] = measure_streamed(vs, stream, args, peaks)
        rec["streamed_adjoint"] = measure_streamed_adjoint(vs, stream, args, peaks)
        rec["streamed_adjoint_records"] = measure_streamed_adjoint(vs, stream, args, peaks, P=16, N=2000,
                                                                   records=True)
        rec["paper_preset"] = measure_paper_preset(vs, stream, args)
    if rank == 0:
        print(json.dumps(rec))
    sim.close()


# ------------------------------------------------------------------------------------------
# the other components of the metric: batched vs plain, adjoint, large robots
# ------------------------------------------------------------------------------------------

def _timed(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def measure_uneven(vs, stream, args, peaks, P=4096, N=5000, plain_robots=64, plain_steps=100):
    """4096 robots, axes from {4,...,12}, occupancy U[0.3, 0.9]: the persistent batched launch
    for 5000 steps, against the plain form (one launch per robot per pass) on a stratified
    sample of 64 robots for 100 steps (a rate: spring updates per second)."""
    pop = W.workload_uneven(P, seed=2)
    sim = vs.Simulator(W.CONFIG, stream=stream)
    sim.set_population_from(pop)
    M, S = sim.counts()
    t0 = time.perf_counter()
    if getattr(args, "no_autotune", False):     # the default routing of every size class
        kinds, threads = np.full(10, -1), np.zeros(10, np.int64)
    else:
        kinds, threads = sim.autotune(20)       # per-size-class kernel choice, state restored
    tune_s = time.perf_counter() - t0
    sim.step(50)                                # warm-up
    sim.timing()
    ms = _timed(stream, lambda: sim.step(N))
    kms, launches = sim.timing()
    batched = float(S.astype(np.int64).sum()) * N / (ms * 1e-3)
    # algorithmic shared-memory bytes of the resident kernels (48 B per spring update, 36 B per
    # mass update) against the shared-memory peak
    batched_gbs = (48.0 * S.astype(np.int64).sum() + 36.0 * M.astype(np.int64).sum()) * N / (ms * 1e-3) / 1e9
    if "smem_gbs" in peaks:
        smem_peak, smem_src = peaks["smem_gbs"], SMEM_PEAK_MEASURED_NOTE
    else:
        smem_peak, smem_src = measured_smem_peak(sim)
    sim.close()
    sub = pop.subset(W.stratified_subset(S, plain_robots))
    cpu = None
    if not getattr(args, "no_cpu_baseline", False):
        cpu = cpu_baseline_population(pop.subset(range(plain_robots)), 500,
                                      f"the first {plain_robots} of the {P} robots, 500 steps")
    res = {}
    for name, path in (("plain", vs.PATH_PLAIN), ("batched_same_sample", vs.PATH_AUTO)):
        s2 = vs.Simulator(W.CONFIG, stream=stream, path=path)
        s2.set_population_from(sub)
        M2, S2 = s2.counts()
        s2.step(5)
        ms2 = _timed(stream, lambda: s2.step(plain_steps))
        res[name] = float(S2.astype(np.int64).sum()) * plain_steps / (ms2 * 1e-3)
        if path == vs.PATH_PLAIN:
            # device-memory bytes of the plain passes: per spring its endpoints, parameters,
            # corner ids and positions (64 B) and six float atomics (48 B); per mass its corner
            # id, u, v and force read, force cleared, u and v written (92 B)
            res["plain_gbs"] = (112.0 * S2.astype(np.int64).sum() + 92.0 * M2.astype(np.int64).sum()) \
                * plain_steps / (ms2 * 1e-3) / 1e9
        s2.close()
    return {"workload": f"{P} robots, axes from {{4,6,8,10,12}}, occupancy U[0.3,0.9], connected, "
                        f"{N} steps", "unit": "spring-updates/s", "batched": batched,
            "batched_ms": ms, "batched_launches": launches, "springs": int(S.sum()),
            "batched_roofline": {"bound": "smem", "achieved": batched_gbs, "peak": smem_peak, "unit": "GB/s",
                                 "frac": batched_gbs / smem_peak, "peak_source": smem_src},
            "autotune": {"skipped": "default routing of every size class"} if getattr(args, "no_autotune", False) else
                        {"classes_max_corners": [64, 128, 192, 256, 384, 768, 1536, 2560, 5120, "more"],
                         "kind (0 lattice per corner, 1 atomic, 2 streamed, 3 lattice compacted, 4 lattice cluster, "
                         "5 lattice in mass-sized groups)": kinds.tolist(),
                         "atomic_threads": threads.tolist(), "seconds": tune_s},
            "plain": res["plain"], "batched_on_plain_sample": res["batched_same_sample"],
            "plain_roofline": {"bound": "hbm", "achieved": res["plain_gbs"], "peak": peaks["hbm_gbs"],
                               "unit": "GB/s", "frac": res["plain_gbs"] / peaks["hbm_gbs"],
                               "note": "launch bound: two launches per robot and step"},
            "plain_sample": f"{plain_robots} robots stratified by spring count, {plain_steps} steps",
            "speedup_vs_plain": batched / res["plain"],
            **({"cpu_baseline": cpu} if cpu else {})}


def measure_adjoint(vs, stream, args, P=512, N=2000, K=100, records=False):
    """512 robots 8x8x8, per-voxel (w, kappa, phi), 2000 steps with checkpoints every 100:
    forward with recording plus the reverse sweep, as gradient evaluations per second.
    records: the forward also keeps every step's record (24 B per corner per step, 17.9 GB
    here) and the backward sweeps them without replaying the segments."""
    import torch
    rng = np.random.default_rng(3)
    pop = W.population_uniform(P, (8, 8, 8), seed=3)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim = vs.Simulator(W.CONFIG, stream=stream)
    sim.set_checkpointing(K)
    sim.set_trajectory_records(records)
    args_pop = (t(pop.mats), t(w), t(kappa), t(phi))
    n = pop.mats.size
    gw = torch.empty(n, device="cuda"); gk = torch.empty_like(gw); gp = torch.empty_like(gw)
    dl = torch.ones(P, dtype=torch.float64, device="cuda")

    def run():
        sim.set_population(pop.dims, args_pop, vs.MODE_PARAMS)
        sim.step(N)
        sim.backward(dl, gw, gk, gp)
    run()                                          # warm-up
    fwd = _timed(stream, lambda: (sim.set_population(pop.dims, args_pop, vs.MODE_PARAMS), sim.step(N)))
    bwd = _timed(stream, lambda: sim.backward(dl, gw, gk, gp))
    _, S = sim.counts()
    sim.close()
    kept = ", every step's record kept" if records else ""
    return {"workload": f"{P} robots 8x8x8, {N} steps, checkpoints every {K}{kept}",
            "grads_per_s": P / ((fwd + bwd) * 1e-3),
            "unit": "robot gradients/s (forward with checkpoints + reverse sweep)", "forward_ms": fwd,
            "backward_ms": bwd, "backward_spring_updates_per_s": float(S.sum()) * N / (bwd * 1e-3)}


def measure_lamarckian(vs, stream, args, P=512, N=2000, K=100):
    """Gradient-assisted co-design generation on 512 robots 8x8x8 (per-voxel parameter genome
    rows, fixed morphology): forward with checkpoints, fitness, the elites picked on the GPU as
    adjoint weights, adjoint of the elites' summed fitness, Lamarckian gradient step, genetic
    operators -- no host round trip.  Generations per second."""
    import torch
    from paper_2405_00698_gb300 import codesign
    rng = np.random.default_rng(3)
    pop = W.population_uniform(P, (8, 8, 8), seed=3)
    w, kappa, phi = W.voxel_params(rng, pop)
    V = 512
    rows = np.concatenate([w.reshape(P, V), kappa.reshape(P, V), phi.reshape(P, V)], axis=1)
    g = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.float32)).cuda()
    mats = torch.from_numpy(np.ascontiguousarray(pop.mats)).cuda()
    sim = vs.Simulator(W.CONFIG, stream=stream)
    evo = W.Evolution()
    state = {"gen": 0, "g": g}

    def generation():
        _, state["g"] = codesign.run_lamarckian(sim, mats, state["g"], (8, 8, 8), 1, N, evo,
                                                eta=(0.02, 50.0, 0.1), checkpoint=K,
                                                first_generation=state["gen"], log=False)
        state["gen"] += 1
    generation()                                      # warm-up
    ms = _timed(stream, generation)
    _, S = sim.counts()
    sim.close()
    return {"workload": f"{P} robots 8x8x8, parameter genome rows, {N} steps, checkpoints every {K}, "
                        f"gradient step on the {evo.elites(P)} elites picked on the GPU", "ms_per_generation": ms,
            "generations_per_s": 1e3 / ms,
            "forward_spring_updates_per_s": float(S.astype(np.int64).sum()) * N / (ms * 1e-3)}


def measure_paper_preset(vs, stream, args, N=20000):
    """The paper's own workload (Table I / Table II): 30 robots on a 5x5x5 grid, time step 1e-5 s
    with the spring and ground dashpots, then one generation with crossover rate 0.4.  20,000
    steps (0.2 s of simulated time) per generation; reported as spring updates and as springs +
    masses per second, next to the paper's 7.89e9 (RTX 3090, unit unstated)."""
    import torch
    pop = W.population_uniform(30, (5, 5, 5), seed=11)
    sim = vs.Simulator(W.PAPER, stream=stream)
    evo = W.PAPER_EVOLUTION
    g = torch.from_numpy(W.one_hot_logits(pop.mats).reshape(pop.P, -1).copy()).cuda()
    out = torch.empty_like(g)
    fit = torch.empty(pop.P, dtype=torch.float64, device="cuda")

    def generation():
        sim.set_population(pop.dims, g, vs.MODE_LOGITS)
        sim.step(N)
        sim.fitness(fit)
        sim.evo_generation(fit, g, out, evo, 0)
    generation()                                      # warm-up
    ms = _timed(stream, generation)
    M, S = sim.counts()
    sim.close()
    Ssum, Msum = float(S.astype(np.int64).sum()), float(M.astype(np.int64).sum())
    return {"workload": f"30 robots 5x5x5 (Table I), Table II physics with dashpots, {N} steps of 1e-5 s, "
                        "one generation (crossover 0.4, elites 0.3, mutation 0.1 / 0.1)",
            "ms_per_generation": ms, "spring_updates_per_s": Ssum * N / (ms * 1e-3),
            "spring_plus_mass_updates_per_s": (Ssum + Msum) * N / (ms * 1e-3),
            "paper_figure": 7892537853, "note": "the paper's figure is on an RTX 3090 with unstated unit and workload"}


def measure_streamed_adjoint(vs, stream, args, peaks, P=64, n=40, N=5000, K=100, records=False):
    """The adjoint on large robots (64 robots 40x40x40 at occupancy 0.7, state in HBM, 5000
    steps): forward with checkpoints every 100 steps, then the backward pass (segment replays
    with recording and the reverse sweep), as robot gradients per second and as algorithmic HBM
    bytes against the measured peak.  records: the forward also keeps every step's record (24 B
    per corner per step) and the backward only sweeps; the whole workload's records would take
    530 GB, so that variant runs on a sample that fits (the caller's P and N)."""
    import torch
    rng = np.random.default_rng(6)
    pop = W.workload_large(P, seed=5, n=n)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim = vs.Simulator(W.CONFIG, stream=stream)
    sim.set_checkpointing(K)
    sim.set_trajectory_records(records)
    args_pop = (t(pop.mats), t(w), t(kappa), t(phi))
    g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
    dl = torch.ones(P, dtype=torch.float64, device="cuda")
    if not records:
        sim.set_population(pop.dims, args_pop, vs.MODE_PARAMS)
        sim.step(2 * K)
        sim.backward(dl, *g)                       # warm-up of the backward's buffers
    sim.set_population(pop.dims, args_pop, vs.MODE_PARAMS)
    sim.step(N)                                    # warm-up: checkpoints, the N-step graph
    if records:
        sim.backward(dl, *g)
    sim.set_population(pop.dims, args_pop, vs.MODE_PARAMS)
    fwd = _timed(stream, lambda: sim.step(N))
    bwd = _timed(stream, lambda: sim.backward(dl, *g))
    M, S = sim.counts()
    sim.close()
    Ssum, Msum = float(S.astype(np.int64).sum()), float(M.astype(np.int64).sum())
    # algorithmic device-memory bytes per step: forward 12 B per spring + 64 B per mass (+ 24 B
    # per mass of records when kept); backward: the replay with records (12 B per spring + 88 B
    # per mass, none when the records are kept) and the reverse step (36 B per spring: parameters
    # and sensitivity sums read and written; 136 B per mass: records and adjoints)
    fwd_gbs = (12.0 * Ssum + (88.0 if records else 64.0) * Msum) * N / (fwd * 1e-3) / 1e9
    bwd_gbs = ((36.0 if records else 48.0) * Ssum + (136.0 if records else 224.0) * Msum) * N / (bwd * 1e-3) / 1e9
    kept = ", every step's record kept" if records else ""
    sample = "" if (P, N) == (64, 5000) else f" (sample of 64 robots x 5000 steps)"
    return {"workload": f"{P} robots {n}^3, occupancy 0.7, per-voxel parameters, {N} steps{sample}, "
                        f"checkpoints every {K}{kept}",
            "grads_per_s": P / ((fwd + bwd) * 1e-3), "forward_ms": fwd, "backward_ms": bwd,
            "forward_roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": fwd_gbs / peaks["hbm_gbs"]},
            "backward_roofline": {"bound": "hbm", "achieved": bwd_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": bwd_gbs / peaks["hbm_gbs"]}}


def measure_streamed(vs, stream, args, peaks, P=64, n=40, N=5000):
    """64 robots 40x40x40 at occupancy 0.7 (Bernoulli, largest component), state in HBM, one
    launch per step, 5000 steps (the N-step loop replayed as one CUDA graph)."""
    pop = W.workload_large(P, seed=5, n=n)
    sim = vs.Simulator(W.CONFIG, stream=stream)
    sim.set_population_from(pop)
    M, S = sim.counts()
    sim.step(20)
    sim.timing()
    ms = _timed(stream, lambda: sim.step(N))
    kms, launches = sim.timing()
    sim.close()
    ups = float(S.astype(np.int64).sum()) * N / (ms * 1e-3)
    # algorithmic bytes per step: per spring its 12 B of parameters, per mass u and v read and
    # written (4 x 16 B)
    alg = (12.0 * S.astype(np.int64).sum() + 64.0 * M.astype(np.int64).sum()) * N
    gbs = alg / (kms * 1e-3) / 1e9
    cpu = None
    if not getattr(args, "no_cpu_baseline", False):
        ncpu = min(P, 16)
        cpu = cpu_baseline_population(pop.subset(range(ncpu)), 50, f"{ncpu} of the {P} robots, 50 steps")
    return {"workload": f"{P} robots {n}^3, occupancy 0.7, {N} steps", "unit": "spring-updates/s",
            "value": ups, "springs_per_robot": float(S.mean()), "masses_per_robot": float(M.mean()),
            "launches": launches, "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                                               "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                                               "note": "the algorithmic bound; measured, the kernel is bound by "
                                                       "instruction issue and load latency (65 % of issue slots, "
                                                       "every spring evaluated by both ends), not by HBM: "
                                                       "populations that fit L2 run no faster"},
            **({"cpu_baseline": cpu} if cpu else {})}


# ------------------------------------------------------------------------------------------
# the CPU oracle (baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_generation(genomes, Bmat, N, nthreads=0):
    """The oracle's pass over a sample: MLP decode, simulation, fitness, one evolution
    generation.  Returns (spring updates, threads used)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    P = genomes.shape[0]
    with ThreadPoolExecutor(max_workers=nthreads if nthreads > 0 else (os.cpu_count() or 4)) as ex:
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
    """The oracle on a sample of the genomes sized to about budget_s seconds: a first chunk of
    16 measures the rate, a second call takes as many further genomes (multiples of 16) as the
    rest of the budget allows."""
    n = 16
    t0 = time.perf_counter()
    upd, th = oracle_generation(genomes[:n], Bmat, N)
    dt = time.perf_counter() - t0
    more = min(len(genomes) - n, int((budget_s - dt) / dt) * n) if dt < budget_s else 0
    if more > 0:
        t1 = time.perf_counter()
        u2, th = oracle_generation(genomes[n:n + more], Bmat, N)
        dt += time.perf_counter() - t1
        upd += u2
        n += more
    # the same pass on one host thread, over two genomes (about a second)
    t2 = time.perf_counter()
    u1, _ = oracle_generation(genomes[:2], Bmat, N, nthreads=1)
    dt1 = time.perf_counter() - t2
    return {"value": upd / dt, "unit": "spring-updates/s", "cores": th, "kind": "oracle",
            "sample": f"{n} of the 1024 genomes, full {N}-step generation (decode, simulate, "
                      f"fitness, evolve), OpenMP over robots; {dt:.1f} s",
            "single_thread": {"value": u1 / dt1, "unit": "spring-updates/s", "cores": 1,
                              "sample": f"2 of the 1024 genomes, full {N}-step generation; {dt1:.1f} s"}}


def cpu_baseline_population(pop, N, sample):
    """The oracle simulating a sample of one of the other workloads (direct materials, no
    decode or evolution), OpenMP over its robots: spring updates per second."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    res = O.run_population(pop, W.CONFIG, N)
    dt = time.perf_counter() - t0
    upd = int(res["S"].astype(np.int64).sum()) * N
    return {"value": upd / dt, "unit": "spring-updates/s", "cores": min(int(res["threads"]), pop.P),
            "kind": "oracle", "sample": f"{sample}; {dt:.1f} s"}


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


def run_case(args):
    """One extra measurement alone, printed as its own JSON object (a profiling aid, not a bench
    line)."""
    import torch
    from paper_2405_00698_gb300 import build as B
    from paper_2405_00698_gb300 import voxsim as vs
    B.build()
    stream = torch.cuda.current_stream()
    peaks, _ = measured_peaks()
    if args.case == "streamed":
        P = args.robots if args.robots != P_ROBOTS else 64
        N = args.sim_steps if args.sim_steps != SIM_STEPS else 5000
        print(json.dumps({"case": args.case, **measure_streamed(vs, stream, args, peaks, P=P, N=N)}))
    elif args.case == "paper_preset":
        print(json.dumps({"case": args.case, **measure_paper_preset(vs, stream, args)}))
    elif args.case == "uneven":
        P = args.robots if args.robots != P_ROBOTS else 4096
        N = args.sim_steps if args.sim_steps != SIM_STEPS else 5000
        print(json.dumps({"case": args.case, **measure_uneven(vs, stream, args, peaks, P=P, N=N)}))
    elif args.case == "adjoint":
        P = args.robots if args.robots != P_ROBOTS else 512
        N = args.sim_steps if args.sim_steps != SIM_STEPS else 2000
        print(json.dumps({"case": args.case, **measure_adjoint(vs, stream, args, P=P, N=N)}))
        print(json.dumps({"case": args.case, **measure_adjoint(vs, stream, args, P=P, N=N, records=True)}))
    else:
        P = args.robots if args.robots != P_ROBOTS else 64
        N = args.sim_steps if args.sim_steps != SIM_STEPS else 5000
        print(json.dumps({"case": args.case, **measure_streamed_adjoint(vs, stream, args, peaks, P=P, N=N)}))
        print(json.dumps({"case": args.case, **measure_streamed_adjoint(vs, stream, args, peaks, P=min(P, 16),
                                                                        N=min(N, 2000), records=True)}))


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
