"""The co-design loop around the library (Section II-C, Section II-D, Fig. 2), its
gradient-assisted variant, and headless trajectory export.

Every generation runs on the GPU through the C ABI: MLP decode of all genomes, simulation,
fitness, then elite selection / crossover / mutation into the next genome matrix.  Between
generations the loop calls an optional hyper-parameter hook in the place the paper gives to its
LLM supervisor (Section II-D: the parameters and populations of the three previous generations
go in, the parameters of the next generation come out).  The LLM itself is an external service
and is not part of this package; `stagnation_hook` is a deterministic stand-in rule.

Diversity is logged per generation (the paper's Fig. 3(b) names a diversity curve without a
definition): the RMS pairwise genome distance and the mean pairwise fraction of differing voxels.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import voxsim as vs
from . import workloads as W


@dataclasses.dataclass
class GenerationRecord:
    generation: int
    best: float
    mean: float
    median: float
    dead: int
    genome_diversity: float
    morphology_diversity: float
    spring_updates: int
    evolution: W.Evolution


Hook = Callable[[Sequence[GenerationRecord], W.Evolution], W.Evolution]


def stagnation_hook(history: Sequence[GenerationRecord], evo: W.Evolution) -> W.Evolution:
    """Stand-in supervisor: when the best fitness has not improved over the last three
    generations, raise the mutation rate and scale by half (up to 0.5 / 0.5); otherwise relax
    them by 10 % toward the configuration values."""
    base = W.Evolution()
    if len(history) >= 3 and history[-1].best <= history[-3].best:
        return dataclasses.replace(evo, mut_rate=min(0.5, evo.mut_rate * 1.5), sigma=min(0.5, evo.sigma * 1.5))
    return dataclasses.replace(evo, mut_rate=evo.mut_rate + 0.1 * (base.mut_rate - evo.mut_rate),
                               sigma=evo.sigma + 0.1 * (base.sigma - evo.sigma))


def run(sim: "vs.Simulator", genomes, B, dims: Sequence[int], generations: int, steps: int,
        evo: W.Evolution = W.Evolution(), hook: Optional[Hook] = None,
        first_generation: int = 0) -> tuple:
    """Run `generations` co-design generations of the MLP-encoded population.

    genomes: CUDA float32 tensor [P, 20998] (the population, updated in place); B: CUDA float32
    [128, 3]; dims: one grid shape for all robots.  Returns (records, final genomes tensor)."""
    import torch
    P = genomes.shape[0]
    d = np.tile(np.asarray(dims, np.int32), (P, 1))
    fit = torch.empty(P, dtype=torch.float64, device=genomes.device)
    other = torch.empty_like(genomes)
    cur = genomes
    records: List[GenerationRecord] = []
    for k in range(generations):
        gen = first_generation + k
        sim.set_population(d, cur, vs.MODE_MLP, B=B)
        sim.step(steps)
        sim.fitness(fit)
        _, S = sim.counts()
        f = fit.cpu().numpy()
        alive = f[np.isfinite(f)]
        gdiv, mdiv = sim.diversity(cur)
        records.append(GenerationRecord(
            generation=gen, best=float(alive.max()) if alive.size else float("-inf"),
            mean=float(alive.mean()) if alive.size else float("nan"),
            median=float(np.median(alive)) if alive.size else float("nan"),
            dead=int(P - alive.size), genome_diversity=gdiv, morphology_diversity=mdiv,
            spring_updates=int(S.astype(np.int64).sum()) * steps, evolution=evo))
        if hook is not None:
            evo = hook(records[-3:], evo)
        sim.evo_generation(fit, cur, other, evo, gen)
        cur, other = other, cur
    return records, cur


def param_bounds(V: int, device="cuda"):
    """Default box of a [w | kappa | phi] genome row: 0 <= w <= 1, kappa >= 0, phi free."""
    import torch
    inf = float("inf")
    lo = torch.tensor([0.0] * V + [0.0] * V + [-inf] * V, dtype=torch.float32, device=device)
    hi = torch.tensor([1.0] * V + [inf] * V + [inf] * V, dtype=torch.float32, device=device)
    return lo, hi


def rank_order(f: np.ndarray) -> np.ndarray:
    """The genetic operators' ranking: fitness descending, index ascending on ties, NaN counted as
    -infinity (after every finite fitness, tied with -infinity by index)."""
    key = np.where(np.isnan(f), -np.inf, f)
    return np.argsort(-key, kind="stable")


def run_lamarckian(sim: "vs.Simulator", mats, genomes, dims: Sequence[int], generations: int,
                   steps: int, evo: W.Evolution = W.Evolution(), eta=(0.0, 0.0, 0.0),
                   checkpoint: int = 100, bounds=None, first_generation: int = 0,
                   log: bool = True) -> tuple:
    """Gradient-assisted co-design on per-voxel parameter genomes (a project extension beside the
    paper's purely genetic loop): the morphology `mats` (CUDA uint8 [P * V]) stays fixed and each
    genome row is [w | kappa | phi] (CUDA float32 [P, 3V], updated in place).  Every generation:
    simulate with checkpoints, take the fitness, run the adjoint of the elites' summed fitness,
    move the elites one gradient step uphill (evo_gradient_step, per-segment steps `eta`, box
    `bounds` = (lo, hi) or the default of param_bounds), then breed the next generation with the
    unchanged genetic operators from the improved elites (their Gaussian mutation is not held to
    the box).  log=False skips the per-generation records (their host reads).  The elites are picked on the GPU (evo_elite_weights): the loop never waits for the
    host between generations except for the records it logs.  Returns (records, final
    genomes)."""
    import torch
    P, G = genomes.shape
    V = G // 3
    d = np.tile(np.asarray(dims, np.int32), (P, 1))
    lo, hi = bounds if bounds is not None else param_bounds(V, genomes.device)
    fit = torch.empty(P, dtype=torch.float64, device=genomes.device)
    dl = torch.zeros(P, dtype=torch.float64, device=genomes.device)
    gw, gk, gp = (torch.empty(P * V, dtype=torch.float32, device=genomes.device) for _ in range(3))
    other = torch.empty_like(genomes)
    cur = genomes
    sim.set_checkpointing(checkpoint)
    records: List[GenerationRecord] = []
    for k in range(generations):
        gen = first_generation + k
        sim.set_population(d, (mats, cur), vs.MODE_PARAM_ROWS)
        sim.step(steps)
        sim.fitness(fit)
        diversity = sim.diversity(cur)[0] if log else float("nan")
        # the elites' summed fitness as the adjoint's loss; every row takes the step (the others'
        # gradients are zero, and the generation below keeps only the elites' rows)
        sim.evo_elite_weights(fit, evo.elites(P), dl)
        sim.backward(dl, gw, gk, gp)
        sim.evo_gradient_step(cur, gw, gk, gp, eta, rows=None, lo=lo, hi=hi)
        if log:
            f = fit.cpu().numpy()
            alive = f[np.isfinite(f)]
            _, S = sim.counts()
            records.append(GenerationRecord(
                generation=gen, best=float(alive.max()) if alive.size else float("-inf"),
                mean=float(alive.mean()) if alive.size else float("nan"),
                median=float(np.median(alive)) if alive.size else float("nan"),
                dead=int(P - alive.size), genome_diversity=diversity,
                morphology_diversity=float("nan"), spring_updates=int(S.astype(np.int64).sum()) * steps,
                evolution=evo))
        sim.evo_generation(fit, cur, other, evo, gen)
        cur, other = other, cur
    return records, cur


def export_trajectory(sim: "vs.Simulator", frames: int, steps_per_frame: int, path: str) -> dict:
    """Headless replacement for the paper's OpenGL renders (Fig. 5): advance the current
    population and store the mass positions every `steps_per_frame` steps in an .npz file
    (positions [frames+1, total masses, 3], mass offsets per robot, grid shapes)."""
    x, _, off = sim.state()
    out = [x]
    for _ in range(frames):
        sim.step(steps_per_frame)
        out.append(sim.state()[0])
    data = dict(positions=np.stack(out), offsets=off, dims=np.asarray(sim.dims),
                steps_per_frame=np.int64(steps_per_frame))
    np.savez_compressed(path, **data)
    return data
