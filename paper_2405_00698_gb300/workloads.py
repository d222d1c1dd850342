"""Seeded synthetic inputs and parameter presets for the voxel soft-robot hot path.

This module holds data only: physical constants, evolution rates, and numpy generators of robot
populations shaped like the workloads of "CUDA-Accelerated Soft Robot Neural Evolution with Large
Language Model Supervision" (arXiv 2405.00698).  It contains none of the method's arithmetic.
Both the CUDA library and the FP64 oracle receive the same arrays produced here.

Material ids (Section II-A): 0 empty, 1 expanding muscle, 2 contracting muscle, 3 soft tissue,
4 bone.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

N_MAT = 5
GENOME_LEN = 20998          # MLP 3 -> gamma(256) -> 64 -> 64 -> 6 weights and biases
PE_M = 128                  # rows of the Gaussian encoding matrix B (Eq. (1), m = 128)
LAYERS = ((256, 64), (64, 64), (64, 6))   # (fan_in, fan_out) per dense layer


@dataclasses.dataclass(frozen=True)
class Physics:
    """Simulation constants.  Defaults are the configuration values of the workloads (time step
    1e-4 s, stiffness 5e3 N/m for muscle and soft tissue, 2e4 N/m for bone, amplitude 0.2 at
    2 Hz, ground 1e5 N/m, friction 1.0 / 0.8, velocity damping 0.999 per step); gravity, point
    mass and rest length are Table II's."""
    dt: float = 1e-4
    gravity: float = 9.81
    mass: float = 0.1
    edge: float = 0.1
    damping: float = 0.999
    k_ground: float = 1e5
    mu_s: float = 1.0
    mu_k: float = 0.8
    freq: float = 2.0
    dead_bound: float = 1e3
    k_mat: Tuple[float, ...] = (0.0, 5e3, 5e3, 5e3, 2e4)
    amp_mat: Tuple[float, ...] = (0.0, 0.2, 0.2, 0.0, 0.0)
    phase_mat: Tuple[float, ...] = (0.0, 0.0, math.pi, 0.0, 0.0)
    ground_on: bool = True
    spring_zeta: float = 0.0    # spring dashpot damping ratio
    ground_zeta: float = 0.0    # ground damping ratio


CONFIG = Physics()

# The paper's own constants (Table II): time step 1e-5 s, muscle 2e3, soft tissue 1e3, bone 1e4
# N/m, spring and ground damping ratios 0.1, muscle amplitude 0.25 with phase pi for the
# contracting muscle, ground 1e5 N/m, static / kinetic friction 0.6 / 1.0; no velocity damping.
PAPER = Physics(dt=1e-5, damping=1.0, mu_s=0.6, mu_k=1.0, k_mat=(0.0, 2e3, 2e3, 1e3, 1e4),
                amp_mat=(0.0, 0.25, 0.25, 0.0, 0.0), spring_zeta=0.1, ground_zeta=0.1)


@dataclasses.dataclass(frozen=True)
class Evolution:
    """Evolution rates: elite fraction 25 %, uniform crossover, Gaussian mutation sigma 0.05 at
    rate 0.1 per gene (configuration values; Table I gives 0.3 / 0.4 / 0.1 / 0.1)."""
    elite_frac: float = 0.25
    mut_rate: float = 0.1
    sigma: float = 0.05
    seed: int = 12345
    cross_rate: float = 1.0

    def elites(self, P: int) -> int:
        return max(1, min(P, math.ceil(self.elite_frac * P - 1e-9)))

    def mut_threshold(self) -> int:
        """Mutation threshold on a 32-bit uniform draw: floor(rate * 2^32), clamped."""
        return int(min(max(self.mut_rate, 0.0) * 4294967296.0, 4294967295.0))

    def keep_threshold(self) -> int:
        """A child skips crossover when its 32-bit draw is below floor((1 - rate) * 2^32)."""
        return int(min(max(1.0 - self.cross_rate, 0.0) * 4294967296.0, 4294967295.0))


# Table I: 100 generations of 30 robots on a 5x5x5 grid; mutation rate 0.1 and scale 0.1,
# crossover rate 0.4, elite fraction 0.3.
PAPER_EVOLUTION = Evolution(elite_frac=0.3, mut_rate=0.1, sigma=0.1, cross_rate=0.4)


@dataclasses.dataclass
class Population:
    """A population of voxel grids.  Voxel grid r has dims[r] = (nx, ny, nz) and occupies
    mats[voxel_off[r] : voxel_off[r+1]], index i + nx*(j + ny*k)."""
    dims: np.ndarray          # int32 [P, 3]
    mats: np.ndarray          # uint8 [sum V]
    voxel_off: np.ndarray     # int64 [P + 1]

    @property
    def P(self) -> int:
        return int(self.dims.shape[0])

    def grid(self, r: int) -> np.ndarray:
        nx, ny, nz = (int(v) for v in self.dims[r])
        return self.mats[self.voxel_off[r]:self.voxel_off[r + 1]].reshape(nz, ny, nx)

    def subset(self, idx: Sequence[int]) -> "Population":
        return make_population([self.dims[r] for r in idx], [self.grid(r) for r in idx])


def make_population(dims: Sequence[Sequence[int]], grids: Sequence[np.ndarray]) -> Population:
    d = np.asarray(dims, dtype=np.int32).reshape(-1, 3)
    sizes = [int(a) * int(b) * int(c) for a, b, c in d]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    mats = np.concatenate([np.asarray(g, dtype=np.uint8).reshape(-1) for g in grids]) \
        if grids else np.zeros(0, np.uint8)
    return Population(d, mats, off)


def uniform_materials(rng: np.random.Generator, dims: Sequence[int]) -> np.ndarray:
    """Every voxel drawn uniformly from the five materials (empty included)."""
    nx, ny, nz = dims
    return rng.integers(0, N_MAT, size=(nz, ny, nx), dtype=np.uint8)


def bernoulli_grid(rng: np.random.Generator, dims: Sequence[int], p: float) -> np.ndarray:
    """Each voxel occupied with probability p, material uniform over the four non-empty ones."""
    nx, ny, nz = dims
    occ = rng.random((nz, ny, nx)) < p
    mat = rng.integers(1, N_MAT, size=(nz, ny, nx), dtype=np.uint8)
    return np.where(occ, mat, 0).astype(np.uint8)


def connected_growth(rng: np.random.Generator, dims: Sequence[int], occupancy: float) -> np.ndarray:
    """A face-connected voxel set of ceil(occupancy * nx*ny*nz) voxels grown from a random seed
    voxel: each round accepts a random half of the free face-neighbours of the current set
    (never more than the target).  Materials uniform over the four non-empty ones."""
    nx, ny, nz = dims
    V = nx * ny * nz
    target = max(1, min(V, math.ceil(occupancy * V - 1e-9)))
    occ = np.zeros((nz, ny, nx), dtype=bool)
    occ[rng.integers(nz), rng.integers(ny), rng.integers(nx)] = True
    count = 1
    while count < target:
        nb = np.zeros_like(occ)
        nb[1:] |= occ[:-1]; nb[:-1] |= occ[1:]
        nb[:, 1:] |= occ[:, :-1]; nb[:, :-1] |= occ[:, 1:]
        nb[:, :, 1:] |= occ[:, :, :-1]; nb[:, :, :-1] |= occ[:, :, 1:]
        cand = np.flatnonzero(nb & ~occ)
        take = cand[rng.random(cand.size) < 0.5]
        if take.size == 0:
            take = cand[:1]
        if count + take.size > target:
            take = rng.choice(take, size=target - count, replace=False)
        occ.reshape(-1)[take] = True
        count += int(take.size)
    mat = rng.integers(1, N_MAT, size=(nz, ny, nx), dtype=np.uint8)
    return np.where(occ, mat, 0).astype(np.uint8)


def one_hot_logits(mats: np.ndarray) -> np.ndarray:
    """Per-voxel five material scores, 1.0 on the given material and 0.0 elsewhere (float32):
    the direct genome that Gaussian mutation can move."""
    m = np.asarray(mats, dtype=np.int64).reshape(-1)
    out = np.zeros((m.size, N_MAT), dtype=np.float32)
    out[np.arange(m.size), m] = 1.0
    return out


def pe_matrix(rng: np.random.Generator, sigma: float = 2.0) -> np.ndarray:
    """B in R^{128 x 3}, entries from N(0, sigma^2) (Eq. (1)), float32."""
    return (rng.standard_normal((PE_M, 3)) * sigma).astype(np.float32)


def mlp_genomes(rng: np.random.Generator, P: int) -> np.ndarray:
    """P genomes of 20998 float32 values: each layer's weights and biases uniform in
    (-1/sqrt(fan_in), 1/sqrt(fan_in)).  Layout W1[64][256], b1, W2[64][64], b2, W3[6][64], b3."""
    parts = []
    for fan_in, fan_out in LAYERS:
        bound = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=(P, fan_out * fan_in)))
        parts.append(rng.uniform(-bound, bound, size=(P, fan_out)))
    g = np.concatenate(parts, axis=1).astype(np.float32)
    assert g.shape[1] == GENOME_LEN
    return np.ascontiguousarray(g)


# ------------------------------------------------------------------------------------------
# Workload recipes (sizes and distributions of the five benchmark configurations).
# ------------------------------------------------------------------------------------------

def population_uniform(P: int, dims: Sequence[int], seed: int) -> Population:
    """P grids of the same shape, each voxel uniform over the five materials."""
    rng = np.random.default_rng(seed)
    return make_population([dims] * P, [uniform_materials(rng, dims) for _ in range(P)])


def population_uneven(P: int, seed: int, sizes=(4, 6, 8, 10, 12), occ=(0.3, 0.9)) -> Population:
    """P grids with each axis drawn independently from `sizes` and occupancy uniform in `occ`,
    grown connected, materials uniform over the four non-empty ones."""
    rng = np.random.default_rng(seed)
    dims, grids = [], []
    for _ in range(P):
        d = [int(rng.choice(sizes)) for _ in range(3)]
        o = float(rng.uniform(*occ))
        dims.append(d)
        grids.append(connected_growth(rng, d, o))
    return make_population(dims, grids)


def population_bernoulli(P: int, dims: Sequence[int], p: float, seed: int) -> Population:
    rng = np.random.default_rng(seed)
    return make_population([dims] * P, [bernoulli_grid(rng, dims, p) for _ in range(P)])


def workload_small(seed: int = 0) -> Population:
    """16 robots on a 4x4x4 grid, materials uniform over the five ids (the parity workload)."""
    return population_uniform(16, (4, 4, 4), seed)


def workload_mlp(P: int = 1024, seed: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """(genomes [P, 20998], B [128, 3]) of the MLP-encoded population on an 8x8x8 grid."""
    rng = np.random.default_rng(seed)
    B = pe_matrix(rng, 2.0)
    return mlp_genomes(rng, P), B


def workload_uneven(P: int = 4096, seed: int = 2) -> Population:
    return population_uneven(P, seed)


def workload_large(P: int = 64, seed: int = 5, n: int = 40, p: float = 0.7) -> Population:
    return population_bernoulli(P, (n, n, n), p, seed)


def voxel_params(rng: np.random.Generator, pop: Population, phys: Physics = CONFIG):
    """Per-voxel material weight, stiffness and phase for the differentiation workload:
    w ~ U(0.5, 1), kappa = the material's stiffness, phi = the material's phase plus U(-0.5, 0.5)
    (float32 arrays over all voxels)."""
    n = pop.mats.size
    w = rng.uniform(0.5, 1.0, n).astype(np.float32)
    kappa = np.asarray(phys.k_mat, dtype=np.float32)[pop.mats]
    phi = (np.asarray(phys.phase_mat, dtype=np.float32)[pop.mats]
           + rng.uniform(-0.5, 0.5, n).astype(np.float32)).astype(np.float32)
    return w, kappa, phi


def stratified_subset(counts: np.ndarray, n: int) -> List[int]:
    """n robot indices spread evenly over the robots sorted by `counts` (e.g. spring counts)."""
    order = np.argsort(counts, kind="stable")
    pick = np.linspace(0, len(order) - 1, num=min(n, len(order))).round().astype(int)
    return [int(order[i]) for i in pick]
