"""Which gradient comparison is posed at the differentiation workload's horizon (an 8x8x8 robot,
2000 steps of 1e-4 s).  CPU only, FP64 oracle on both sides.

A float32 implementation differs from FP64 by roundings of the size of one float32 ulp in every
input and every step.  Perturbing only the inputs by that much (each voxel stiffness scaled by
1 +- 6e-8) already flips stick / slip decisions of the FP64 run, and the FP64 adjoint gradient
of the perturbed run leaves the 1e-3 bar (scaled |dg| / max(|g|, 1e-3 max|g|)) on a large share
of the voxels: against the free FP64 run no float32 implementation can be held to 1e-3.  Along
fixed contact modes (one run's modes imposed on both sides) the same perturbation moves the
FP64 central differences by well under 1e-3: the gradient parity of the adjoint is therefore
defined along the oracle run's contact modes (tests/test_gpu_adjoint.py,
tests/test_gpu_full_size.py)."""
import numpy as np

from paper_2405_00698_gb300 import workloads as W

PHYS = W.CONFIG
N = 2000


def workload_robot(r=0):
    rng = np.random.default_rng(3)
    pop = W.population_uniform(512, (8, 8, 8), seed=3)
    w, kappa, phi = W.voxel_params(rng, pop)
    a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
    base = dict(w=w[a:b].astype(np.float64), kappa=kappa[a:b].astype(np.float64),
                phi=phi[a:b].astype(np.float64))
    return pop.grid(r), base


def perturbed(base):
    signs = np.random.default_rng(7).choice([-1.0, 1.0], size=base["kappa"].size)
    return dict(base, kappa=base["kappa"] * (1.0 + 6e-8 * signs))


def scaled(g_ref, g):
    sc = np.maximum(np.abs(g_ref), 1e-3 * np.abs(g_ref).max())
    return np.abs(g - g_ref) / sc


def test_free_run_gradient_leaves_the_bar_under_float32_sized_input_changes(orc):
    grid, base = workload_robot()
    kept = np.flatnonzero(orc.lcc(grid, (8, 8, 8)) > 0)
    pert = perturbed(base)
    _, h0 = orc.fitness_after(grid, (8, 8, 8), PHYS, N, **base)
    _, h1 = orc.fitness_after(grid, (8, 8, 8), PHYS, N, **pert)
    assert h0 != h1, "the perturbation must flip some contact decision"
    _, *g0 = orc.adjoint(grid, (8, 8, 8), PHYS, N, **base)
    _, *g1 = orc.adjoint(grid, (8, 8, 8), PHYS, N, **pert)
    e = np.concatenate([scaled(a[kept], b[kept]) for a, b in zip(g0, g1)])
    assert np.mean(e > 1e-3) > 0.2


def test_fixed_mode_differences_stay_within_the_bar_under_the_same_changes(orc):
    grid, base = workload_robot()
    kept = np.flatnonzero(orc.lcc(grid, (8, 8, 8)) > 0)
    pert = perturbed(base)
    _, modes, _ = orc.fitness_after_modes(grid, (8, 8, 8), PHYS, N, **base)
    _, *g0 = orc.adjoint(grid, (8, 8, 8), PHYS, N, **base)
    gmax = {"w": np.abs(g0[0][kept]).max(), "kappa": np.abs(g0[1][kept]).max(), "phi": np.abs(g0[2][kept]).max()}
    pick = np.random.default_rng(44)
    for _ in range(6):
        name = ("w", "kappa", "phi")[pick.integers(3)]
        v = int(pick.choice(kept))
        h = 1e-6 * max(1.0, abs(base[name][v]))
        fd = []
        for p in (base, pert):
            ap = dict(p, **{name: p[name].copy()}); ap[name][v] += h
            am = dict(p, **{name: p[name].copy()}); am[name][v] -= h
            fp, _, _ = orc.fitness_after_modes(grid, (8, 8, 8), PHYS, N, force=modes, **ap)
            fm, _, _ = orc.fitness_after_modes(grid, (8, 8, 8), PHYS, N, force=modes, **am)
            fd.append((fp - fm) / (2 * h))
        assert abs(fd[1] - fd[0]) <= 1e-3 * max(abs(fd[0]), 1e-3 * gmax[name]), (name, v, fd)
