"""GPU vs oracle parity of decode, largest component, topology, time stepping and fitness.

Tolerances: integer work (materials, kept voxels, mass corners, spring endpoints, counts) is
bit-exact; positions after the run within 1e-4 of the robot size s * max(n) (max-norm), fitness
within 1e-3 relative with a floor of 1e-3 * s (see tests/parity.py for robots whose trajectory
crosses a stick/slip switch within float32 rounding); spring parameters within float32
rounding."""
import dataclasses

import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W
from tests.parity import FIT_TOL, POS_TOL, check_population

pytestmark = pytest.mark.gpu

PHYS = W.CONFIG


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build
    build.build()
    from paper_2405_00698_gb300 import voxsim
    return voxsim


def run_both(vs, orc, pop, phys, nsteps, **kw):
    sim = vs.Simulator(phys, **kw)
    sim.set_population_from(pop)
    sim.step(nsteps)
    f = sim.fitness()
    x, v, off = sim.state()
    M, S = sim.counts()
    ref = orc.run_population(pop, phys, nsteps, want_x=True)
    sim.close()
    return dict(f=f, x=x, off=off, M=M, S=S), ref


def test_small_workload_1000_steps(vs, orc):
    """16 robots, 4x4x4, materials uniform over the five ids, 1000 steps."""
    pop = W.workload_small(seed=0)
    g, ref = run_both(vs, orc, pop, PHYS, 1000)
    assert np.array_equal(g["M"], ref["M"]) and np.array_equal(g["S"], ref["S"])
    check_population(orc, pop, PHYS, 1000, g["f"], g["x"], g["off"], ref)


def test_topology_bit_exact(vs, orc):
    pop = W.population_uneven(24, seed=21, sizes=(1, 2, 3, 5, 7, 9))
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    vox = sim.voxels()
    topo = sim.topology()
    mo = so = 0
    for r in range(pop.P):
        R = orc.Robot(pop.grid(r), pop.dims[r], PHYS)
        t = R.topology()
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        assert np.array_equal(vox["kept"][a:b], t["kept"]), r
        assert topo["M"][r] == R.M and topo["S"][r] == R.S, r
        assert np.array_equal(topo["mass_corner"][mo:mo + R.M], t["mass_corner"]), r
        ab = topo["ab"][so:so + R.S]
        assert np.array_equal(ab[:, 0], t["a"]) and np.array_equal(ab[:, 1], t["b"]), r
        sp = topo["params"][so:so + R.S].astype(np.float64)
        assert np.allclose(sp[:, 0], t["L0"], rtol=1e-6)
        assert np.allclose(sp[:, 1], t["k"], rtol=1e-6)
        assert np.allclose(sp[:, 2], t["alpha"], atol=1e-6)
        assert np.allclose(sp[:, 3], t["beta"], atol=1e-6)
        mo += R.M
        so += R.S
    sim.close()


def test_uneven_population_ragged_sizes(vs, orc):
    """Grids from 1 to 12 voxels per axis, several tiles and ragged tails of threads."""
    pop = W.population_uneven(40, seed=22, sizes=(1, 3, 4, 6, 8, 12))
    g, ref = run_both(vs, orc, pop, PHYS, 400)
    assert np.array_equal(g["S"], ref["S"])
    check_population(orc, pop, PHYS, 400, g["f"], g["x"], g["off"], ref)


@pytest.mark.parametrize("threads", [32, 96, 256, 1024])
def test_thread_counts_agree(vs, orc, threads):
    pop = W.population_uneven(8, seed=23, sizes=(4, 8, 12))
    g, ref = run_both(vs, orc, pop, PHYS, 300, threads=threads)
    check_population(orc, pop, PHYS, 300, g["f"], g["x"], g["off"], ref)


def test_empty_and_degenerate_robots(vs, orc):
    grids = [np.zeros((2, 2, 2), np.uint8),              # empty: no masses, fitness 0
             np.full((1, 1, 1), 4, np.uint8),            # one voxel
             np.array([[[1, 0, 2]]], np.uint8),          # two components of equal size
             np.full((1, 1, 12), 3, np.uint8)]           # a rod
    pop = W.make_population([g.shape[::-1] for g in grids], grids)
    g, ref = run_both(vs, orc, pop, PHYS, 500)
    assert list(g["M"]) == list(ref["M"]) and g["M"][0] == 0
    assert g["f"][0] == 0.0
    check_population(orc, pop, PHYS, 500, g["f"], g["x"], g["off"], ref)


def test_split_calls_continue_time(vs, orc):
    """step(300) + step(700) equals step(1000): the actuation clock runs across calls."""
    pop = W.workload_small(seed=3).subset(range(6))
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    sim.step(300)
    sim.step(700)
    x, _, off = sim.state()
    f = sim.fitness()
    ref = orc.run_population(pop, PHYS, 1000, want_x=True)
    check_population(orc, pop, PHYS, 1000, f, x, off, ref)
    sim.close()


def test_no_ground_conserves_centroid(vs):
    phys = dataclasses.replace(PHYS, gravity=0.0, ground_on=False, damping=1.0)
    pop = W.workload_small(seed=4)
    sim = vs.Simulator(phys)
    sim.set_population_from(pop)
    sim.step(1000)
    assert np.abs(sim.fitness()).max() < 1e-5
    sim.close()


def test_dead_robot_scores_minus_infinity(vs, orc):
    phys = dataclasses.replace(PHYS, dt=2e-2)      # far beyond the stability limit
    pop = W.workload_small(seed=5).subset(range(3))
    sim = vs.Simulator(phys)
    sim.set_population_from(pop)
    sim.step(200)
    f = sim.fitness()
    ref = orc.run_population(pop, phys, 200)
    assert np.all(np.isneginf(f)) and np.all(np.isneginf(ref["fitness"]))
    sim.close()


def test_logits_mode(vs, orc):
    rng = np.random.default_rng(31)
    pop = W.population_uniform(6, (5, 4, 3), seed=31)
    logits = rng.standard_normal((pop.mats.size, 5)).astype(np.float32)
    logits[::7, 2] = logits[::7, 1]                  # exact ties go to the lower id
    sim = vs.Simulator(PHYS)
    sim.set_population(pop.dims, logits, vs.MODE_LOGITS)
    vox = sim.voxels()
    assert np.array_equal(vox["decoded"], np.argmax(logits, axis=1).astype(np.uint8))
    sim.step(300)
    f = sim.fitness()
    x, _, off = sim.state()
    ref_pop = W.make_population(pop.dims, [np.argmax(logits[pop.voxel_off[r]:pop.voxel_off[r + 1]], axis=1)
                                           .astype(np.uint8) for r in range(pop.P)])
    ref = orc.run_population(ref_pop, PHYS, 300, want_x=True)
    check_population(orc, ref_pop, PHYS, 300, f, x, off, ref)
    sim.close()


def test_params_mode(vs, orc):
    rng = np.random.default_rng(32)
    pop = W.population_uniform(5, (4, 4, 4), seed=32)
    w, kappa, phi = W.voxel_params(rng, pop)
    sim = vs.Simulator(PHYS)
    sim.set_population(pop.dims, (pop.mats, w, kappa, phi), vs.MODE_PARAMS)
    sim.step(800)
    f = sim.fitness()
    x, _, off = sim.state()
    ref = orc.run_population(pop, PHYS, 800, w=w, kappa=kappa, phi=phi, want_x=True)
    check_population(orc, pop, PHYS, 800, f, x, off, ref, w=w, kappa=kappa, phi=phi)
    sim.close()


def test_device_inputs(vs, orc):
    import torch
    pop = W.workload_small(seed=6).subset(range(5))
    sim = vs.Simulator(PHYS)
    sim.set_population(pop.dims, torch.from_numpy(pop.mats).cuda(), vs.MODE_MATERIALS)
    sim.step(200)
    out = torch.empty(pop.P, dtype=torch.float64, device="cuda")
    sim.fitness(out)
    torch.cuda.synchronize()
    x, _, off = sim.state()
    ref = orc.run_population(pop, PHYS, 200, want_x=True)
    check_population(orc, pop, PHYS, 200, out.cpu().numpy(), x, off, ref)
    sim.close()


def test_invalid_inputs_rejected(vs):
    sim = vs.Simulator(PHYS)
    with pytest.raises(vs.VoxsimError):
        sim.step(10)                                   # no population yet
    bad = np.full(8, 9, np.uint8)
    with pytest.raises(vs.VoxsimError):
        sim.set_population([[2, 2, 2]], bad)
    with pytest.raises(vs.VoxsimError):
        sim.set_population([[0, 2, 2]], np.zeros(0, np.uint8))
    with pytest.raises(vs.VoxsimError):
        sim.set_population([[65, 1, 1]], np.zeros(65, np.uint8))
    sim.close()


def test_gather_stepping_is_bit_reproducible(vs):
    """The lattice-gather path sums every mass's forces in a fixed order: two runs agree bitwise."""
    pop = W.population_uneven(30, seed=24, sizes=(2, 4, 6, 8))
    out = []
    for _ in range(2):
        sim = vs.Simulator(PHYS, accumulate=vs.ACC_GATHER)
        sim.set_population_from(pop)
        sim.step(700)
        x, v, _ = sim.state()
        out.append((x, v, sim.fitness()))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


def test_atomic_path_matches_oracle(vs, orc):
    """Every robot on the shared-memory-atomic kernel (the path of robots with more corners than a
    lattice block holds)."""
    pop = W.population_uneven(20, seed=25, sizes=(3, 5, 8, 12))
    g, ref = run_both(vs, orc, pop, PHYS, 500, accumulate=vs.ACC_ATOMIC)
    check_population(orc, pop, PHYS, 500, g["f"], g["x"], g["off"], ref)


def test_atomic_kernel_spring_tiers(vs, orc):
    """Full robots on the atomic kernel whose springs span its three stores: each thread's first
    16 springs in tensor memory (1024 threads), the next ones in shared memory as far as they fit
    beside the state, the rest read from device memory every step (12 x 12 x 13: 26,197 springs,
    16,384 in tensor memory, about 7,900 in shared memory, about 1,900 from L2)."""
    rng = np.random.default_rng(27)
    dims = [(12, 12, 13), (12, 12, 12), (7, 9, 11)]
    grids = [W.bernoulli_grid(rng, d, 1.0) for d in dims]
    pop = W.make_population(dims, grids)
    g, ref = run_both(vs, orc, pop, PHYS, 300, accumulate=vs.ACC_ATOMIC)
    assert np.array_equal(g["S"], ref["S"]) and int(g["S"][0]) > 16384 + 8192
    check_population(orc, pop, PHYS, 300, g["f"], g["x"], g["off"], ref)


def test_shared_memory_probe(vs):
    """The shared-memory bandwidth probe (the resident kernels' roofline denominator) returns a
    rate between 30 % and 110 % of 128 B per clock per SM at the 2.07 GHz maximum clock."""
    import torch
    sim = vs.Simulator(PHYS)
    g = sim.measure_smem_bandwidth()
    sim.close()
    nominal = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2.07
    assert 0.3 * nominal < g < 1.1 * nominal, (g, nominal)


def test_gather_mode_keeps_large_robots_deterministic(vs):
    """Under bit-reproducible stepping a robot larger than a lattice block runs on a kernel with
    the same fixed summation order (a cluster of lattice blocks), and two runs agree bitwise."""
    pop = W.population_uneven(3, seed=26, sizes=(12,))
    out = []
    for _ in range(2):
        sim = vs.Simulator(PHYS, accumulate=vs.ACC_GATHER)
        sim.set_population_from(pop)
        sim.step(101)
        out.append(sim.state()[0])
        sim.close()
    assert np.array_equal(out[0], out[1])


def test_maximum_and_ragged_grids(vs, orc):
    """Grids at the largest extent per axis (64): a sparse 64x64x64 robot (its largest component
    on the streamed path), a 64-voxel rod along each axis, and a 1x64x2 sheet, in one population
    with a small robot; 30 steps against the oracle."""
    rng = np.random.default_rng(31)
    dims = [(64, 64, 64), (64, 1, 1), (1, 64, 1), (1, 1, 64), (1, 64, 2), (3, 2, 2)]
    grids = [W.bernoulli_grid(rng, dims[0], 0.35)] + [np.full(d[::-1], 4, np.uint8) for d in dims[1:]]
    pop = W.make_population(dims, grids)
    g, ref = run_both(vs, orc, pop, PHYS, 30)
    assert np.array_equal(g["M"], ref["M"]) and np.array_equal(g["S"], ref["S"])
    assert g["M"][0] > 20000
    check_population(orc, pop, PHYS, 30, g["f"], g["x"], g["off"], ref)


def test_empty_population(vs):
    """A population of no robots: every call succeeds and does nothing."""
    sim = vs.Simulator(PHYS)
    sim.set_population(np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    sim.step(100)
    assert sim.fitness().size == 0
    M, S = sim.counts()
    assert M.size == 0 and S.size == 0
    sim.close()
