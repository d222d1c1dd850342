"""The paper's own constants (Table I / Table II): time step 1e-5 s, muscle / soft / bone
stiffness 2e3 / 1e3 / 1e4 N/m, spring and ground damping ratios 0.1, amplitude 0.25, friction
0.6 / 1.0; 30 robots on a 5x5x5 grid; crossover rate 0.4, elite fraction 0.3, mutation 0.1 / 0.1.
Every stepping path against the oracle, and the evolution step with its crossover rate."""
import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W
from tests.parity import check_population

pytestmark = pytest.mark.gpu
PHYS = W.PAPER


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


@pytest.mark.parametrize("kw", [{}, {"accumulate": 1}, {"path": 2}, {"path": 3}],
                         ids=["lattice", "atomic", "streamed", "plain"])
def test_paper_preset_population(vs, orc, kw):
    pop = W.population_uniform(30, (5, 5, 5), seed=97)
    sim = vs.Simulator(PHYS, **kw)
    sim.set_population_from(pop)
    sim.step(2000)
    x, v, off = sim.state()
    f = sim.fitness()
    sim.close()
    ref = orc.run_population(pop, PHYS, 2000, want_x=True)
    check_population(orc, pop, PHYS, 2000, f, x, off, ref)


def test_streamed_equals_lattice_with_dashpots(vs):
    pop = W.population_uniform(6, (5, 5, 5), seed=98)
    out = []
    for kw in ({}, {"path": 2}):
        sim = vs.Simulator(PHYS, **kw)
        sim.set_population_from(pop)
        sim.step(333)
        out.append(sim.state()[:2])
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_split_groups_with_degenerate_robots(vs, orc):
    """A population smaller than the SM count with dashpots runs its robots of up to 384 corners
    as split groups (a helper thread per corner): an empty robot, one voxel, two equal
    components, a rod, a 6x6x6 robot (343 corners: the largest split slot) and a 5x5x5 robot
    against the oracle, and bitwise against the streamed path (which never splits)."""
    rng = np.random.default_rng(99)
    grids = [np.zeros((2, 2, 2), np.uint8), np.full((1, 1, 1), 4, np.uint8),
             np.array([[[1, 0, 2]]], np.uint8), np.full((1, 1, 12), 3, np.uint8),
             W.uniform_materials(rng, (6, 6, 6)), W.uniform_materials(rng, (5, 5, 5))]
    pop = W.make_population([g.shape[::-1] for g in grids], grids)
    out = []
    for kw in ({}, {"path": 2}):
        sim = vs.Simulator(PHYS, **kw)
        sim.set_population_from(pop)
        sim.step(1500)
        out.append(sim.state() + (sim.fitness(),))
        sim.close()
    (x, v, off, f), (x2, v2, _, f2) = out
    assert np.array_equal(x, x2) and np.array_equal(v, v2) and np.array_equal(f, f2)
    assert f[0] == 0.0
    ref = orc.run_population(pop, PHYS, 1500, want_x=True)
    check_population(orc, pop, PHYS, 1500, f, x, off, ref)


def test_split_and_unsplit_groups_in_one_launch(vs, orc):
    """With dashpots and few robots, robots of up to 384 corners run split while an 8x8x8 robot
    (729 corners) runs unsplit in the same launch of the split instantiation: bitwise against the
    streamed path and against the oracle."""
    rng = np.random.default_rng(100)
    shapes = [(8, 8, 8), (5, 5, 5), (3, 4, 2)]
    pop = W.make_population(shapes, [W.uniform_materials(rng, d) for d in shapes])
    out = []
    for kw in ({}, {"path": 2}):
        sim = vs.Simulator(PHYS, **kw)
        sim.set_population_from(pop)
        sim.step(800)
        out.append(sim.state() + (sim.fitness(),))
        sim.close()
    (x, v, off, f), (x2, v2, _, f2) = out
    assert np.array_equal(x, x2) and np.array_equal(v, v2) and np.array_equal(f, f2)
    ref = orc.run_population(pop, PHYS, 800, want_x=True)
    check_population(orc, pop, PHYS, 800, f, x, off, ref)


def test_paper_evolution_crossover_rate(vs, orc):
    import torch
    rng = np.random.default_rng(99)
    P, G = 30, 5 * 5 * 5 * 5
    evo = W.PAPER_EVOLUTION
    f = rng.standard_normal(P)
    g = rng.standard_normal((P, G)).astype(np.float32)
    sim = vs.Simulator(PHYS)
    out = torch.empty((P, G), device="cuda")
    par = torch.empty((P, 2), dtype=torch.int32, device="cuda")
    mask = torch.empty((P, G), dtype=torch.uint8, device="cuda")
    sim.evo_generation(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), out, evo, 7, par, mask)
    torch.cuda.synchronize()
    ref = orc.evo_generation(f, g, evo.elites(P), evo.seed, 7, evo.mut_threshold(), evo.sigma, evo.keep_threshold())
    assert np.array_equal(par.cpu().numpy(), ref["parents"]) and np.array_equal(mask.cpu().numpy(), ref["mask"])
    mut = ref["mutate"] == 1
    o = out.cpu().numpy()
    assert np.array_equal(o[~mut], ref["genomes"][~mut].astype(np.float32))
    assert np.abs(o[mut] - ref["genomes"][mut]).max(initial=0.0) < 4e-6
    sim.close()


def test_adjoint_refuses_damped_physics(vs):
    sim = vs.Simulator(PHYS)
    with pytest.raises(vs.VoxsimError):
        sim.set_checkpointing(100)
    sim.close()
