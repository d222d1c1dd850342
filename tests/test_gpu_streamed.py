"""The streamed path (state in device memory, one launch per step) for robots too large for one
SM: bit-identical to the resident lattice path where both apply (same arithmetic, same
summation order), and within tolerance of the oracle on large robots."""
import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W
from tests.parity import check_population

pytestmark = pytest.mark.gpu
PHYS = W.CONFIG


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


def run(vs, pop, nsteps, **kw):
    sim = vs.Simulator(PHYS, **kw)
    sim.set_population_from(pop)
    sim.step(nsteps)
    x, v, off = sim.state()
    f = sim.fitness()
    sim.close()
    return x, v, off, f


@pytest.mark.parametrize("nsteps", [301, 400])
def test_streamed_equals_resident_lattice_bitwise(vs, nsteps):
    pop = W.population_uneven(12, seed=70, sizes=(2, 4, 6, 8))
    a = run(vs, pop, nsteps)
    b = run(vs, pop, nsteps, path=vs.PATH_STREAMED)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])


def test_forty_cube_instantiation_equals_the_generic_kernel(vs):
    """Streamed robots that are all 40 x 40 x 40 run the compile-time instantiation of that
    grid; one robot of another grid added sends the same robots through the generic kernel.
    States and fitness agree bit for bit (an odd step count leaves the newest state in the
    alternate buffer)."""
    rng = np.random.default_rng(76)
    dims = [(40, 40, 40), (40, 40, 40)]
    grids = [W.bernoulli_grid(rng, d, 0.7) for d in dims]
    extra = W.bernoulli_grid(rng, (30, 20, 25), 0.7)
    pop = W.make_population(dims, grids)
    both = W.make_population(dims + [(30, 20, 25)], grids + [extra])
    a = run(vs, pop, 151, path=vs.PATH_STREAMED)
    b = run(vs, both, 151, path=vs.PATH_STREAMED)
    n = int(a[2][-1])
    assert np.array_equal(a[0], b[0][:n]) and np.array_equal(a[1], b[1][:n])
    assert np.array_equal(a[3], b[3][:2])


def test_large_robots_match_oracle(vs, orc):
    """Bernoulli(0.7) grids of 16^3 and 20x18x22 voxels (more corners than one SM holds)."""
    grids = [W.bernoulli_grid(np.random.default_rng(71), (16, 16, 16), 0.7),
             W.bernoulli_grid(np.random.default_rng(72), (20, 18, 22), 0.7)]
    pop = W.make_population([(16, 16, 16), (20, 18, 22)], grids)
    x, v, off, f = run(vs, pop, 300)
    ref = orc.run_population(pop, PHYS, 300, want_x=True)
    check_population(orc, pop, PHYS, 300, f, x, off, ref)


def test_mixed_population_all_paths(vs, orc):
    """One population with lattice (small), atomic-resident (12^3) and streamed (18^3) robots."""
    rng = np.random.default_rng(73)
    dims = [(4, 4, 4), (8, 8, 8), (12, 12, 12), (18, 18, 18), (3, 5, 2)]
    grids = [W.bernoulli_grid(rng, d, 0.75) for d in dims]
    pop = W.make_population(dims, grids)
    x, v, off, f = run(vs, pop, 251)
    ref = orc.run_population(pop, PHYS, 251, want_x=True)
    check_population(orc, pop, PHYS, 251, f, x, off, ref)


def test_plain_baseline_path_matches_oracle(vs, orc):
    """The paper's organisation (one launch per robot per pass) kept as the measured baseline."""
    pop = W.population_uneven(10, seed=74, sizes=(2, 4, 7))
    x, v, off, f = run(vs, pop, 300, path=vs.PATH_PLAIN)
    ref = orc.run_population(pop, PHYS, 300, want_x=True)
    check_population(orc, pop, PHYS, 300, f, x, off, ref)
