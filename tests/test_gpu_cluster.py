"""The cluster lattice kernel (robots of more than 768 corners cut into 2..8 slabs of whole
corner layers, one CTA each, boundary positions and forces through distributed shared memory),
the bit-reproducible choice for such robots.  Same arithmetic and summation order as the
streamed path, so the two must agree bit for bit; and the FP64 oracle within the stated
tolerances."""
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


def run(vs, pop, phys, nsteps, **kw):
    sim = vs.Simulator(phys, **kw)
    sim.set_population_from(pop)
    sim.step(nsteps)
    x, v, off = sim.state()
    f = sim.fitness()
    _, launches = sim.timing()
    sim.close()
    return x, v, f, off, launches


# (dims, slabs): 13 layers of 81 corners in 2 slabs, 13 of 169 in 4, 41 of 49 in 3, 21 of 121
# in 4, 31 of 169 in 8
SHAPES = [((8, 8, 12), 2), ((12, 12, 12), 4), ((6, 6, 40), 3), ((10, 10, 20), 4), ((12, 12, 30), 8)]


@pytest.mark.parametrize("phys_name", ["CONFIG", "PAPER"])
def test_cluster_equals_streamed_bitwise(vs, phys_name):
    phys = getattr(W, phys_name)
    rng = np.random.default_rng(100)
    dims = [d for d, _ in SHAPES]
    pop = W.make_population(dims, [W.bernoulli_grid(rng, d, 0.8) for d in dims])
    n = 300 if phys_name == "CONFIG" else 800
    a = run(vs, pop, phys, n, accumulate=vs.ACC_GATHER, path=vs.PATH_RESIDENT)
    b = run(vs, pop, phys, n, path=vs.PATH_STREAMED)
    assert a[4] < 20                      # resident launches (one per cluster size), not per step
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_cluster_matches_oracle(vs, orc):
    rng = np.random.default_rng(101)
    dims = [(8, 8, 12), (12, 12, 12), (6, 6, 40)]
    pop = W.make_population(dims, [W.bernoulli_grid(rng, d, 0.7) for d in dims])
    x, v, f, off, launches = run(vs, pop, PHYS, 500, accumulate=vs.ACC_GATHER)
    assert launches < 20                  # clusters, not the streamed path's launch per step
    ref = orc.run_population(pop, PHYS, 500, want_x=True)
    check_population(orc, pop, PHYS, 500, f, x, off, ref)


def test_cluster_in_a_mixed_population(vs, orc):
    """Lattice blocks, clusters and the streamed path in one population and one call."""
    rng = np.random.default_rng(102)
    dims = [(4, 4, 4), (8, 8, 12), (3, 5, 2), (12, 12, 12), (30, 30, 10)]
    pop = W.make_population(dims, [W.bernoulli_grid(rng, d, 0.75) for d in dims])
    x, v, f, off, _ = run(vs, pop, PHYS, 250, accumulate=vs.ACC_GATHER)
    ref = orc.run_population(pop, PHYS, 250, want_x=True)
    check_population(orc, pop, PHYS, 250, f, x, off, ref)
