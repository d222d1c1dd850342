"""The per-size-class autotuner of the stepping kernels: it leaves the state untouched, its
choices keep parity with the oracle, and it never picks a non-deterministic kernel when
bit-reproducibility is required."""
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


def test_autotune_preserves_state_and_parity(vs, orc):
    pop = W.population_uneven(60, seed=80, sizes=(2, 4, 6, 10, 12, 15))
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    sim.step(100)
    x_before, v_before, _ = sim.state()
    kind, threads = sim.autotune(20)
    x_after, v_after, _ = sim.state()
    assert np.array_equal(x_before, x_after) and np.array_equal(v_before, v_after)
    assert set(kind.tolist()) <= {0, 1, 2, 3, 4}
    sim.step(300)
    x, _, off = sim.state()
    f = sim.fitness()
    sim.close()
    ref = orc.run_population(pop, PHYS, 400, want_x=True)
    check_population(orc, pop, PHYS, 400, f, x, off, ref)


def test_autotune_under_gather_stays_deterministic(vs):
    pop = W.population_uneven(30, seed=81, sizes=(3, 5, 8))
    runs = []
    for _ in range(2):
        sim = vs.Simulator(PHYS, accumulate=vs.ACC_GATHER)
        sim.set_population_from(pop)
        kind, _ = sim.autotune(10)
        assert 1 not in kind.tolist()            # the atomic kernel sums in arbitrary order
        sim.step(200)
        runs.append(sim.state()[0])
        sim.close()
    assert np.array_equal(runs[0], runs[1])
