"""The variants of the lattice-gather kernel (a thread per mass in a slot sized by the robot's
corners; springs compacted per direction onto the first threads; several robots per block in
groups sized by their mass counts) evaluate the same springs with the same arithmetic and sum
every mass's forces in the same order, so they must agree bit for bit: on uniform, uneven and
MLP-decoded populations, with the spring and ground dashpots of the paper's preset, and as the
forward run the checkpointed adjoint replays.  The compacted and the mass-packed variants are
also held against the FP64 oracle directly."""
import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W
from tests.parity import check_population

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


def run(vs, pop, phys, nsteps, lattice, **kw):
    sim = vs.Simulator(phys, lattice=lattice, **kw)
    sim.set_population_from(pop)
    sim.step(nsteps)
    x, v, off = sim.state()
    f = sim.fitness()
    sim.close()
    return x, v, f, off


CASES = {
    "uniform-4cube": lambda: W.population_uniform(40, (4, 4, 4), seed=70),
    "uneven": lambda: W.population_uneven(60, seed=71, sizes=(2, 3, 4, 6, 8)),
    "sparse-8cube": lambda: W.population_bernoulli(20, (8, 8, 8), 0.45, seed=72),
    "full-8cube": lambda: W.population_bernoulli(4, (8, 8, 8), 1.0, seed=73),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("phys_name", ["CONFIG", "PAPER"])
@pytest.mark.parametrize("variant", ["COMPACT", "PACKED"])
def test_variants_agree_bitwise(vs, case, phys_name, variant):
    pop = CASES[case]()
    phys = getattr(W, phys_name)
    n = 600 if phys_name == "CONFIG" else 1500
    a = run(vs, pop, phys, n, vs.LATTICE_CORNER, path=vs.PATH_RESIDENT)
    b = run(vs, pop, phys, n, getattr(vs, "LATTICE_" + variant), path=vs.PATH_RESIDENT)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("variant", ["CORNER", "PACKED"])
def test_segmented_queue_equals_whole_runs(vs, variant):
    """With more work items than SMs (and enough steps) the per-corner and the mass-packed
    launches queue every item's steps as segments, each waiting for its item's previous segment;
    with at most one item per SM every item runs whole.  The same robots stepped either way agree
    bit for bit (8x8x8 robots at occupancy 0.7 have too many masses to share a block)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    P = sms + 48
    pop = W.population_bernoulli(P, (8, 8, 8), 0.7, seed=75)
    n = 700
    lattice = getattr(vs, "LATTICE_" + variant)
    a = run(vs, pop, W.CONFIG, n, lattice, path=vs.PATH_RESIDENT)
    parts = [run(vs, pop.subset(list(idx)), W.CONFIG, n, lattice, path=vs.PATH_RESIDENT)
             for idx in (range(0, sms), range(sms, P))]
    assert np.array_equal(a[0], np.concatenate([b[0] for b in parts]))
    assert np.array_equal(a[1], np.concatenate([b[1] for b in parts]))
    assert np.array_equal(a[2], np.concatenate([b[2] for b in parts]))


def test_packed_blocks_on_a_large_uneven_population(vs):
    """More lattice robots than SMs: several robots of mixed mass counts share each block (up to
    15 groups, the shared-memory budget binding for many small robots); the result is bitwise
    the one-robot-per-slot kernel's."""
    pop = W.population_uneven(700, seed=78, sizes=(2, 3, 4, 6, 8), occ=(0.2, 0.95))
    a = run(vs, pop, W.CONFIG, 300, vs.LATTICE_CORNER, path=vs.PATH_RESIDENT)
    b = run(vs, pop, W.CONFIG, 300, vs.LATTICE_PACKED, path=vs.PATH_RESIDENT)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_variants_agree_on_mlp_population(vs):
    import torch
    G, B = W.workload_mlp(P=48, seed=74)
    dims = np.tile(np.array([8, 8, 8], np.int32), (48, 1))
    out = []
    for lattice in (vs.LATTICE_CORNER, vs.LATTICE_COMPACT, vs.LATTICE_PACKED):
        sim = vs.Simulator(W.CONFIG, lattice=lattice)
        sim.set_population(dims, torch.from_numpy(G).cuda(), vs.MODE_MLP, B=torch.from_numpy(B).cuda())
        sim.step(400)
        out.append(sim.state()[:2])
        sim.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])


@pytest.mark.parametrize("variant", ["COMPACT", "PACKED"])
def test_variant_matches_oracle(vs, orc, variant):
    pop = W.population_uneven(24, seed=75, sizes=(3, 4, 6, 8), occ=(0.3, 0.7))
    x, v, f, off = run(vs, pop, W.CONFIG, 1000, getattr(vs, "LATTICE_" + variant))
    ref = orc.run_population(pop, W.CONFIG, 1000, want_x=True)
    check_population(orc, pop, W.CONFIG, 1000, f, x, off, ref)


def test_adjoint_after_either_variant(vs):
    """The adjoint replays its segments with its own kernel: its gradient is the same whichever
    variant ran the recorded forward pass (up to the order of the per-voxel float atomics that
    gather the spring sensitivities)."""
    import torch
    rng = np.random.default_rng(76)
    pop = W.population_uniform(8, (4, 4, 4), seed=76)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    grads = []
    for lattice in (vs.LATTICE_CORNER, vs.LATTICE_COMPACT, vs.LATTICE_PACKED):
        sim = vs.Simulator(W.CONFIG, lattice=lattice)
        sim.set_checkpointing(50)
        sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
        sim.step(300)
        n = pop.mats.size
        g = [torch.empty(n, device="cuda") for _ in range(3)]
        sim.backward(t(np.ones(pop.P)), *g)
        torch.cuda.synchronize()
        grads.append([a.cpu().numpy() for a in g])
        sim.close()
    for other in grads[1:]:
        for a, b in zip(grads[0], other):
            assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()


def test_autotune_reports_the_variant(vs):
    pop = W.population_uneven(200, seed=77, sizes=(4, 6, 8))
    sim = vs.Simulator(W.CONFIG, accumulate=vs.ACC_GATHER)
    sim.set_population_from(pop)
    kinds, _ = sim.autotune(20)
    sim.close()
    assert set(int(k) for k in kinds[:6]) <= {0, 3}
    sim = vs.Simulator(W.CONFIG, accumulate=vs.ACC_GATHER, lattice=vs.LATTICE_CORNER)
    sim.set_population_from(pop)
    kinds, _ = sim.autotune(20)
    sim.close()
    assert set(int(k) for k in kinds[:6]) <= {0}


def test_mass_groups_for_large_sparse_robots(vs, orc):
    """Robots of more than 768 corners but at most 768 masses run on the lattice kernel in
    mass-sized thread groups (SIM_LATTICE_PACKED asks for it; the autotuner may choose it): the
    same bits as the other deterministic kernels for such robots (the cluster of lattice blocks
    under bit-reproducible accumulation), and the oracle's trajectory."""
    rng = np.random.default_rng(79)
    dims = [(10, 10, 10), (12, 12, 8), (9, 11, 10), (12, 12, 12)]
    grids = [W.connected_growth(rng, d, occ) for d, occ in zip(dims, (0.3, 0.25, 0.35, 0.2))]
    pop = W.make_population(dims, grids)
    sim = vs.Simulator(W.CONFIG)
    sim.set_population_from(pop)
    M, _ = sim.counts()
    sim.close()
    C = np.array([(a + 1) * (b + 1) * (c + 1) for a, b, c in dims])
    assert np.all(C > 768) and np.all(M <= 768), (C, M)
    a = run(vs, pop, W.CONFIG, 500, vs.LATTICE_PACKED, accumulate=vs.ACC_GATHER)
    b = run(vs, pop, W.CONFIG, 500, vs.LATTICE_CORNER, accumulate=vs.ACC_GATHER)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    ref = orc.run_population(pop, W.CONFIG, 500, want_x=True)
    check_population(orc, pop, W.CONFIG, 500, a[2], a[0], a[3], ref)


def test_autotuner_may_choose_mass_groups(vs):
    """On a population of large sparse robots the autotuner's candidates for their size classes
    include the mass-sized groups (kind 5); whatever it picks, the run stays within the classes'
    admissible kinds and keeps the fitness finite."""
    pop = W.population_uneven(400, seed=80, sizes=(10, 12), occ=(0.2, 0.35))
    sim = vs.Simulator(W.CONFIG)
    sim.set_population_from(pop)
    kinds, _ = sim.autotune(20)
    sim.step(100)
    f = sim.fitness()
    sim.close()
    assert set(int(k) for k in kinds[6:9]) <= {1, 2, 4, 5}
    assert np.all(np.isfinite(f))


def test_eight_cube_instantiation_equals_the_generic_kernel(vs):
    """A population of 8 x 8 x 8 robots only runs the per-corner kernel's compile-time 8-cube
    instantiation; adding one robot of another grid sends the same robots through the generic
    one.  Their states and fitness agree bit for bit."""
    pop = W.population_bernoulli(24, (8, 8, 8), 0.8, seed=73)
    other = W.population_bernoulli(1, (5, 7, 6), 0.8, seed=74)
    both = W.make_population([tuple(d) for d in pop.dims] + [tuple(other.dims[0])],
                             [pop.grid(r) for r in range(pop.P)] + [other.grid(0)])
    a = run(vs, pop, W.CONFIG, 600, vs.LATTICE_CORNER)
    b = run(vs, both, W.CONFIG, 600, vs.LATTICE_CORNER)
    n = int(a[3][-1])
    assert np.array_equal(a[0], b[0][:n]) and np.array_equal(a[1], b[1][:n])
    assert np.array_equal(a[2], b[2][:pop.P])
