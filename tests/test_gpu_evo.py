"""GPU vs oracle parity of one evolution generation, fed the same fitness vector and genomes.

Bit-exact: the rank order, the parent indices, the crossover masks, every gene that was not
mutated (a bitwise copy), and the set of mutated genes.  Mutated genes: the FP32 Box-Muller draw
vs the oracle's FP64 one, within 2e-6 absolute (sigma 0.05, |z| < 7)."""
import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    s = voxsim.Simulator(W.CONFIG)
    yield s
    s.close()


def gpu_generation(sim, f, g, evo, gen, inplace=False):
    import torch
    P, G = g.shape
    ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    gt = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    out = gt if inplace else torch.empty_like(gt)
    par = torch.empty((P, 2), dtype=torch.int32, device="cuda")
    mask = torch.empty((P, G), dtype=torch.uint8, device="cuda")
    sim.evo_generation(ft, gt, out, evo, gen, par, mask)
    torch.cuda.synchronize()
    return out.cpu().numpy(), par.cpu().numpy(), mask.cpu().numpy()


def check(orc, sim, f, g, evo, gen, inplace=False):
    P, G = g.shape
    out, par, mask = gpu_generation(sim, f, g, evo, gen, inplace)
    ref = orc.evo_generation(f, g, evo.elites(P), evo.seed, gen, evo.mut_threshold(), evo.sigma)
    assert np.array_equal(par, ref["parents"])
    E = evo.elites(P)
    assert np.array_equal(mask[E:], ref["mask"][E:])
    mut = ref["mutate"] == 1
    assert np.array_equal(out[~mut], ref["genomes"][~mut].astype(np.float32))
    assert np.abs(out[mut] - ref["genomes"][mut]).max(initial=0.0) < 2e-6
    return ref


def test_mlp_population_shape(orc, sim):
    rng = np.random.default_rng(40)
    P = 1024
    g = W.mlp_genomes(rng, P)
    f = rng.standard_normal(P)
    ref = check(orc, sim, f, g, W.Evolution(), 3)
    assert ref["mutate"].sum() > 0


def test_ties_nan_and_infinities(orc, sim):
    rng = np.random.default_rng(41)
    P, G = 37, 1001
    f = np.round(rng.standard_normal(P), 1)           # many exact ties
    f[[0, 5, 9]] = np.nan
    f[[1, 2]] = -np.inf
    f[3] = np.inf
    check(orc, sim, f, rng.standard_normal((P, G)).astype(np.float32), W.Evolution(seed=7), 11)


@pytest.mark.parametrize("frac", [1e-9, 1.0])
def test_extreme_elite_counts(orc, sim, frac):
    rng = np.random.default_rng(42)
    P, G = 20, 333
    evo = W.Evolution(elite_frac=frac)
    check(orc, sim, rng.standard_normal(P), rng.standard_normal((P, G)).astype(np.float32), evo, 0)


def test_in_place(orc, sim):
    rng = np.random.default_rng(43)
    P, G = 64, 777
    check(orc, sim, rng.standard_normal(P), rng.standard_normal((P, G)).astype(np.float32),
          W.Evolution(mut_rate=0.5), 100, inplace=True)


def test_single_robot_and_single_gene(orc, sim):
    rng = np.random.default_rng(44)
    check(orc, sim, rng.standard_normal(1), rng.standard_normal((1, 1)).astype(np.float32), W.Evolution(), 1)
    check(orc, sim, rng.standard_normal(9), rng.standard_normal((9, 1)).astype(np.float32), W.Evolution(), 2)


def test_direct_genome_generation_after_simulation(orc, sim):
    """The small workload: simulate, score, then evolve the one-hot material genomes."""
    from paper_2405_00698_gb300 import voxsim
    pop = W.workload_small(seed=0)
    s = voxsim.Simulator(W.CONFIG)
    s.set_population_from(pop)
    s.step(1000)
    f = s.fitness()
    s.close()
    g = W.one_hot_logits(pop.mats).reshape(pop.P, -1)
    check(orc, sim, f, g, W.Evolution(), 0)


def test_bad_arguments(sim):
    import torch
    from paper_2405_00698_gb300 import voxsim
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = torch.zeros((4, 8), device="cuda")
    with pytest.raises(voxsim.VoxsimError):
        sim.evo_generation(f, g, g, W.Evolution(), 1 << 19)


def test_evolution_from_the_host_uploaded_genomes(sim):
    """A population set from host MLP genomes evolves from the library's own device copy
    (genomes_in NULL): bit for bit the generation of the same genomes passed from the device.
    Without host genome rows, or with a size that does not match them, NULL is refused."""
    import torch
    from paper_2405_00698_gb300 import voxsim as vs
    rng = np.random.default_rng(17)
    P = 40
    genomes, B = W.mlp_genomes(rng, P), W.pe_matrix(rng)
    dims = np.tile(np.int32([4, 4, 4]), (P, 1))
    pinned = torch.from_numpy(genomes).pin_memory()
    sim.set_population(dims, pinned, vs.MODE_MLP, B=torch.from_numpy(B).pin_memory())
    f = torch.from_numpy(np.round(rng.standard_normal(P), 1)).cuda()
    evo = W.Evolution(seed=5)
    a = torch.empty((P, W.GENOME_LEN), device="cuda")
    sim.evo_generation(f, None, a, evo, 3)
    b = torch.empty_like(a)
    sim.evo_generation(f, torch.from_numpy(genomes).cuda(), b, evo, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(vs.VoxsimError):                   # size mismatch
        sim.evo_generation(f[:20], None, a[:20], evo, 3)
    sim.set_population(dims, torch.from_numpy(genomes).cuda(), vs.MODE_MLP, B=torch.from_numpy(B).cuda())
    with pytest.raises(vs.VoxsimError):                   # device genomes: no library copy
        sim.evo_generation(f, None, a, evo, 3)
