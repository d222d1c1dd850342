"""Whole-trajectory records (sim_set_trajectory_records): the forward keeps every step's record
in device memory (resident lattice and streamed robots) and the backward sweeps it without
replaying.
Against the checkpointed replay of the same run: the forward (fitness) and the contact modes are
bitwise the same, the gradients the same up to the order of the per-voxel atomic sums
(relative 1e-5 of the largest entry, as between checkpoint intervals); against the FP64
oracle's adjoint, 1e-3 as in the other adjoint tests.  Also: stepping that is not a recorded
call (the autotuner's trial runs) leaves a recorded run intact."""
import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PHYS = W.CONFIG
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(vs, pop, w, kappa, phi, nsteps, K, records, modes_of=(), dL=None, repeat=1, impose=None, **kw):
    import torch
    sim = vs.Simulator(PHYS, **kw)
    sim.set_checkpointing(K)
    sim.set_trajectory_records(records)
    sim.set_population(pop.dims, (_t(pop.mats), _t(w), _t(kappa), _t(phi)), vs.MODE_PARAMS)
    for r, m in (impose or {}).items():
        sim.impose_contact_modes(r, m)
    sim.step(nsteps)
    f = sim.fitness()
    modes = [sim.contact_modes(r, nsteps) for r in modes_of]
    outs = []
    for i in range(repeat):
        g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
        dl = np.ones(pop.P) if dL is None else dL
        sim.backward(_t(dl * (i + 1)), *g)
        torch.cuda.synchronize()
        outs.append([a.cpu().numpy() for a in g])
    sim.close()
    return f, outs, modes


def close(g, ref, tol=1e-5):
    return np.abs(g - ref).max() <= tol * max(np.abs(ref).max(), 1e-30)


@pytest.mark.parametrize("dims,nsteps,K", [((4, 4, 4), 300, 100), ((5, 3, 2), 257, 64), ((8, 8, 8), 200, 50)])
def test_records_equal_checkpointed_replay(vs, dims, nsteps, K):
    rng = np.random.default_rng(120)
    pop = W.population_bernoulli(5, dims, 0.8, seed=120)
    w, kappa, phi = W.voxel_params(rng, pop)
    fa, ga, ma = run(vs, pop, w, kappa, phi, nsteps, K, False, modes_of=(0, 4))
    fb, gb, mb = run(vs, pop, w, kappa, phi, nsteps, K, True, modes_of=(0, 4))
    assert np.array_equal(fa, fb)                     # recording does not change the forward run
    for x, y in zip(ma, mb):
        assert np.array_equal(x, y)                   # modes read from the records = replayed modes
        assert (x > 0).any()                          # the robots do touch the ground
    for x, y in zip(ga[0], gb[0]):
        assert close(y, x)


def test_records_match_oracle_adjoint(vs, orc):
    """The replay-free sweep over kept records, along the oracle run's contact modes, against
    the oracle's FP64 adjoint: every robot within the bar."""
    from tests.parity import oracle_corner_modes, robot_params
    rng = np.random.default_rng(121)
    dims, nsteps = (4, 4, 4), 350
    pop = W.population_uniform(4, dims, seed=121)
    w, kappa, phi = W.voxel_params(rng, pop)
    impose = {r: oracle_corner_modes(orc, pop.grid(r), dims, nsteps, robot_params(pop, r, w, kappa, phi))
              for r in range(pop.P)}
    _, g, _ = run(vs, pop, w, kappa, phi, nsteps, 100, True, impose=impose)
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        _, rw, rk, rp = orc.adjoint(pop.grid(r), dims, PHYS, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = [np.abs(x[a:b] - y).max() / max(np.abs(y).max(), 1e-30) for x, y in zip(g[0], (rw, rk, rp))]
        assert max(errs) <= GRAD_TOL, (r, errs)


def test_records_repeatable_and_mixed_with_streamed_robots(vs):
    """A population with lattice and streamed robots, both sweeping their records; a second
    backward on the same run gives the scaled gradient; both equal the all-checkpointed run."""
    rng = np.random.default_rng(122)
    shapes = ((3, 3, 3), (9, 9, 9), (4, 3, 2))
    pop = W.make_population(shapes, [W.bernoulli_grid(rng, d, 0.8) for d in shapes])
    w, kappa, phi = W.voxel_params(rng, pop)
    fa, ga, _ = run(vs, pop, w, kappa, phi, 180, 50, False)
    fb, gb, _ = run(vs, pop, w, kappa, phi, 180, 50, True, repeat=2)
    assert np.array_equal(fa, fb)
    for x, y in zip(ga[0], gb[0]):
        assert close(y, x)
    for g1, g2 in zip(gb[0], gb[1]):
        assert close(g2, 2.0 * g1)


def test_streamed_records_equal_checkpointed_replay(vs):
    """Robots on the streamed path keep their records too (written by the streamed step kernel
    during the forward run): the same forward, contact modes and gradients as the replay."""
    rng = np.random.default_rng(125)
    pop = W.population_bernoulli(3, (6, 5, 4), 0.8, seed=125)
    w, kappa, phi = W.voxel_params(rng, pop)
    fa, ga, ma = run(vs, pop, w, kappa, phi, 230, 60, False, modes_of=(0, 2), path=vs.PATH_STREAMED)
    fb, gb, mb = run(vs, pop, w, kappa, phi, 230, 60, True, modes_of=(0, 2), repeat=2, path=vs.PATH_STREAMED)
    assert np.array_equal(fa, fb)
    for x, y in zip(ma, mb):
        assert np.array_equal(x, y)
        assert (x > 0).any()
    for x, y in zip(ga[0], gb[0]):
        assert close(y, x)
    for g1, g2 in zip(gb[0], gb[1]):
        assert close(g2, 2.0 * g1)


def test_records_that_do_not_fit_fail_cleanly(vs):
    """Records of 100,000 steps of 512 robots 8x8x8 would need ~900 GB: sim_step_n fails with
    SIM_ENOMEM before stepping, no recorded run is left, and the context keeps working."""
    import torch
    pop = W.population_uniform(512, (8, 8, 8), seed=126)
    sim = vs.Simulator(PHYS)
    sim.set_checkpointing(100)
    sim.set_trajectory_records(True)
    sim.set_population_from(pop)
    with pytest.raises(vs.VoxsimError) as err:
        sim.step(100_000)
    assert err.value.status == vs.SIM_ENOMEM
    g = torch.empty(pop.mats.size, device="cuda")
    with pytest.raises(vs.VoxsimError):
        sim.backward(torch.ones(pop.P, dtype=torch.float64, device="cuda"), g, g, g)
    sim.set_trajectory_records(False)
    sim.step(50)
    f = sim.fitness()
    sim.close()
    ref = vs.Simulator(PHYS)
    ref.set_population_from(pop)
    ref.step(50)
    assert np.array_equal(f, ref.fitness())
    ref.close()


def test_switching_records_discards_the_recorded_run(vs):
    import torch
    pop = W.population_uniform(2, (3, 3, 3), seed=123)
    sim = vs.Simulator(PHYS)
    sim.set_checkpointing(10)
    sim.set_trajectory_records(True)
    sim.set_population_from(pop)
    sim.step(30)
    sim.set_trajectory_records(False)
    g = torch.empty(pop.mats.size, device="cuda")
    with pytest.raises(vs.VoxsimError):
        sim.backward(torch.ones(2, dtype=torch.float64, device="cuda"), g, g, g)
    sim.close()


@pytest.mark.parametrize("records", [False, True], ids=["checkpoints", "records"])
def test_autotune_leaves_a_recorded_run_intact(vs, records):
    """The autotuner's trial runs (longer than the recorded call) neither write checkpoints nor
    records: a backward after tuning gives the gradient of the recorded run (replayed from the
    checkpoints, as tuning rebuilt the routing).  Deterministic accumulation keeps every robot
    on the lattice kernels through the tuning."""
    import torch
    rng = np.random.default_rng(124)
    pop = W.population_uniform(3, (4, 4, 4), seed=124)
    w, kappa, phi = W.voxel_params(rng, pop)
    ref_f, ref_g, _ = run(vs, pop, w, kappa, phi, 60, 20, records, accumulate=vs.ACC_GATHER)
    sim = vs.Simulator(PHYS, accumulate=vs.ACC_GATHER)
    sim.set_checkpointing(20)
    sim.set_trajectory_records(records)
    sim.set_population(pop.dims, (_t(pop.mats), _t(w), _t(kappa), _t(phi)), vs.MODE_PARAMS)
    sim.step(60)
    f = sim.fitness()
    sim.autotune(200)
    g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
    sim.backward(_t(np.ones(pop.P)), *g)
    torch.cuda.synchronize()
    sim.close()
    assert np.array_equal(f, ref_f)
    for x, y in zip(ref_g[0], g):
        assert close(y.cpu().numpy(), x)
