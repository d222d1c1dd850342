"""The co-design loop with its hyper-parameter hook, the GPU diversity reductions against the
oracle's pairwise definitions, and the headless trajectory export."""
import dataclasses

import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W

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


def test_diversity_matches_oracle(vs, orc):
    import torch
    rng = np.random.default_rng(95)
    g = W.mlp_genomes(rng, 40)
    pop = W.population_uniform(40, (4, 4, 4), seed=95)
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    gd, md = sim.diversity(torch.from_numpy(g).cuda())
    kept = np.stack([orc.lcc(pop.grid(r), (4, 4, 4)) for r in range(pop.P)])
    assert abs(gd - orc.genome_diversity(g)) <= 1e-9 * orc.genome_diversity(g)
    assert abs(md - orc.morphology_diversity(kept)) <= 1e-12
    sim.close()


def test_codesign_loop_calls_the_hook_with_three_generations(vs):
    import torch
    from paper_2405_00698_gb300 import codesign
    rng = np.random.default_rng(96)
    P = 32
    genomes, B = W.mlp_genomes(rng, P), W.pe_matrix(rng)
    seen = []

    def hook(history, evo):
        seen.append([h.generation for h in history])
        return dataclasses.replace(evo, sigma=evo.sigma * 0.5)

    sim = vs.Simulator(PHYS)
    recs, final = codesign.run(sim, torch.from_numpy(genomes).cuda(), torch.from_numpy(B).cuda(), (4, 4, 4),
                               generations=5, steps=200, hook=hook)
    sim.close()
    assert [r.generation for r in recs] == [0, 1, 2, 3, 4]
    assert seen == [[0], [0, 1], [0, 1, 2], [1, 2, 3], [2, 3, 4]]
    assert abs(recs[-1].evolution.sigma - W.Evolution().sigma * 0.5 ** 4) < 1e-12
    for r in recs:
        assert np.isfinite(r.best) and r.genome_diversity > 0 and 0 <= r.morphology_diversity <= 1
    assert final.shape == (P, W.GENOME_LEN)


def test_stagnation_hook_rule(vs):
    from paper_2405_00698_gb300 import codesign
    evo = W.Evolution()
    mk = lambda g, b: codesign.GenerationRecord(g, b, 0, 0, 0, 1.0, 0.5, 0, evo)
    up = codesign.stagnation_hook([mk(0, 1.0), mk(1, 0.9), mk(2, 1.0)], evo)
    assert up.mut_rate == pytest.approx(0.15) and up.sigma == pytest.approx(0.075)
    down = codesign.stagnation_hook([mk(0, 1.0), mk(1, 1.1), mk(2, 1.2)], up)
    assert evo.mut_rate < down.mut_rate < up.mut_rate


def test_trajectory_export(vs, orc, tmp_path):
    from paper_2405_00698_gb300 import codesign
    pop = W.workload_small(seed=0).subset(range(3))
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    data = codesign.export_trajectory(sim, frames=4, steps_per_frame=50, path=str(tmp_path / "traj.npz"))
    sim.close()
    saved = np.load(tmp_path / "traj.npz")
    assert saved["positions"].shape[0] == 5 and np.array_equal(saved["positions"], data["positions"])
    ref = orc.run_population(pop, PHYS, 200, want_x=True)
    off = saved["offsets"]
    for r in range(pop.P):
        R = orc.Robot(pop.grid(r), (4, 4, 4), PHYS)
        x0, _ = R.state()
        assert np.allclose(saved["positions"][0][off[r]:off[r + 1]], x0, atol=1e-7)
        assert np.abs(saved["positions"][4][off[r]:off[r + 1]] - ref["x"][r]).max() < 1e-4 * 0.4
