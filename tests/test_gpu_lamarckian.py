"""Gradient-assisted co-design: genome rows [w | kappa | phi] of per-voxel parameters on a fixed
morphology, the adjoint's gradient, and the Lamarckian step that moves chosen genomes uphill
before the unchanged genetic operators breed from them.

The step is checked against the FP64 oracle's adjoint (same rows, same step sizes and bounds,
within the gradient tolerance of the adjoint tests scaled by the step), rows outside the list
stay bitwise unchanged, and a small step raises the oracle's FP64 fitness of most robots."""
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


def make(P, dims, seed):
    rng = np.random.default_rng(seed)
    pop = W.population_uniform(P, dims, seed=seed)
    w, kappa, phi = W.voxel_params(rng, pop)
    V = int(np.prod(dims))
    rows = np.concatenate([w.reshape(P, V), kappa.reshape(P, V), phi.reshape(P, V)], axis=1)
    return pop, w, kappa, phi, np.ascontiguousarray(rows, dtype=np.float32)


def test_param_rows_mode_equals_params_mode(vs):
    import torch
    pop, w, kappa, phi, rows = make(10, (4, 3, 3), 80)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = []
    for mode, g in ((vs.MODE_PARAMS, (t(pop.mats), t(w), t(kappa), t(phi))),
                    (vs.MODE_PARAM_ROWS, (t(pop.mats), t(rows)))):
        sim = vs.Simulator(PHYS)
        sim.set_population(pop.dims, g, mode)
        sim.step(500)
        out.append((sim.state()[0], sim.fitness()))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    # host inputs take the same path
    sim = vs.Simulator(PHYS)
    sim.set_population(pop.dims, (pop.mats, rows), vs.MODE_PARAM_ROWS)
    sim.step(500)
    assert np.array_equal(sim.state()[0], out[0][0])
    sim.close()


def gpu_step(vs, pop, rows, nsteps, K, chosen, eta, bounds=None):
    import torch
    P, G = rows.shape
    V = G // 3
    sim = vs.Simulator(PHYS)
    sim.set_checkpointing(K)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = t(rows)
    sim.set_population(pop.dims, (t(pop.mats), g), vs.MODE_PARAM_ROWS)
    sim.step(nsteps)
    f = sim.fitness()
    dl = np.zeros(P)
    dl[chosen] = 1.0
    gw, gk, gp = (torch.empty(P * V, device="cuda") for _ in range(3))
    sim.backward(t(dl), gw, gk, gp)
    lo = hi = None
    if bounds is not None:
        lo, hi = t(bounds[0]), t(bounds[1])
    sim.evo_gradient_step(g, gw, gk, gp, eta, rows=chosen, lo=lo, hi=hi)
    torch.cuda.synchronize()
    grads = [a.cpu().numpy().reshape(P, V) for a in (gw, gk, gp)]
    sim.close()
    return f, g.cpu().numpy(), grads


def test_gradient_step_matches_oracle(vs, orc):
    dims, nsteps, K = (3, 3, 3), 300, 100
    pop, w, kappa, phi, rows = make(6, dims, 81)
    P, G = rows.shape
    V = G // 3
    chosen = [0, 2, 5]
    eta = (0.05, 2.0e3, 0.5)
    lo = np.array([0.0] * V + [0.0] * V + [-np.inf] * V, np.float32)
    hi = np.array([1.0] * V + [np.inf] * V + [np.inf] * V, np.float32)
    f, out, grads = gpu_step(vs, pop, rows, nsteps, K, chosen, eta, (lo, hi))
    for r in range(P):
        if r not in chosen:
            assert np.array_equal(out[r], rows[r])
            continue
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        _, rw, rk, rp = orc.adjoint(pop.grid(r), dims, PHYS, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        steps = np.concatenate([eta[0] * rw, eta[1] * rk, eta[2] * rp])
        expect = np.clip(rows[r].astype(np.float64) + steps, lo, hi)
        scale = np.concatenate([np.full(V, eta[0] * np.abs(rw).max()), np.full(V, eta[1] * np.abs(rk).max()),
                                np.full(V, eta[2] * np.abs(rp).max())])
        err = np.abs(out[r] - expect)
        assert np.all(err <= GRAD_TOL * scale + 2e-7 * np.abs(expect) + 1e-12), (r, err.max())
    # the bounds hold
    assert np.all(out[:, :V] >= 0.0) and np.all(out[:, :V] <= 1.0) and np.all(out[:, V:2 * V] >= 0.0)


def test_small_step_raises_fp64_fitness(vs, orc):
    dims, nsteps, K = (4, 4, 3), 400, 100
    pop, w, kappa, phi, rows = make(12, dims, 82)
    P, G = rows.shape
    V = G // 3
    # step sizes from a probe gradient: a parameter change of ~1 % of each segment's scale
    f0, _, grads = gpu_step(vs, pop, rows, nsteps, K, list(range(P)), (0.0, 0.0, 0.0))
    eta = (0.01 / max(np.abs(grads[0]).max(), 1e-30), 10.0 / max(np.abs(grads[1]).max(), 1e-30),
           0.01 / max(np.abs(grads[2]).max(), 1e-30))
    _, out, _ = gpu_step(vs, pop, rows, nsteps, K, list(range(P)), eta)
    up = 0
    for r in range(P):
        before, _ = orc.fitness_after(pop.grid(r), dims, PHYS, nsteps, rows[r, :V], rows[r, V:2 * V], rows[r, 2 * V:])
        after, _ = orc.fitness_after(pop.grid(r), dims, PHYS, nsteps, out[r, :V], out[r, V:2 * V], out[r, 2 * V:])
        up += after > before
    assert up >= 0.75 * P, up


def test_gradient_step_rejects_bad_arguments(vs):
    import torch
    pop, w, kappa, phi, rows = make(4, (3, 3, 3), 83)
    P, G = rows.shape
    sim = vs.Simulator(PHYS)
    g = torch.from_numpy(rows).cuda()
    sim.set_population(pop.dims, (pop.mats, rows), vs.MODE_PARAM_ROWS)
    gw = torch.zeros(P * (G // 3), device="cuda")
    with pytest.raises(vs.VoxsimError):
        sim.evo_gradient_step(g, gw, gw, gw, (1.0, 1.0, 1.0), rows=[0, 4])
    with pytest.raises(vs.VoxsimError):
        sim.evo_gradient_step(g[:, :-1].contiguous(), gw, gw, gw, (1.0, 1.0, 1.0))
    with pytest.raises(vs.VoxsimError):
        sim.evo_gradient_step(g, gw, gw, gw, (float("nan"), 1.0, 1.0))
    sim.close()
    # robots on different grid shapes cannot form genome rows
    mixed = W.population_uneven(4, seed=84, sizes=(2, 3))
    sim = vs.Simulator(PHYS)
    with pytest.raises(vs.VoxsimError):
        sim.set_population(mixed.dims, (mixed.mats, np.zeros((4, 81), np.float32)), vs.MODE_PARAM_ROWS)
    sim.close()


def test_lamarckian_loop(vs):
    import torch
    from paper_2405_00698_gb300 import codesign
    pop, w, kappa, phi, rows = make(16, (4, 4, 4), 85)
    P, G = rows.shape
    V = G // 3
    sim = vs.Simulator(PHYS)
    g = torch.from_numpy(rows).cuda()
    mats = torch.from_numpy(np.ascontiguousarray(pop.mats)).cuda()
    recs, final = codesign.run_lamarckian(sim, mats, g, (4, 4, 4), generations=3, steps=300,
                                          evo=W.Evolution(), eta=(0.02, 50.0, 0.1), checkpoint=100)
    sim.close()
    assert len(recs) == 3 and all(np.isfinite(r.best) for r in recs)
    # (the box holds right after the gradient step; the children's Gaussian mutation may leave it)
    out = final.cpu().numpy()
    assert np.all(np.isfinite(out)) and not np.array_equal(out, rows)


def test_elite_weights_follow_the_rank_order(vs):
    """evo_elite_weights marks the E best robots with finite fitness in evo_generation's order:
    fitness descending, ties by ascending index, NaN and -inf last (never elites)."""
    import torch
    from paper_2405_00698_gb300 import codesign
    rng = np.random.default_rng(86)
    f = np.round(rng.standard_normal(300), 1)
    f[[3, 17, 40]] = np.nan
    f[[5, 6]] = -np.inf
    f[[7]] = np.inf
    sim = vs.Simulator(PHYS)
    for E in (0, 1, 75, 298, 300):
        out = torch.full((300,), 7.0, dtype=torch.float64, device="cuda")
        sim.evo_elite_weights(torch.from_numpy(f).cuda(), E, out)
        torch.cuda.synchronize()
        want = np.zeros(300)
        for r in codesign.rank_order(f)[:E]:
            if np.isfinite(f[r]):
                want[r] = 1.0
        assert np.array_equal(out.cpu().numpy(), want), E
    with pytest.raises(vs.VoxsimError):
        sim.evo_elite_weights(torch.zeros(4, dtype=torch.float64, device="cuda"), 5,
                              torch.zeros(4, dtype=torch.float64, device="cuda"))
    sim.close()
