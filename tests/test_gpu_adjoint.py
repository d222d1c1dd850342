"""The checkpointed adjoint (reverse-mode gradient of fitness with respect to the per-voxel
material weight, stiffness and actuation phase) against the FP64 oracle's adjoint and against
FP64 central finite differences of the oracle.

The gradient of a run with ground contact is the gradient of one piece of a piecewise-smooth
map: the stick / slip decisions select the piece.  The FP64 oracle decides them; its run's
contact modes are imposed on the GPU run (sim_impose_contact_modes), and the finite differences
are taken along the same modes, so both sides differentiate the same piece and no sample is
discarded.  Tolerance: per robot, max_v |g_gpu - g_ref| <= 1e-3 * max_v |g_ref| for each
parameter kind against the oracle's adjoint; per sample |g - fd| <= 1e-3 max(|fd|, 1e-3 max|g|)
against the differences."""
import dataclasses

import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W
from tests.parity import oracle_corner_modes, robot_params

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


def gpu_grads(vs, pop, w, kappa, phi, nsteps, K, dL=None, phys=PHYS, impose=None):
    """GPU fitness and gradients; impose: {robot: corner modes} imposed before stepping."""
    import torch
    sim = vs.Simulator(phys)
    sim.set_checkpointing(K)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
    for r, modes in (impose or {}).items():
        sim.impose_contact_modes(r, modes)
    sim.step(nsteps)
    f = sim.fitness()
    n = pop.mats.size
    gw = torch.empty(n, device="cuda"); gk = torch.empty_like(gw); gp = torch.empty_like(gw)
    dl = t(np.ones(pop.P) if dL is None else dL)
    sim.backward(dl, gw, gk, gp)
    torch.cuda.synchronize()
    sim.close()
    return f, gw.cpu().numpy(), gk.cpu().numpy(), gp.cpu().numpy()


def rel_grad_err(g, ref):
    scale = np.abs(ref).max()
    return float(np.abs(g - ref).max() / scale) if scale > 0 else float(np.abs(g).max())


@pytest.mark.parametrize("dims,nsteps,K", [((3, 3, 3), 350, 100), ((4, 4, 4), 500, 64), ((5, 3, 2), 200, 200)])
def test_adjoint_matches_oracle_adjoint(vs, orc, dims, nsteps, K):
    """Every robot's gradient, along the oracle run's contact modes, against the oracle's FP64
    adjoint of that run."""
    rng = np.random.default_rng(60)
    pop = W.population_uniform(6, dims, seed=60)
    w, kappa, phi = W.voxel_params(rng, pop)
    impose = {r: oracle_corner_modes(orc, pop.grid(r), dims, nsteps, robot_params(pop, r, w, kappa, phi))
              for r in range(pop.P)}
    f, gw, gk, gp = gpu_grads(vs, pop, w, kappa, phi, nsteps, K, impose=impose)
    worst = []
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        fr, rw, rk, rp = orc.adjoint(pop.grid(r), dims, PHYS, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = (rel_grad_err(gw[a:b], rw), rel_grad_err(gk[a:b], rk), rel_grad_err(gp[a:b], rp))
        worst.append(max(errs))
    assert max(worst) <= GRAD_TOL, worst


def test_adjoint_matches_fp64_finite_differences(vs, orc):
    """Central differences (h = 1e-6, FP64 oracle) along the oracle run's contact modes, on
    random parameters of a 4x4x4 population: every sample within the bar."""
    rng = np.random.default_rng(61)
    dims, nsteps = (4, 4, 4), 400
    pop = W.population_uniform(3, dims, seed=61)
    w, kappa, phi = W.voxel_params(rng, pop)
    bases = [robot_params(pop, r, w, kappa, phi) for r in range(pop.P)]
    impose = {r: oracle_corner_modes(orc, pop.grid(r), dims, nsteps, bases[r]) for r in range(pop.P)}
    _, gw, gk, gp = gpu_grads(vs, pop, w, kappa, phi, nsteps, 100, impose=impose)
    checked, failed = 0, []
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        kept = np.flatnonzero(orc.lcc(pop.grid(r), dims) > 0)
        base = bases[r]
        _, mass_modes, _ = orc.fitness_after_modes(pop.grid(r), dims, PHYS, nsteps, **base)
        grads = {"w": gw[a:b], "kappa": gk[a:b], "phi": gp[a:b]}
        for name in ("w", "kappa", "phi"):
            for v in rng.choice(kept, 6, replace=False):
                h = 1e-6 * max(1.0, abs(base[name][v]))
                ap = base[name].copy(); ap[v] += h
                am = base[name].copy(); am[v] -= h
                fp, _, _ = orc.fitness_after_modes(pop.grid(r), dims, PHYS, nsteps, force=mass_modes, **{**base, name: ap})
                fm, _, _ = orc.fitness_after_modes(pop.grid(r), dims, PHYS, nsteps, force=mass_modes, **{**base, name: am})
                fd = (fp - fm) / (2 * h)
                scale = max(abs(fd), 1e-3 * np.abs(grads[name]).max())
                checked += 1
                if abs(grads[name][v] - fd) > GRAD_TOL * scale:
                    failed.append((r, name, int(v), float(grads[name][v]), fd))
    assert checked == 54
    assert not failed, failed


def test_imposing_a_runs_own_modes_repeats_it_bit_for_bit(vs):
    """A run whose contact modes are imposed from its own recording takes the same steps."""
    import torch
    rng = np.random.default_rng(66)
    pop = W.population_uniform(5, (4, 4, 4), seed=66)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (t(pop.mats), t(w), t(kappa), t(phi))
    sim = vs.Simulator(PHYS)
    sim.set_checkpointing(100)
    sim.set_population(pop.dims, args, vs.MODE_PARAMS)
    sim.step(300)
    x_free, v_free, _ = sim.state()
    own = {r: sim.contact_modes(r, 300) for r in range(pop.P)}
    assert any((m != 0).any() for m in own.values())
    sim.set_population(pop.dims, args, vs.MODE_PARAMS)
    for r, m in own.items():
        sim.impose_contact_modes(r, m)
    sim.step(300)
    x_imp, v_imp, _ = sim.state()
    assert np.array_equal(x_free, x_imp) and np.array_equal(v_free, v_imp)
    sim.close()


def test_imposed_oracle_modes_follow_the_oracle_run(vs, orc):
    """With the oracle's modes imposed, the GPU trajectory stays within the position bar of the
    oracle's along the same modes, and a mode sequence that differs from the natural one (every
    contact held stuck) is followed too."""
    import torch
    from tests.parity import POS_TOL
    rng = np.random.default_rng(67)
    dims, n = (4, 4, 4), 600
    pop = W.population_uniform(3, dims, seed=67)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for variant in ("oracle", "stuck"):
        sim = vs.Simulator(PHYS)
        sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
        forced = {}
        for r in range(pop.P):
            base = robot_params(pop, r, w, kappa, phi)
            modes = oracle_corner_modes(orc, pop.grid(r), dims, n, base)
            if variant == "stuck":
                modes = np.where(modes != 0, 1, 0).astype(np.uint8)
            forced[r] = modes
            sim.impose_contact_modes(r, modes)
        sim.step(n)
        x, _, off = sim.state()
        sim.close()
        for r in range(pop.P):
            base = robot_params(pop, r, w, kappa, phi)
            R = orc.Robot(pop.grid(r), dims, PHYS, **base)
            R.simulate_modes(forced[r][:, R.topology()["mass_corner"]])
            ref, _ = R.state()                   # the oracle's final positions along the same modes
            xr = x[off[r]:off[r + 1]].astype(np.float64)
            err = np.abs(xr - ref).max() / (PHYS.edge * max(dims))
            assert err < POS_TOL, (variant, r, err)


def test_impose_contact_modes_rejects_bad_input(vs):
    import torch
    pop = W.population_uniform(2, (3, 3, 3), seed=68)
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    with pytest.raises(vs.VoxsimError):
        sim.impose_contact_modes(5, np.zeros((10, 64), np.uint8))         # robot out of range
    with pytest.raises(vs.VoxsimError):
        sim.impose_contact_modes(0, np.full((10, 64), 4, np.uint8))       # mode out of range
    sim.impose_contact_modes(0, np.zeros((10, 64), np.uint8))
    with pytest.raises(vs.VoxsimError):
        sim.impose_contact_modes(1, np.zeros((11, 64), np.uint8))         # another length
    sim.impose_contact_modes(None, None)
    sim.impose_contact_modes(1, np.zeros((11, 64), np.uint8))
    sim.close()
    damped = vs.Simulator(W.PAPER)
    damped.set_population_from(pop)
    with pytest.raises(vs.VoxsimError):
        damped.impose_contact_modes(0, np.zeros((10, 64), np.uint8))
    damped.close()


def test_checkpoint_interval_does_not_change_the_gradient(vs):
    rng = np.random.default_rng(62)
    pop = W.population_uniform(4, (4, 4, 4), seed=62)
    w, kappa, phi = W.voxel_params(rng, pop)
    ref = gpu_grads(vs, pop, w, kappa, phi, 300, 300)
    for K in (1, 37, 100):
        out = gpu_grads(vs, pop, w, kappa, phi, 300, K)
        assert np.array_equal(out[0], ref[0])
        for g, gr in zip(out[1:], ref[1:]):
            assert np.allclose(g, gr, rtol=1e-5, atol=1e-6 * np.abs(gr).max())


def test_adjoint_weighted_sum_is_linear(vs):
    """dL/df enters linearly: gradients of 2 f_0 - f_1 are 2 g_0 and -g_1 robot by robot."""
    rng = np.random.default_rng(63)
    pop = W.population_uniform(2, (3, 3, 3), seed=63)
    w, kappa, phi = W.voxel_params(rng, pop)
    _, g1, _, _ = gpu_grads(vs, pop, w, kappa, phi, 200, 50)
    _, g2, _, _ = gpu_grads(vs, pop, w, kappa, phi, 200, 50, dL=np.array([2.0, -1.0]))
    assert np.allclose(g2[:27], 2 * g1[:27], rtol=1e-5, atol=1e-9)
    assert np.allclose(g2[27:], -g1[27:], rtol=1e-5, atol=1e-9)


def test_autograd_function(vs, orc):
    import torch
    rng = np.random.default_rng(64)
    pop = W.population_uniform(3, (3, 3, 3), seed=64)
    w, kappa, phi = W.voxel_params(rng, pop)
    sim = vs.Simulator(PHYS)
    t = lambda a, g=False: torch.tensor(np.ascontiguousarray(a), device="cuda", requires_grad=g)
    W_, K_, F_ = t(w, True), t(kappa, True), t(phi, True)
    Fn = vs.fitness_function()
    f = Fn.apply(sim, pop.dims, t(pop.mats), W_, K_, F_, 300, 100)
    (f * torch.tensor([1.0, 0.5, -1.0], device="cuda", dtype=torch.float64)).sum().backward()
    for r, s in zip(range(3), (1.0, 0.5, -1.0)):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        _, rw, _, _ = orc.adjoint(pop.grid(r), (3, 3, 3), PHYS, 300, s, w[a:b], kappa[a:b], phi[a:b])
        assert rel_grad_err(W_.grad.cpu().numpy()[a:b], rw) < GRAD_TOL
    sim.close()


def test_backward_needs_a_recorded_run(vs):
    import torch
    sim = vs.Simulator(PHYS)
    pop = W.population_uniform(1, (2, 2, 2), seed=0)
    sim.set_population_from(pop)
    sim.step(10)
    g = torch.empty(8, device="cuda")
    with pytest.raises(vs.VoxsimError):
        sim.backward(torch.ones(1, dtype=torch.float64, device="cuda"), g, g, g)
    sim.close()
    with pytest.raises(vs.VoxsimError):
        vs.Simulator(PHYS, accumulate=vs.ACC_ATOMIC).set_checkpointing(10)


@pytest.mark.parametrize("path", [0, 2], ids=["lattice", "streamed"])
def test_backward_can_be_repeated_on_one_recorded_run(vs, path):
    """The checkpoints survive a backward pass: a second call on the same forward run with
    another dL/df gives the scaled gradient."""
    import torch
    rng = np.random.default_rng(65)
    pop = W.population_uniform(3, (4, 3, 3), seed=65)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim = vs.Simulator(PHYS, path=path)
    sim.set_checkpointing(40)
    sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
    sim.step(200)
    out = []
    for scale in (1.0, 3.0):
        g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
        sim.backward(t(np.full(pop.P, scale)), *g)
        torch.cuda.synchronize()
        out.append([a.cpu().numpy() for a in g])
    sim.close()
    for g1, g3 in zip(*out):       # float32 sums: linear up to rounding, relative to the largest entry
        assert np.abs(g3 - 3.0 * g1).max() <= 1e-5 * np.abs(g3).max()


def test_adjoint_through_saturated_slip(vs, orc):
    """Table II's friction order (mu_s = 0.6 < mu_k = 1.0) without dashpots: contact corners pass
    through saturated slip (the kinetic friction cancels the horizontal force), on the GPU as in
    the oracle; the gradient along the oracle's modes matches the oracle's adjoint."""
    phys = dataclasses.replace(PHYS, mu_s=0.6, mu_k=1.0)
    rng = np.random.default_rng(69)
    dims, nsteps = (4, 4, 4), 500
    pop = W.population_uniform(4, dims, seed=69)
    w, kappa, phi = W.voxel_params(rng, pop, phys)
    impose, saturated = {}, False
    for r in range(pop.P):
        modes = oracle_corner_modes(orc, pop.grid(r), dims, nsteps, robot_params(pop, r, w, kappa, phi), phys)
        saturated |= bool((modes == 3).any())
        impose[r] = modes
    assert saturated, "the runs must pass through saturated slip"
    f, gw, gk, gp = gpu_grads(vs, pop, w, kappa, phi, nsteps, 100, phys=phys, impose=impose)
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        fr, rw, rk, rp = orc.adjoint(pop.grid(r), dims, phys, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = (rel_grad_err(gw[a:b], rw), rel_grad_err(gk[a:b], rk), rel_grad_err(gp[a:b], rp))
        assert max(errs) <= GRAD_TOL, (r, errs)
        assert abs(f[r] - fr) <= 1e-3 * max(abs(fr), 1e-3 * phys.edge), (r, f[r], fr)
