"""The checkpointed adjoint (reverse-mode gradient of fitness with respect to the per-voxel
material weight, stiffness and actuation phase) against the FP64 oracle's adjoint and against
FP64 central finite differences of the oracle.

Tolerance: per robot, max_v |g_gpu - g_ref| <= 1e-3 * max_v |g_ref| for each parameter kind
(the float32 trajectory and the float32 reverse sweep against FP64); finite differences are
taken only where the +h and -h runs keep the same contact-mode sequence."""
import dataclasses

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


def gpu_grads(vs, pop, w, kappa, phi, nsteps, K, dL=None, phys=PHYS):
    import torch
    sim = vs.Simulator(phys)
    sim.set_checkpointing(K)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
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
    rng = np.random.default_rng(60)
    pop = W.population_uniform(6, dims, seed=60)
    w, kappa, phi = W.voxel_params(rng, pop)
    f, gw, gk, gp = gpu_grads(vs, pop, w, kappa, phi, nsteps, K)
    worst = []
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        fr, rw, rk, rp = orc.adjoint(pop.grid(r), dims, PHYS, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = (rel_grad_err(gw[a:b], rw), rel_grad_err(gk[a:b], rk), rel_grad_err(gp[a:b], rp))
        worst.append(max(errs))
    bad = [r for r, e in enumerate(worst) if e > GRAD_TOL]
    assert len(bad) <= 1, (bad, worst)


def test_adjoint_matches_fp64_finite_differences(vs, orc):
    """Central differences (h = 1e-6, FP64 oracle) on random parameters of a 4x4x4 population."""
    rng = np.random.default_rng(61)
    dims, nsteps = (4, 4, 4), 400
    pop = W.population_uniform(3, dims, seed=61)
    w, kappa, phi = W.voxel_params(rng, pop)
    _, gw, gk, gp = gpu_grads(vs, pop, w, kappa, phi, nsteps, 100)
    checked, failed = 0, []
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        kept = np.flatnonzero(orc.lcc(pop.grid(r), dims) > 0)
        base = {"w": w[a:b].astype(np.float64), "kappa": kappa[a:b].astype(np.float64),
                "phi": phi[a:b].astype(np.float64)}
        grads = {"w": gw[a:b], "kappa": gk[a:b], "phi": gp[a:b]}
        for name in ("w", "kappa", "phi"):
            for v in rng.choice(kept, 6, replace=False):
                h = 1e-6 * max(1.0, abs(base[name][v]))
                ap = base[name].copy(); ap[v] += h
                am = base[name].copy(); am[v] -= h
                fp, hp = orc.fitness_after(pop.grid(r), dims, PHYS, nsteps, **{**base, name: ap})
                fm, hm = orc.fitness_after(pop.grid(r), dims, PHYS, nsteps, **{**base, name: am})
                if hp != hm:
                    continue
                fd = (fp - fm) / (2 * h)
                scale = max(abs(fd), 1e-3 * np.abs(grads[name]).max())
                checked += 1
                if abs(grads[name][v] - fd) > GRAD_TOL * scale:
                    failed.append((r, name, int(v), float(grads[name][v]), fd))
    assert checked >= 20
    assert len(failed) <= checked // 20, failed


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
