"""The adjoint of robots too large for one SM (the streamed path: state, records and adjoints in
device memory, one launch per reverse step) against the FP64 oracle's adjoint, and against the
resident lattice adjoint on robots both paths can run.  Checkpointing moves robots that would
run on the atomic kernel to the deterministic streamed path.

Tolerance as in the resident adjoint tests: per robot and parameter kind,
max |g_gpu - g_ref| <= 1e-3 max |g_ref|."""
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


def grads(vs, pop, w, kappa, phi, nsteps, K, **kw):
    import torch
    sim = vs.Simulator(PHYS, **kw)
    sim.set_checkpointing(K)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
    sim.step(nsteps)
    f = sim.fitness()
    n = pop.mats.size
    g = [torch.empty(n, device="cuda") for _ in range(3)]
    sim.backward(t(np.ones(pop.P)), *g)
    torch.cuda.synchronize()
    sim.close()
    return f, [a.cpu().numpy() for a in g]


def rel(g, ref):
    scale = np.abs(ref).max()
    return float(np.abs(g - ref).max() / scale) if scale > 0 else float(np.abs(g).max())


def test_streamed_adjoint_equals_resident_adjoint(vs):
    rng = np.random.default_rng(90)
    pop = W.population_uniform(6, (4, 4, 3), seed=90)
    w, kappa, phi = W.voxel_params(rng, pop)
    fa, ga = grads(vs, pop, w, kappa, phi, 350, 100)
    fb, gb = grads(vs, pop, w, kappa, phi, 350, 100, path=vs.PATH_STREAMED)
    assert np.array_equal(fa, fb)                       # the forward runs agree bitwise
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        for x, y in zip(ga, gb):
            assert rel(y[a:b], x[a:b]) < 1e-4


@pytest.mark.parametrize("dims,nsteps,K", [((10, 9, 8), 240, 100), ((12, 12, 6), 150, 64)])
def test_large_robot_adjoint_matches_oracle(vs, orc, dims, nsteps, K):
    rng = np.random.default_rng(91)
    pop = W.population_bernoulli(2, dims, 0.8, seed=91)
    w, kappa, phi = W.voxel_params(rng, pop)
    f, g = grads(vs, pop, w, kappa, phi, nsteps, K)
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        fr, rw, rk, rp = orc.adjoint(pop.grid(r), dims, PHYS, nsteps, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = (rel(g[0][a:b], rw), rel(g[1][a:b], rk), rel(g[2][a:b], rp))
        assert max(errs) <= GRAD_TOL, (r, errs)


def test_mixed_population_adjoint(vs, orc):
    """Lattice and streamed robots in one population: each robot's gradient from its own path."""
    rng = np.random.default_rng(92)
    pop = W.make_population([(3, 3, 3), (9, 9, 9), (4, 3, 2)],
                            [W.bernoulli_grid(rng, d, 0.8) for d in ((3, 3, 3), (9, 9, 9), (4, 3, 2))])
    w, kappa, phi = W.voxel_params(rng, pop)
    f, g = grads(vs, pop, w, kappa, phi, 200, 50)
    for r in range(pop.P):
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        fr, rw, rk, rp = orc.adjoint(pop.grid(r), pop.dims[r], PHYS, 200, 1.0, w[a:b], kappa[a:b], phi[a:b])
        errs = (rel(g[0][a:b], rw), rel(g[1][a:b], rk), rel(g[2][a:b], rp))
        assert max(errs) <= GRAD_TOL, (r, errs)


def test_checkpointing_routes_atomic_robots_to_the_streamed_path(vs):
    """A 12x12x12 robot fits one SM's shared memory and runs on the atomic kernel by default;
    with checkpointing on it runs streamed (deterministic), and turning it off again restores
    the atomic route."""
    pop = W.population_bernoulli(2, (12, 12, 12), 0.7, seed=93)
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    sim.step(5)
    _, launches_atomic = sim.timing()
    sim.set_checkpointing(20)
    sim.step(40)
    _, launches_streamed = sim.timing()
    assert launches_streamed >= 40                    # one launch per step
    sim.set_checkpointing(0)
    sim.step(40)
    _, launches_back = sim.timing()
    assert launches_back < 40
    sim.close()


def test_forty_cube_adjoint_equals_the_generic_kernel(vs):
    """The streamed adjoint's compile-time 40 x 40 x 40 instantiation against the generic kernel
    (one robot of another grid added): the forward runs agree bitwise, the gradients up to the
    order of the per-voxel atomic sums."""
    rng = np.random.default_rng(91)
    dims = [(40, 40, 40)]
    g40 = [W.bernoulli_grid(rng, dims[0], 0.7)]
    extra = W.bernoulli_grid(rng, (26, 22, 24), 0.7)
    pop = W.make_population(dims, g40)
    both = W.make_population(dims + [(26, 22, 24)], g40 + [extra])
    w, kappa, phi = W.voxel_params(rng, both)
    n = pop.mats.size
    fa, ga = grads(vs, pop, w[:n], kappa[:n], phi[:n], 120, 50, path=vs.PATH_STREAMED)
    fb, gb = grads(vs, both, w, kappa, phi, 120, 50, path=vs.PATH_STREAMED)
    assert np.array_equal(fa, fb[:1])
    for x, y in zip(ga, gb):
        assert rel(y[:n], x) < 1e-5
