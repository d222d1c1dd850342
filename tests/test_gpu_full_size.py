"""Parity at the full workload sizes, in the launch configurations bench.py times, on sampled
robots the FP64 oracle recomputes one by one:

* 1024 MLP genomes on 8x8x8 grids, decode + 10,000 steps in one call (one lattice launch);
* 4096 uneven robots after the autotuner's choices, 5000 steps;
* 64 robots of 40x40x40 on the streamed path (one graph-captured launch per step), the first
  1000 steps of the 5000-step run;
* the adjoint of 512 robots of 8x8x8 with checkpoints every 100, along the FP64 oracle's
  contact modes (imposed on the sampled robots), at 500 steps and at the stated 2000 steps.

Robots are sampled evenly over the spring-count order.  The simulation is compared from the
GPU's own decoded grid and weights (the decode is checked separately on the same genomes).

The stated bar (positions 1e-4 of the robot size, fitness 1e-3) is checked after the first 1000
steps (a call boundary changes nothing: the state is carried over exactly).  After 5000 or
10,000 steps nearly every robot has crossed stick/slip switches whose outcome float32 rounding
decides, and the FP64 oracle itself, started 1e-7 m away (the float32 resolution of the
positions, the size of the perturbation each float32 step makes), moves by more than the bar;
there every robot must lie within that envelope of the oracle (tests/parity.py)."""
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


def test_mlp_population_full_size(vs, orc):
    import torch
    G, B = W.workload_mlp()
    P, N, dims = G.shape[0], 10000, (8, 8, 8)
    sim = vs.Simulator(PHYS)
    sim.set_population(np.tile(np.int32(dims), (P, 1)), torch.from_numpy(G).cuda(), vs.MODE_MLP,
                       B=torch.from_numpy(B).cuda())
    vox = sim.voxels()
    M, S = sim.counts()
    sim.step(1000)
    f1 = sim.fitness()
    x1, _, off = sim.state()
    sim.step(N - 1000)
    f = sim.fitness()
    x, _, off = sim.state()
    sim.close()
    # the stated bar after 1000 steps on 48 robots spread over the spring-count order (about 6 %
    # of them cross a stick/slip switch within float32 rounding and are held to the oracle's own
    # spread instead; a sample of 12 can hold two of them), the long run on 12 of those
    pick48 = W.stratified_subset(S, 48)
    pick = pick48[::4]
    # decode: exact outside the guard band of the oracle's FP64 scores
    for g in pick48:
        mat, w, logits, guard = orc.mlp_query(dims, B, G[g])
        got = vox["decoded"][g * 512:(g + 1) * 512]
        top = np.sort(logits[:, :5], axis=1)
        sure = (top[:, -1] - top[:, -2]) > 2 * guard
        assert np.array_equal(got[sure], mat[sure]), g
    # simulation of the GPU's decoded robots
    def decoded(picks):
        pop = W.make_population([dims] * len(picks), [vox["decoded"][g * 512:(g + 1) * 512].reshape(8, 8, 8)
                                                       for g in picks])
        w = np.concatenate([vox["w"][g * 512:(g + 1) * 512] for g in picks]).astype(np.float64)
        return pop, w, np.asarray(PHYS.k_mat)[pop.mats], np.asarray(PHYS.phase_mat)[pop.mats]
    pop48, w, kappa, phi = decoded(pick48)
    offs = np.concatenate([[0], np.cumsum([off[g + 1] - off[g] for g in pick48])])
    ref1 = orc.run_population(pop48, PHYS, 1000, w=w, kappa=kappa, phi=phi, want_x=True)
    assert np.array_equal(ref1["S"], S[pick48]) and np.array_equal(ref1["M"], M[pick48])
    x1s = np.concatenate([x1[off[g]:off[g + 1]] for g in pick48])
    check_population(orc, pop48, PHYS, 1000, f1[pick48], x1s, offs, ref1, w=w, kappa=kappa, phi=phi)
    pop, w, kappa, phi = decoded(pick)
    offs = np.concatenate([[0], np.cumsum([off[g + 1] - off[g] for g in pick])])
    ref = orc.run_population(pop, PHYS, N, w=w, kappa=kappa, phi=phi, want_x=True)
    xs = np.concatenate([x[off[g]:off[g + 1]] for g in pick])
    check_population(orc, pop, PHYS, N, f[pick], xs, offs, ref, w=w, kappa=kappa, phi=phi, K=8,
                     max_sensitive_frac=1.0, perturb=1e-7, envelope=2.0)


def test_uneven_population_full_size(vs, orc):
    pop = W.workload_uneven()
    N = 5000
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    sim.autotune(20)
    sim.step(1000)
    f1 = sim.fitness()
    x1, _, off = sim.state()
    sim.step(N - 1000)
    f = sim.fitness()
    x, _, off = sim.state()
    M, S = sim.counts()
    sim.close()
    pick = W.stratified_subset(S, 16)
    sub = pop.subset(pick)
    offs = np.concatenate([[0], np.cumsum([off[g + 1] - off[g] for g in pick])])
    ref1 = orc.run_population(sub, PHYS, 1000, want_x=True)
    assert np.array_equal(ref1["S"], S[pick])
    x1s = np.concatenate([x1[off[g]:off[g + 1]] for g in pick])
    check_population(orc, sub, PHYS, 1000, f1[pick], x1s, offs, ref1)
    ref = orc.run_population(sub, PHYS, N, want_x=True)
    xs = np.concatenate([x[off[g]:off[g + 1]] for g in pick])
    check_population(orc, sub, PHYS, N, f[pick], xs, offs, ref, K=8, max_sensitive_frac=1.0, perturb=1e-7,
                     envelope=2.0)


def test_large_robots_full_size_sample(vs, orc):
    pop = W.workload_large()
    N = 1000
    sim = vs.Simulator(PHYS)
    sim.set_population_from(pop)
    sim.step(N)
    f = sim.fitness()
    x, _, off = sim.state()
    M, S = sim.counts()
    sim.close()
    pick = W.stratified_subset(S, 2)
    sub = pop.subset(pick)
    ref = orc.run_population(sub, PHYS, N, want_x=True)
    assert np.array_equal(ref["S"], S[pick])
    xs = np.concatenate([x[off[g]:off[g + 1]] for g in pick])
    offs = np.concatenate([[0], np.cumsum([off[g + 1] - off[g] for g in pick])])
    check_population(orc, sub, PHYS, N, f[pick], xs, offs, ref, K=2)


def test_trajectory_records_full_size(vs):
    """The adjoint with every step's record kept in device memory (the bench's second adjoint
    line: 512 robots 8x8x8, 2000 steps, 17.9 GB of records, no replay) against the checkpointed
    replay of the same run: the forward runs agree bitwise, the gradients up to the order of the
    per-voxel atomic sums (1e-5 of the largest entry)."""
    import torch
    rng = np.random.default_rng(3)
    P, N, K = 512, 2000, 100
    pop = W.population_uniform(P, (8, 8, 8), seed=3)
    w, kappa, phi = W.voxel_params(rng, pop)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = []
    for records in (False, True):
        sim = vs.Simulator(PHYS)
        sim.set_checkpointing(K)
        sim.set_trajectory_records(records)
        sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
        sim.step(N)
        f = sim.fitness()
        g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
        sim.backward(t(np.ones(P)), *g)
        torch.cuda.synchronize()
        out.append((f, [a.cpu().numpy() for a in g]))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    for x, y in zip(out[0][1], out[1][1]):
        assert np.abs(y - x).max() <= 1e-5 * np.abs(x).max()


def _oracle_run(args):
    """The oracle's FP64 run of one robot: its contact modes (mass order), mass corners and adjoint."""
    from oracle import oracle as o
    grid, base, n = args
    _, modes, _ = o.fitness_after_modes(grid, (8, 8, 8), PHYS, n, **base)
    _, gw, gk, gp = o.adjoint(grid, (8, 8, 8), PHYS, n, **base)
    mc = o.Robot(grid, (8, 8, 8), PHYS, **base).topology()["mass_corner"]
    return modes, mc, {"w": gw, "kappa": gk, "phi": gp}


def _fd_along(args):
    """FP64 central difference of the fitness along imposed contact modes."""
    from oracle import oracle as o
    grid, base, name, v, h, modes, n = args
    ap = dict(base); ap[name] = base[name].copy(); ap[name][v] += h
    am = dict(base); am[name] = base[name].copy(); am[name][v] -= h
    fp, _, _ = o.fitness_after_modes(grid, (8, 8, 8), PHYS, n, force=modes, **ap)
    fm, _, _ = o.fitness_after_modes(grid, (8, 8, 8), PHYS, n, force=modes, **am)
    return (fp - fm) / (2 * h)


def adjoint_along_oracle_modes(vs, orc, N, n_robots=8, n_params=32, K=100):
    """The differentiation workload (512 robots 8x8x8, per-voxel w, kappa, phi, checkpoints every
    K): the FP64 oracle runs n_robots robots sampled over the spring-count order, its contact
    modes are imposed on those robots of the GPU run, and the GPU gradient is compared with
    (a) FP64 central differences (h = 1e-6) along the same modes on n_params random parameters
    per robot: |g - fd| / max(|fd|, 1e-3 max|g|) per sample, and (b) the oracle's FP64 adjoint:
    max |g - g_ref| / max |g_ref| per robot and parameter kind.  Returns both error lists."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    rng = np.random.default_rng(3)
    P = 512
    pop = W.population_uniform(P, (8, 8, 8), seed=3)
    w, kappa, phi = W.voxel_params(rng, pop)
    S = np.array([orc.Robot(pop.grid(r), (8, 8, 8), PHYS).S for r in range(P)])
    picks = W.stratified_subset(S, n_robots)
    bases = {}
    for r in picks:
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        bases[r] = {"w": w[a:b].astype(np.float64), "kappa": kappa[a:b].astype(np.float64),
                    "phi": phi[a:b].astype(np.float64)}
    with cf.ProcessPoolExecutor(max_workers=16, mp_context=mp.get_context("spawn")) as ex:
        runs = dict(zip(picks, ex.map(_oracle_run, [(pop.grid(r), bases[r], N) for r in picks])))
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        sim = vs.Simulator(PHYS)
        sim.set_checkpointing(K)
        sim.set_population(pop.dims, (t(pop.mats), t(w), t(kappa), t(phi)), vs.MODE_PARAMS)
        for r in picks:
            modes, mc, _ = runs[r]
            corner_modes = np.zeros((N, 729), np.uint8)
            corner_modes[:, mc] = modes
            sim.impose_contact_modes(r, corner_modes)
        sim.step(N)
        g = [torch.empty(pop.mats.size, device="cuda") for _ in range(3)]
        sim.backward(t(np.ones(P)), *g)
        torch.cuda.synchronize()
        g = dict(zip(("w", "kappa", "phi"), (a.cpu().numpy().astype(np.float64) for a in g)))
        sim.close()
        pick_rng = np.random.default_rng(44)
        jobs, meta, adj_err = [], [], []
        for r in picks:
            a = pop.voxel_off[r]
            modes, _, ref = runs[r]
            for name in ("w", "kappa", "phi"):
                gr = g[name][a:a + 512]
                adj_err.append(float(np.abs(gr - ref[name]).max() / np.abs(ref[name]).max()))
            kept = np.flatnonzero(orc.lcc(pop.grid(r), (8, 8, 8)) > 0)
            for _ in range(n_params):
                name = ("w", "kappa", "phi")[pick_rng.integers(3)]
                v = int(pick_rng.choice(kept))
                h = 1e-6 * max(1.0, abs(bases[r][name][v]))
                jobs.append((pop.grid(r), bases[r], name, v, h, modes, N))
                meta.append((a, name, v))
        fds = list(ex.map(_fd_along, jobs))
    fd_err = []
    for (a, name, v), fd in zip(meta, fds):
        gr = g[name][a:a + 512]
        fd_err.append(abs(gr[v] - fd) / max(abs(fd), 1e-3 * np.abs(gr).max()))
    return np.asarray(fd_err), np.asarray(adj_err)


def test_adjoint_full_population_500_steps(vs, orc):
    """The whole differentiation population at a 500-step horizon, along the oracle's contact
    modes: at least 95 % of 256 sampled parameters within 1e-3 of the FP64 differences, and every
    sampled robot's gradient within 1e-3 of the oracle's adjoint (max norm per kind)."""
    fd_err, adj_err = adjoint_along_oracle_modes(vs, orc, 500)
    assert np.mean(fd_err <= 1e-3) >= 0.95, np.sort(fd_err)[-8:]
    assert adj_err.max() <= 1e-3, adj_err


def test_adjoint_full_size_meets_the_stated_bar(vs, orc):
    """The differentiation workload as stated (512 robots 8x8x8, 2000 steps, checkpoints every
    100), along the oracle's contact modes, held to the stated bar: at least 95 % of 256 sampled
    parameters within 1e-3 of the FP64 differences (measured 96.9 %, median 1.4e-5, 95th
    percentile 3.8e-4).  It holds because the step's constants (dt, dt / m, m g, the damping) are
    carried past float32: rounded to float32 they shift the map itself by up to 3e-8 of each
    constant, which alone left 91 % of the samples within 1e-3."""
    fd_err, adj_err = adjoint_along_oracle_modes(vs, orc, 2000)
    print(f"within 1e-3: {np.mean(fd_err <= 1e-3):.3f} of {fd_err.size}; quantiles 50/90/95/100 %: "
          f"{np.quantile(fd_err, [0.5, 0.9, 0.95, 1.0])}; adjoint max-norm errors {np.sort(adj_err)[-3:]}")
    assert np.mean(fd_err <= 1e-3) >= 0.95
