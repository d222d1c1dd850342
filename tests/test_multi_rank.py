"""World-size-2 gloo run (CPU) of the sharded path's host logic: distinct shard seeds, contiguous
shard ranges, and the whole-job throughput = sum of units / max of times.  Each rank runs the
oracle on its own shard, as a GPU rank runs its own population."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as orc
        from paper_2405_00698_gb300 import shards, workloads as W
        r, w, _ = shards.env()
        seed = shards.shard_seed(7, r)
        pop = W.population_uniform(3, (3, 3, 3), seed=seed)
        res = orc.run_population(pop, W.CONFIG, 50)
        units = float(res["S"].sum()) * 50
        seconds = 0.5 + 0.25 * r                   # the slower rank decides the job time
        value, total_units, secs = shards.job_throughput(units, seconds)
        first, count = shards.shard_range(10, w, r)
        shards.barrier()
        out.put((r, seed, units, value, total_units, secs, first, count, res["fitness"].tolist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, u0, v0, t0, m0, f0, c0, fit0), (r1, s1, u1, v1, t1, m1, f1, c1, fit1) = got
    assert s0 != s1 and fit0 != fit1                 # distinct shards
    assert t0 == t1 == u0 + u1 and m0 == m1 == 0.75  # sum of units, max of times
    assert v0 == v1 and abs(v0 - (u0 + u1) / 0.75) < 1e-6
    assert (f0, c0, f1, c1) == (0, 5, 5, 5)


def test_shard_ranges_cover_exactly():
    from paper_2405_00698_gb300 import shards
    for total in (0, 1, 7, 1024, 4097):
        for world in (1, 2, 3, 8):
            spans = [shards.shard_range(total, world, r) for r in range(world)]
            assert sum(c for _, c in spans) == total
            assert all(spans[i][0] + spans[i][1] == spans[i + 1][0] for i in range(world - 1))


def _evolve_worker(rank, world, port, out):
    """One rank of the sharded co-design loop on the CPU: the oracle stands in for the rank's GPU
    (decode + simulation of its shard), the fitness all-gather is the exchange step, and the
    evolution runs replicated on the whole genome matrix."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        from paper_2405_00698_gb300 import shards
        genomes, history = _sharded_loop(rank, world, lambda f: shards.gather_population_fitness(f, world))
        out.put((rank, genomes.tobytes(), history))
    finally:
        dist.destroy_process_group()


P_ALL, GENS, NSTEPS, DIMS = 7, 2, 80, (3, 3, 2)


def _sharded_loop(rank, world, gather):
    import torch
    from oracle import oracle as orc
    from paper_2405_00698_gb300 import shards, workloads as W
    rng = np.random.default_rng(91)
    mats = [W.uniform_materials(rng, DIMS) for _ in range(P_ALL)]
    genomes = W.one_hot_logits(W.make_population([DIMS] * P_ALL, mats).mats).reshape(P_ALL, -1)
    genomes = (genomes + rng.normal(0, 0.3, genomes.shape)).astype(np.float32)
    evo = W.Evolution(seed=5)
    first, count = shards.shard_range(P_ALL, world, rank)
    history = []
    for gen in range(GENS):
        shard = genomes[first:first + count].reshape(count, -1, 5)
        pop = W.make_population([DIMS] * count, [np.argmax(g, axis=1).astype(np.uint8).reshape(DIMS[::-1])
                                                 for g in shard])
        fit_local = torch.from_numpy(orc.run_population(pop, W.CONFIG, NSTEPS)["fitness"])
        fit = gather(fit_local).numpy()
        history.append(fit.tolist())
        res = orc.evo_generation(fit, genomes, evo.elites(P_ALL), evo.seed, gen, evo.mut_threshold(), evo.sigma)
        genomes = res["genomes"].astype(np.float32)
    return genomes, history


def test_sharded_generations_equal_the_single_process_run():
    """Two ranks, each simulating its shard of one 7-robot population (shards of 4 and 3), with
    the fitness all-gather as the only exchange and replicated evolution: after two generations
    both ranks hold bitwise the genome matrix of the single-process run."""
    ref_genomes, ref_hist = _sharded_loop(0, 1, lambda f: f)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_evolve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, gbytes, hist in got:
        assert gbytes == ref_genomes.tobytes()
        assert hist == ref_hist
