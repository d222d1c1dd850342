"""Host-side logic on the CPU: the seeded workload generators keep the properties the workloads
are defined by (face-connected robots of the requested size, the uneven population's size and
occupancy ranges), population bookkeeping, the evolution thresholds, the stratified robot sample,
and the host ranking used to pick elite rows, which must agree with the oracle's rank order."""
import collections
import math

import numpy as np
import pytest

from paper_2405_00698_gb300 import codesign, workloads as W


def _face_connected(grid: np.ndarray) -> bool:
    occ = np.argwhere(grid > 0)
    if len(occ) == 0:
        return True
    seen = {tuple(occ[0])}
    todo = collections.deque([tuple(occ[0])])
    occupied = {tuple(p) for p in occ}
    while todo:
        k, j, i = todo.popleft()
        for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            q = (k + dk, j + dj, i + di)
            if q in occupied and q not in seen:
                seen.add(q)
                todo.append(q)
    return len(seen) == len(occupied)


@pytest.mark.parametrize("dims,occ", [((4, 4, 4), 0.3), ((6, 10, 4), 0.55), ((12, 12, 12), 0.9), ((1, 1, 5), 1.0)])
def test_connected_growth_size_connectivity_materials(dims, occ):
    rng = np.random.default_rng(1)
    for _ in range(5):
        g = W.connected_growth(rng, dims, occ)
        V = dims[0] * dims[1] * dims[2]
        assert g.shape == (dims[2], dims[1], dims[0])
        assert int((g > 0).sum()) == max(1, math.ceil(occ * V - 1e-9))
        assert _face_connected(g)
        assert set(np.unique(g[g > 0]).tolist()) <= {1, 2, 3, 4}


def test_uneven_population_ranges():
    pop = W.population_uneven(64, seed=2)
    assert pop.P == 64
    for r in range(pop.P):
        d = pop.dims[r]
        assert all(int(x) in (4, 6, 8, 10, 12) for x in d)
        g = pop.grid(r)
        V = g.size
        n = int((g > 0).sum())
        assert math.ceil(0.3 * V - 1e-9) <= n <= math.ceil(0.9 * V - 1e-9)
        assert _face_connected(g)
    # every size appears on some axis in a sample this large
    assert set(pop.dims.reshape(-1).tolist()) == {4, 6, 8, 10, 12}


def test_population_offsets_and_subset():
    rng = np.random.default_rng(3)
    shapes = [(2, 3, 4), (5, 1, 2), (3, 3, 3)]
    grids = [W.uniform_materials(rng, s) for s in shapes]
    pop = W.make_population(shapes, grids)
    assert pop.voxel_off.tolist() == [0, 24, 34, 61]
    for r, g in enumerate(grids):
        assert np.array_equal(pop.grid(r), g)
    sub = pop.subset([2, 0])
    assert sub.P == 2 and np.array_equal(sub.grid(0), grids[2]) and np.array_equal(sub.grid(1), grids[0])


def test_evolution_thresholds():
    e = W.Evolution()
    assert e.elites(1024) == 256 and e.elites(30) == 8 and e.elites(1) == 1
    assert W.PAPER_EVOLUTION.elites(30) == 9                 # ceil(0.3 * 30)
    assert e.mut_threshold() == int(0.1 * 2 ** 32)
    assert e.keep_threshold() == 0                          # crossover always
    assert W.PAPER_EVOLUTION.keep_threshold() == int(0.6 * 2 ** 32)
    assert W.Evolution(mut_rate=1.0).mut_threshold() == 2 ** 32 - 1
    assert W.Evolution(cross_rate=0.0).keep_threshold() == 2 ** 32 - 1


def test_stratified_subset_spans_the_counts():
    counts = np.array([50, 10, 40, 30, 20, 60, 5, 45])
    pick = W.stratified_subset(counts, 4)
    assert len(set(pick)) == 4
    assert int(np.argmin(counts)) in pick and int(np.argmax(counts)) in pick
    assert W.stratified_subset(counts, 100) == list(np.argsort(counts, kind="stable"))


def test_rank_order_matches_the_oracle(orc):
    rng = np.random.default_rng(4)
    f = rng.integers(-3, 4, size=40).astype(np.float64)     # many ties
    f[[3, 17]] = np.nan
    f[[5, 30]] = -np.inf
    order = codesign.rank_order(f)
    g = rng.standard_normal((40, 2)).astype(np.float32)
    ref = orc.evo_generation(f, g, 10, 1, 0, 0, 0.0)["order"]
    assert np.array_equal(order, ref)
    # descending fitness, index ascending on ties, NaN counted as -infinity
    key = np.where(np.isnan(f), -np.inf, f)
    for a, b in zip(order[:-1], order[1:]):
        assert key[a] > key[b] or (key[a] == key[b] and a < b)


def test_stagnation_hook():
    base = W.Evolution()
    rec = lambda best: codesign.GenerationRecord(0, best, 0.0, 0.0, 0, 0.0, 0.0, 0, base)
    up = codesign.stagnation_hook([rec(0.1), rec(0.2), rec(0.3)], base)
    assert up.mut_rate == pytest.approx(base.mut_rate) and up.sigma == pytest.approx(base.sigma)
    flat = codesign.stagnation_hook([rec(0.3), rec(0.2), rec(0.3)], base)
    assert flat.mut_rate == pytest.approx(1.5 * base.mut_rate) and flat.sigma == pytest.approx(1.5 * base.sigma)
    hot = W.Evolution(mut_rate=0.45, sigma=0.45)
    capped = codesign.stagnation_hook([rec(0.3)] * 3, hot)
    assert capped.mut_rate == 0.5 and capped.sigma == 0.5
    relaxed = codesign.stagnation_hook([rec(0.1), rec(0.2), rec(0.3)], hot)
    assert relaxed.mut_rate == pytest.approx(0.45 + 0.1 * (base.mut_rate - 0.45))
