"""The benchmark's per-workload CPU baselines (the FP64 oracle simulating a sample of the uneven
population and of the large robots, all host cores) and the oracle's thread-count argument: a
count given to one call holds for that call only, so a single-threaded measurement does not leave
the next all-cores measurement single-threaded.  Both run without a GPU on small samples."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2405_00698_gb300 import workloads as W  # noqa: E402


def test_population_baseline_reports_a_rate_over_the_sample():
    pop = W.workload_uneven(4096, seed=2).subset(range(8))
    rec = bench.cpu_baseline_population(pop, 20, "the first 8 of the 4096 robots, 20 steps")
    assert rec["kind"] == "oracle" and rec["unit"] == "spring-updates/s"
    assert rec["value"] > 0 and 1 <= rec["cores"] <= pop.P
    assert rec["sample"].startswith("the first 8 of the 4096 robots, 20 steps; ")


def test_thread_count_holds_for_one_call_only():
    pop = W.population_uniform(4, (3, 3, 3), seed=5)
    default = O.run_population(pop, W.CONFIG, 5)["threads"]
    one = O.run_population(pop, W.CONFIG, 5, nthreads=1)
    after = O.run_population(pop, W.CONFIG, 5)
    assert one["threads"] == 1 and after["threads"] == default
    assert np.array_equal(one["fitness"], after["fitness"])
