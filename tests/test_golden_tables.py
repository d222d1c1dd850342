"""The paper's printed constants (tests/golden: Table I and Table II as printed) against the
presets the paper's own workload runs with (workloads.PAPER, workloads.PAPER_EVOLUTION) and the
material table they expand to (material ids: 0 empty, 1 expanding muscle, 2 contracting muscle,
3 soft tissue, 4 bone)."""
import math
import os

from paper_2405_00698_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                out[k] = [float(x) for x in v]
    return out


def test_table1_matches_paper_evolution_preset():
    t = table("table1_general_parameters.txt")
    e = W.PAPER_EVOLUTION
    assert e.mut_rate == t["mutation_rate"][0] and e.sigma == t["mutation_scale"][0]
    assert e.cross_rate == t["crossover_rate"][0] and e.elite_frac == t["elite_fraction"][0]
    P = int(t["population_size"][0])
    assert e.elites(P) == math.ceil(0.3 * 30 - 1e-9) == 9
    # crossover rate 0.4: 60 % of the children copy their first parent
    assert e.keep_threshold() == int(0.6 * 2 ** 32)
    assert e.mut_threshold() == int(0.1 * 2 ** 32)


def test_table2_matches_paper_physics_preset():
    t = table("table2_simulation_parameters.txt")
    p = W.PAPER
    assert p.gravity == t["gravity"][0] and p.mass == t["mass_per_index"][0]
    assert p.edge == t["rest_length"][0] and p.dt == t["time_step"][0]
    assert p.k_mat == (0.0, t["k_muscle"][0], t["k_muscle"][0], t["k_soft_tissue"][0], t["k_bone"][0])
    assert p.amp_mat[1] == p.amp_mat[2] == t["muscle_max_amplitude"][0] and p.amp_mat[3] == p.amp_mat[4] == 0.0
    assert p.phase_mat[2] == t["muscle_max_phase"][0] and p.phase_mat[1] == 0.0
    assert p.spring_zeta == t["spring_damping_ratio"][0] and p.ground_zeta == t["ground_damping_ratio"][0]
    assert p.k_ground == t["ground_elastic_coefficient"][0]
    assert p.mu_s == t["static_friction"][0] and p.mu_k == t["kinetic_friction"][0]
    assert p.damping == 1.0             # the table's damping is the dashpots, not a velocity factor
