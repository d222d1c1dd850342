"""Pins of three oracle functions that the invariants alone leave free: the stick / slip friction
law (Section II-C, Table II friction rows), the muscle actuation clock L(t) = L0 (1 + a sin(w t +
phi)) at t = n dt (Section II-A/II-C, Table II actuation rows), and the counter-based SplitMix64
generator of the evolutionary operators (Section II-C, Table I).  CPU only.

Each expected value comes from outside the oracle: a brute-force sum of Hooke forces over the 28
springs of one voxel, a forced linear recurrence iterated in numpy, and published SplitMix64
outputs.  A swapped mu_s / mu_k, a flipped slip direction, a wrong angular frequency or phase,
or an actuation clock off by one step fails one of them."""
import dataclasses
import itertools
import math

import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W

CONFIG = W.CONFIG


def one_voxel(mat):
    return np.full((1, 1, 1), mat, dtype=np.uint8)


def hooke_forces(x, x0, k):
    """Force on every corner of one voxel (8 corners, all 28 pairs joined by a spring of
    stiffness k and rest length = rest distance), by brute force over the pairs."""
    F = np.zeros_like(x)
    for i, j in itertools.combinations(range(8), 2):
        d = x[j] - x[i]
        l = np.linalg.norm(d)
        L0 = np.linalg.norm(x0[j] - x0[i])
        f = k * (l - L0) * d / l
        F[i] += f
        F[j] -= f
    return F


def sheared_cube(orc, phys, mat, shear, p, v0=(0.0, 0.0)):
    """A one-voxel cube whose bottom corners sit at z = -p (penetrating the ground) and whose top
    layer is shifted horizontally by `shear`; all corners start with horizontal velocity v0."""
    r = orc.Robot(one_voxel(mat), (1, 1, 1), phys)
    x0, _ = r.state()
    bottom = x0[:, 2] == 0.0
    x = x0.copy()
    x[:, 2] -= p
    x[~bottom, 0] += shear[0]
    x[~bottom, 1] += shear[1]
    v = np.zeros_like(x)
    v[:, 0], v[:, 1] = v0
    r.set_state(x, v, 0)
    return r, x0, x, v, bottom


def friction_expectation(phys, F, v, p, bottom, mu_s, mu_k, clamp):
    """One semi-implicit Euler step of every corner under the Coulomb stick / slip law written
    from its definition: below the ground the normal force k_g p is added; a corner sticks
    (horizontal force and velocity zeroed) when |F_h| <= mu_s F_n, else kinetic friction of
    magnitude mu_k F_n opposes F_h (with `clamp`, never more than |F_h|).  Returns the new
    velocities and the regime of every bottom corner."""
    m, dt, c = phys.mass, phys.dt, phys.damping
    Fn = phys.k_ground * p
    out = np.empty_like(v)
    regimes = {}
    for i in range(8):
        f = F[i].copy()
        f[2] -= m * phys.gravity
        vi = v[i].copy()
        if bottom[i]:
            f[2] += Fn
            fh = math.hypot(f[0], f[1])
            if fh <= mu_s * Fn:
                regimes[i] = ("stick", fh / Fn)
                f[:2] = 0.0
                vi[:2] = 0.0
            else:
                regimes[i] = ("slip", fh / Fn)
                kin = mu_k * Fn
                if clamp:
                    kin = min(kin, fh)
                f[:2] -= kin * f[:2] / fh
        out[i] = c * (vi + dt * f / m)
    return out, regimes


# shears of the top layer and target ratios |F_h| / F_n of the corner with the largest horizontal
# force: a ratio of 0.9 lies between mu_k = 0.8 and mu_s = 1.0 of the configurations (must stick;
# swapped coefficients would slip), 1.3 and 3 must slip with kinetic friction mu_k F_n
@pytest.mark.parametrize("shear", [(0.004, 0.0), (0.003, -0.002), (-0.0015, 0.0035)])
@pytest.mark.parametrize("ratio", [0.5, 0.9, 1.3, 3.0])
def test_friction_stick_and_slip_one_step(orc, shear, ratio):
    phys = CONFIG
    assert phys.mu_k < phys.mu_s
    mat = 4
    k = phys.k_mat[mat]
    # the sheared geometry does not depend on p, so the forces are fixed first and p chosen after
    r, x0, x, v, bottom = sheared_cube(orc, phys, mat, shear, 0.0)
    F = hooke_forces(x, x0, k)
    fh_max = max(math.hypot(*F[i, :2]) for i in range(8) if bottom[i])
    p = fh_max / (phys.k_ground * ratio)
    r, x0, x, v, bottom = sheared_cube(orc, phys, mat, shear, p)
    F = hooke_forces(x, x0, k)
    v1_ref, regimes = friction_expectation(phys, F, v, p, bottom, phys.mu_s, phys.mu_k, clamp=False)
    # keep clear of the threshold, where FP64 rounding of the two force sums could disagree
    assert all(abs(q - phys.mu_s) > 1e-6 for _, q in regimes.values())
    r.simulate(1)
    x1, v1 = r.state()
    for i, (kind, _) in regimes.items():
        if kind == "stick":                 # stuck corners keep their horizontal position exactly
            assert v1[i, 0] == 0.0 and v1[i, 1] == 0.0
            assert x1[i, 0] == x[i, 0] and x1[i, 1] == x[i, 1]
    assert np.allclose(v1, v1_ref, rtol=0, atol=1e-12)
    assert np.allclose(x1, x + phys.dt * v1_ref, rtol=0, atol=1e-14)
    kinds = {kind for kind, _ in regimes.values()}
    if ratio < phys.mu_s:
        assert "stick" in kinds
        if ratio > phys.mu_k:      # the band between the two coefficients sticks
            assert any(kind == "stick" and q > phys.mu_k for kind, q in regimes.values())
    else:
        assert "slip" in kinds


def test_friction_slip_direction_and_magnitude(orc):
    """A slipping corner loses exactly mu_k F_n along its horizontal force: the velocity change
    against the ground-free step is c dt mu_k F_n / m, antiparallel to F_h."""
    phys = CONFIG
    free = dataclasses.replace(phys, ground_on=False)
    shear, mat = (0.003, -0.002), 4
    r, x0, x, v, bottom = sheared_cube(orc, phys, mat, shear, 0.0)
    F = hooke_forces(x, x0, phys.k_mat[mat])
    fh = np.array([np.hypot(*F[i, :2]) for i in range(8)])
    p = fh[bottom].min() / (phys.k_ground * 2.5)          # every bottom corner slips
    a, *_ = sheared_cube(orc, phys, mat, shear, p)
    b, *_ = sheared_cube(orc, free, mat, shear, p)
    a.simulate(1); b.simulate(1)
    _, va = a.state()
    _, vb = b.state()
    Fn = phys.k_ground * p
    for i in np.nonzero(bottom)[0]:
        dv = va[i, :2] - vb[i, :2]
        u = F[i, :2] / fh[i]
        expect = -phys.damping * phys.dt * phys.mu_k * Fn / phys.mass * u
        assert np.allclose(dv, expect, rtol=0, atol=1e-12), i
    for i in np.nonzero(~bottom)[0]:
        assert np.array_equal(va[i], vb[i])


# ------------------------------------------------------------------------------------------
# Actuation clock: a driven breathing cube
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mat,w,phi", [(1, None, None), (2, None, None), (1, 0.7, 0.9), (2, 0.55, -2.3)])
def test_driven_breathing_cube_forced_recurrence(orc, mat, w, phi):
    """One muscle voxel, gravity and ground off.  All 28 springs share the same relative rest
    length 1 + a sin(w t + phi), so a uniform scaling about the centre stays a uniform scaling:
    with y = scale - 1 the corner equation is y'' = -(8 k / m)(y - a sin(w t + phi)).  Semi-implicit
    Euler with velocity damping c and the clock t_n = n dt turns it into the forced recurrence
        ydot_{n+1} = c (ydot_n - dt (8 k / m)(y_n - a sin(w n dt + phi))),  y_{n+1} = y_n + dt ydot_{n+1},
    w = 2 pi freq, which numpy iterates from rest.  The oracle's corners must follow
    x_n = centre + (1 + y_n)(x_0 - centre)."""
    phys = dataclasses.replace(CONFIG, gravity=0.0, ground_on=False)
    if w is None:
        r = orc.Robot(one_voxel(mat), (1, 1, 1), phys)
        k, a, ph = phys.k_mat[mat], phys.amp_mat[mat], phys.phase_mat[mat]
    else:
        kappa = phys.k_mat[mat]
        r = orc.Robot(one_voxel(mat), (1, 1, 1), phys, w=[w], kappa=[kappa], phi=[phi])
        k, a, ph = w * kappa, w * phys.amp_mat[mat], phi
    assert a > 0
    x0, _ = r.state()
    centre = x0.mean(axis=0)
    om0sq = 8.0 * k / phys.mass
    om = 2.0 * math.pi * phys.freq
    dt, c = phys.dt, phys.damping
    checks = {1, 2, 3, 10, 137, 1000, 2600}
    y, yd, done = 0.0, 0.0, 0
    for n in range(max(checks)):
        yd = c * (yd - dt * om0sq * (y - a * math.sin(om * n * dt + ph)))
        y = y + dt * yd
        if n + 1 in checks:
            r.simulate(n + 1 - done)
            done = n + 1
            x, _ = r.state()
            assert np.allclose(x, centre + (1.0 + y) * (x0 - centre), rtol=0, atol=1e-12), n + 1
    assert abs(y) > 1e-3, "the drive must move the cube"


def test_actuation_clock_starts_at_zero_and_counts_steps(orc):
    """Started at step n0 (set_state), the clock reads t = n0 dt: a cube restarted from the state
    of step 400 continues exactly as the uninterrupted run."""
    phys = dataclasses.replace(CONFIG, gravity=0.0, ground_on=False)
    a = orc.Robot(one_voxel(1), (1, 1, 1), phys)
    b = orc.Robot(one_voxel(1), (1, 1, 1), phys)
    a.simulate(400)
    xa, va = a.state()
    b.set_state(xa, va, 400)
    a.simulate(300); b.simulate(300)
    assert np.array_equal(a.state()[0], b.state()[0])
    c = orc.Robot(one_voxel(1), (1, 1, 1), phys)
    c.set_state(xa, va, 401)                 # one step late: a different drive
    c.simulate(300)
    assert np.abs(c.state()[0] - a.state()[0]).max() > 1e-9


# ------------------------------------------------------------------------------------------
# SplitMix64: published outputs
# ------------------------------------------------------------------------------------------

# The first five outputs of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) seeded with 0 and
# with 1234567: the generator's widely published reference values.
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                    0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
SPLITMIX64_SEED1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                          4593380528125082431, 16408922859458223821]


@pytest.mark.parametrize("seed,outputs", [(0, SPLITMIX64_SEED0), (1234567, SPLITMIX64_SEED1234567)])
def test_rng_draws_are_splitmix64_outputs(orc, seed, outputs):
    """The draw for counter n (generation, child, gene, purpose packed into n) is the high half
    of output number n of the SplitMix64 stream seeded with the seed; counters 0..4 are
    generation 0, child 0, gene 0 with purposes 0..4."""
    for n, out in enumerate(outputs):
        assert orc.rng_draw(seed, 0, 0, 0, n) == out >> 32, n


# Table II prints mu_s = 0.6 below mu_k = 1.0.  A corner with mu_s F_n < |F_h| < mu_k F_n then
# slips, and a kinetic friction of mu_k F_n would exceed the force it opposes and reverse it.
# The reading taken: kinetic friction removes at most |F_h| (the slipping corner keeps its
# velocity, the horizontal force drops to zero), i.e. F_h <- F_h - min(mu_k F_n, |F_h|) F_h / |F_h|.
@pytest.mark.parametrize("shear", [(0.004, 0.0), (0.003, -0.002)])
@pytest.mark.parametrize("ratio", [0.4, 0.8, 1.5])
def test_paper_friction_never_reverses_the_horizontal_force(orc, shear, ratio):
    phys = W.PAPER
    assert phys.mu_s < phys.mu_k
    mat = 4
    k = phys.k_mat[mat]
    v0 = (0.02, -0.01)      # a uniform drift: no dashpot force, but stick and slip differ
    r, x0, x, v, bottom = sheared_cube(orc, phys, mat, shear, 0.0, v0)
    F = hooke_forces(x, x0, k)
    fh_max = max(math.hypot(*F[i, :2]) for i in range(8) if bottom[i])
    p = fh_max / (phys.k_ground * ratio)
    r, x0, x, v, bottom = sheared_cube(orc, phys, mat, shear, p, v0)
    F = hooke_forces(x, x0, k)
    v1_ref, regimes = friction_expectation(phys, F, v, p, bottom, phys.mu_s, phys.mu_k, clamp=True)
    assert all(abs(q - phys.mu_s) > 1e-6 and abs(q - phys.mu_k) > 1e-6 for _, q in regimes.values())
    r.simulate(1)
    _, v1 = r.state()
    assert np.allclose(v1, v1_ref, rtol=0, atol=1e-12)
    for i, (kind, q) in regimes.items():
        dv = v1[i, :2] - v[i, :2]
        if kind == "slip":
            # the horizontal velocity change never points against the spring force
            assert dv @ F[i, :2] >= -1e-15
            if q < phys.mu_k:                    # saturated: no horizontal force at all
                assert np.array_equal(v1[i, :2], v[i, :2] * phys.damping)
