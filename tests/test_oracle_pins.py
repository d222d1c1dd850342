"""Pins of the FP64 oracle against facts fixed outside it: closed forms, invariants, library
routines and brute force.  CPU only."""
import dataclasses
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2405_00698_gb300 import workloads as W

PHYS = W.CONFIG
FREE = dataclasses.replace(PHYS, gravity=0.0, ground_on=False, damping=1.0)


def full_grid(nx, ny, nz, mat=3):
    return np.full((nz, ny, nx), mat, dtype=np.uint8)


# ------------------------------------------------------------------------------------------
# Topology: brute-force counts and closed forms
# ------------------------------------------------------------------------------------------

def test_one_voxel_counts(orc):
    r = orc.Robot(full_grid(1, 1, 1), (1, 1, 1), PHYS)
    assert (r.M, r.S) == (8, 28)
    t = r.topology()
    L = np.sort(t["L0"])
    s = PHYS.edge
    assert np.allclose(L[:12], s) and np.allclose(L[12:24], s * math.sqrt(2)) and np.allclose(L[24:], s * math.sqrt(3))


def test_two_voxels_face_adjacent(orc):
    r = orc.Robot(full_grid(2, 1, 1), (2, 1, 1), PHYS)
    assert (r.M, r.S) == (12, 50)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (4, 4, 4), (3, 5, 2), (8, 8, 8)])
def test_full_grid_closed_form(orc, dims):
    nx, ny, nz = dims
    r = orc.Robot(full_grid(*dims), dims, PHYS)
    M = (nx + 1) * (ny + 1) * (nz + 1)
    edges = nx * (ny + 1) * (nz + 1) + ny * (nx + 1) * (nz + 1) + nz * (nx + 1) * (ny + 1)
    faces = 2 * (nx * ny * (nz + 1) + nx * nz * (ny + 1) + ny * nz * (nx + 1))
    S = edges + faces + 4 * nx * ny * nz
    assert (r.M, r.S) == (M, S)
    if nx == ny == nz:
        n = nx
        assert S == 3 * n * (n + 1) ** 2 + 6 * n * n * (n + 1) + 4 * n ** 3


def test_spring_order_and_params(orc):
    rng = np.random.default_rng(3)
    g = W.uniform_materials(rng, (4, 3, 5))
    r = orc.Robot(g, (4, 3, 5), PHYS)
    t = r.topology()
    a, b = t["a"].astype(np.int64), t["b"].astype(np.int64)
    assert np.all(a < b)
    key = a * (r.M + 1) + b
    assert np.all(np.diff(key) > 0), "springs sorted by (a, b) and unique"
    assert np.all(np.diff(t["mass_corner"]) > 0)
    # the stiffness of a spring lies between the smallest and largest material stiffness
    kept = t["kept"]
    ks = np.asarray(PHYS.k_mat)[kept[kept > 0]]
    assert t["k"].min() >= ks.min() - 1e-9 and t["k"].max() <= ks.max() + 1e-9


def test_homogeneous_material_spring_params(orc):
    """A single-material robot has every spring at that material's stiffness, whatever the
    number of voxels sharing the spring (mean of equal values)."""
    rng = np.random.default_rng(4)
    g = (rng.random((4, 4, 4)) < 0.7).astype(np.uint8) * 4
    r = orc.Robot(g, (4, 4, 4), PHYS)
    t = r.topology()
    assert np.allclose(t["k"], PHYS.k_mat[4], rtol=0, atol=1e-9)
    assert np.all(t["alpha"] == 0) and np.all(t["beta"] == 0)


def test_muscle_actuation_coefficients(orc):
    """A single expanding-muscle voxel: alpha = amplitude, beta = 0; contracting: alpha = -amp."""
    for mat, sign in ((1, 1.0), (2, -1.0)):
        r = orc.Robot(full_grid(1, 1, 1, mat), (1, 1, 1), PHYS)
        t = r.topology()
        assert np.allclose(t["alpha"], sign * PHYS.amp_mat[mat], atol=1e-15)
        assert np.allclose(t["beta"], 0.0, atol=1e-15)


# ------------------------------------------------------------------------------------------
# Largest connected component: library routine and exhaustive small cases
# ------------------------------------------------------------------------------------------

def scipy_lcc(grid):
    """Largest face-connected component by scipy.ndimage.label (labels follow C-order scan, so a
    lower label holds a smaller linear index); ties keep the lowest label."""
    lab, n = ndi.label(grid > 0, structure=ndi.generate_binary_structure(3, 1))
    if n == 0:
        return np.zeros_like(grid)
    sizes = np.bincount(lab.reshape(-1), minlength=n + 1)[1:]
    best = int(np.argmax(sizes)) + 1
    return np.where(lab == best, grid, 0).astype(np.uint8)


def test_lcc_all_2x2x2(orc):
    for bits in range(256):
        g = np.array([(bits >> i) & 1 for i in range(8)], dtype=np.uint8).reshape(2, 2, 2) * 3
        ref = scipy_lcc(g).reshape(-1)
        assert np.array_equal(orc.lcc(g, (2, 2, 2), "bfs"), ref), bits
        assert np.array_equal(orc.lcc(g, (2, 2, 2), "uf"), ref), bits


@pytest.mark.parametrize("seed", range(6))
def test_lcc_random(orc, seed):
    rng = np.random.default_rng(100 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 13, 3))
    g = W.bernoulli_grid(rng, dims, float(rng.uniform(0.2, 0.6)))
    ref = scipy_lcc(g).reshape(-1)
    assert np.array_equal(orc.lcc(g, dims, "bfs"), ref)
    assert np.array_equal(orc.lcc(g, dims, "uf"), ref)


def test_lcc_tie_keeps_smallest_index(orc):
    g = np.zeros((1, 1, 5), np.uint8)
    g[0, 0, 0] = 2; g[0, 0, 1] = 2; g[0, 0, 3] = 4; g[0, 0, 4] = 4
    out = orc.lcc(g, (5, 1, 1))
    assert list(out) == [2, 2, 0, 0, 0]


# ------------------------------------------------------------------------------------------
# Integrator and force law: closed forms
# ------------------------------------------------------------------------------------------

def test_breathing_cube_discrete_closed_form(orc):
    """A one-voxel cube (one material, no actuation, no gravity, no ground, no damping) scaled
    about its centre by (1 + eps) stays a uniform scaling: every spring force is
    k (lambda - 1) (q0 - p0), and the corner equation is lambda'' = -(8 k / m)(lambda - 1).
    Semi-implicit Euler maps y = lambda - 1 by a linear map of determinant 1 whose rotation angle
    satisfies cos(theta) = 1 - (omega dt)^2 / 2, so y_n = eps cos(n theta) + b sin(n theta) with
    b = -eps (omega dt)^2 / (2 sin theta)."""
    r = orc.Robot(full_grid(1, 1, 1, 3), (1, 1, 1), FREE)
    x0, _ = r.state()
    c = x0.mean(axis=0)
    eps = 0.01
    r.set_state(c + (1 + eps) * (x0 - c), np.zeros_like(x0), 0)
    k, m, dt = FREE.k_mat[3], FREE.mass, FREE.dt
    h = math.sqrt(8 * k / m) * dt
    theta = math.acos(1 - h * h / 2)
    b = -eps * h * h / (2 * math.sin(theta))
    for n in (1, 7, 100, 1000):
        r.simulate(n - (0 if n == 1 else prev))
        prev = n
        x, _ = r.state()
        y = eps * math.cos(n * theta) + b * math.sin(n * theta)
        assert np.allclose(x, c + (1 + y) * (x0 - c), rtol=0, atol=1e-13), n


@pytest.mark.parametrize("damping", [1.0, 0.999])
def test_free_fall(orc, damping):
    """A passive robot with no ground falls as a rigid body: v_n = -g dt c (1 - c^n) / (1 - c)
    (or -g dt n for c = 1) and x_n = x_0 + dt * sum_{i<=n} v_i."""
    phys = dataclasses.replace(PHYS, ground_on=False, damping=damping)
    rng = np.random.default_rng(5)
    g = (rng.random((3, 3, 3)) < 0.8).astype(np.uint8) * 4
    r = orc.Robot(g, (3, 3, 3), phys)
    x0, _ = r.state()
    N = 500
    r.simulate(N)
    x, v = r.state()
    gdt = phys.gravity * phys.dt
    idx = np.arange(1, N + 1)
    vs = -gdt * idx if damping == 1.0 else -gdt * damping * (1 - damping ** idx) / (1 - damping)
    assert np.allclose(v[:, 2], vs[-1], rtol=1e-9, atol=1e-12)
    assert np.allclose(v[:, :2], 0.0, atol=1e-10)
    assert np.allclose(x[:, 2], x0[:, 2] + phys.dt * vs.sum(), rtol=0, atol=1e-10)
    if damping == 1.0:
        assert np.allclose(x[:, 2], x0[:, 2] - gdt * phys.dt * N * (N + 1) / 2, atol=1e-10)


def test_momentum_and_centroid_conserved_with_actuation(orc):
    """Internal central forces (springs, actuated) conserve momentum: with gravity, ground and
    damping off the centroid stays put and the fitness is 0."""
    rng = np.random.default_rng(6)
    g = W.uniform_materials(rng, (4, 4, 4))
    r = orc.Robot(g, (4, 4, 4), FREE)
    x0, _ = r.state()
    for _ in range(4):
        r.simulate(250)
        x, v = r.state()
        assert np.allclose(v.sum(axis=0) * FREE.mass, 0.0, atol=1e-12)
        assert np.allclose(x.mean(axis=0), x0.mean(axis=0), atol=1e-13)
    assert abs(r.fitness()) < 1e-13
    assert np.abs(x - x0).max() > 1e-4, "actuation must move the masses"


def test_energy_no_secular_drift(orc):
    """Passive robot, everything dissipative off, random initial velocities: the symplectic
    integrator keeps the energy within a bounded band, with no drift over 1e5 steps."""
    rng = np.random.default_rng(7)
    g = full_grid(2, 1, 1, 4)
    r = orc.Robot(g, (2, 1, 1), FREE)
    t = r.topology()
    x0, _ = r.state()
    v0 = rng.normal(0, 0.05, x0.shape)
    v0 -= v0.mean(axis=0)
    r.set_state(x0, v0, 0)

    def energy():
        x, v = r.state()
        d = x[t["b"]] - x[t["a"]]
        l = np.linalg.norm(d, axis=1)
        return 0.5 * FREE.mass * (v * v).sum() + 0.5 * (t["k"] * (l - t["L0"]) ** 2).sum()

    E = [energy()]
    for _ in range(100):
        r.simulate(1000)
        E.append(energy())
    E = np.asarray(E)
    assert np.abs(E - E[0]).max() / E[0] < 0.05
    assert abs(E[-20:].mean() - E[:20].mean()) / E[0] < 0.01


def test_mirror_symmetric_robot_has_zero_fitness(orc):
    """A robot mirror-symmetric in x with the same actuation on both sides keeps its centroid
    x fixed (ground and friction included): fitness 0."""
    rng = np.random.default_rng(8)
    half = W.uniform_materials(rng, (2, 4, 3))
    half[:, :, 1] = np.maximum(half[:, :, 1], 3)   # keep the halves connected across the plane
    g = np.concatenate([half, half[:, :, ::-1]], axis=2)
    r = orc.Robot(g, (4, 4, 3), PHYS)
    r.simulate(300)
    assert abs(r.fitness()) < 1e-9


def test_translation_invariance(orc):
    rng = np.random.default_rng(9)
    g = W.uniform_materials(rng, (4, 4, 4))
    a = orc.Robot(g, (4, 4, 4), PHYS)
    b = orc.Robot(g, (4, 4, 4), PHYS)
    x0, v0 = b.state()
    b.set_state(x0 + np.array([0.25, -0.5, 0.0]), v0, 0)
    a.simulate(200); b.simulate(200)
    # fitness is measured from the built pose, so the shifted copy reads the 0.25 m offset too
    assert abs(a.fitness() - (b.fitness() - 0.25)) < 1e-9
    xa, _ = a.state(); xb, _ = b.state()
    assert np.allclose(xa + np.array([0.25, -0.5, 0.0]), xb, atol=1e-9)


def test_resting_cube_penetration(orc):
    """A one-voxel bone cube settles on the ground; at rest the ground carries the weight:
    sum over the four bottom corners of k_g (-z) = 8 m g."""
    r = orc.Robot(full_grid(1, 1, 1, 4), (1, 1, 1), PHYS)
    r.simulate(20000)
    x, v = r.state()
    bottom = x[:, 2] < PHYS.edge / 2
    assert bottom.sum() == 4
    load = (PHYS.k_ground * -x[bottom, 2]).sum()
    assert abs(load - 8 * PHYS.mass * PHYS.gravity) / (8 * PHYS.mass * PHYS.gravity) < 1e-3
    assert np.abs(v).max() < 1e-4


# ------------------------------------------------------------------------------------------
# Encoding: Eq. (1) special cases, bf16 rounding vs torch, MLP vs numpy matmul
# ------------------------------------------------------------------------------------------

def np_round_bf16(x):
    """Round float64 values to bfloat16 by integer arithmetic on the float64 bit pattern:
    bfloat16 keeps 7 of float64's 52 stored mantissa bits, so 45 bits go, ties to even."""
    x = np.asarray(x, dtype=np.float64)
    b = x.view(np.uint64).copy()
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    b = b + np.uint64((1 << 44) - 1) + lsb
    b &= ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


def test_bf16_rounding_matches_torch_for_float32(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    xs = np.concatenate([rng.standard_normal(2000), rng.uniform(-1e-3, 1e-3, 500),
                         [0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    ref = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([orc.round_bf16(float(v)) for v in xs])
    assert np.array_equal(got, ref)
    assert np.array_equal(np_round_bf16(xs.astype(np.float64)), ref)


def test_bf16_rounding_double_inputs(orc):
    rng = np.random.default_rng(11)
    xs = rng.standard_normal(5000) * np.exp(rng.uniform(-20, 20, 5000))
    got = np.array([orc.round_bf16(float(v)) for v in xs])
    assert np.array_equal(got, np_round_bf16(xs))


def test_pe_zero_matrix(orc):
    out = orc.pe_table((3, 2, 4), np.zeros((128, 3), np.float32))
    assert np.all(out[:, :128] == 1.0) and np.all(out[:, 128:] == 0.0)


def test_pe_matches_numpy(orc):
    rng = np.random.default_rng(12)
    B = W.pe_matrix(rng)
    dims = (8, 8, 8)
    out = orc.pe_table(dims, B)
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    v = np.stack([(i + 0.5) / 8, (j + 0.5) / 8, (k + 0.5) / 8], axis=-1).reshape(-1, 3)
    proj = 2 * np.pi * (v @ B.astype(np.float64).T)
    assert np.allclose(out, np.concatenate([np.cos(proj), np.sin(proj)], axis=1), atol=1e-12)


def numpy_mlp(dims, B, genome):
    """The same MLP from numpy matmuls with bf16 rounding at the operand points."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.stack([(i + 0.5) / nx, (j + 0.5) / ny, (k + 0.5) / nz], axis=-1).reshape(-1, 3)
    proj = 2 * np.pi * (v @ B.astype(np.float64).T)
    g = np_round_bf16(np.concatenate([np.cos(proj), np.sin(proj)], axis=1))
    w = genome.astype(np.float64)
    W1 = np_round_bf16(w[:16384].reshape(64, 256)); b1 = w[16384:16448]
    W2 = np_round_bf16(w[16448:20544].reshape(64, 64)); b2 = w[20544:20608]
    W3 = np_round_bf16(w[20608:20992].reshape(6, 64)); b3 = w[20992:]
    h1 = np_round_bf16(np.maximum(g @ W1.T + b1, 0))
    h2 = np_round_bf16(np.maximum(h1 @ W2.T + b2, 0))
    return h2 @ W3.T + b3


def test_mlp_matches_numpy(orc):
    rng = np.random.default_rng(13)
    genomes, B = W.mlp_genomes(rng, 3), W.pe_matrix(rng)
    for g in genomes:
        mat, w, logits, guard = orc.mlp_query((8, 8, 8), B, g)
        ref = numpy_mlp((8, 8, 8), B, g)
        # different summation order can flip a bf16 rounding of h1 / h2; the guard bounds it
        assert np.all(np.abs(logits - ref).max(axis=1) <= guard + 1e-12)
        top = np.sort(ref[:, :5], axis=1)
        sure = (top[:, -1] - top[:, -2]) > 2 * guard
        assert np.array_equal(mat[sure], np.argmax(ref[sure, :5], axis=1))
        assert sure.mean() > 0.8
        assert np.allclose(w, 1 / (1 + np.exp(-logits[:, 5])), rtol=1e-14)


def test_mlp_zero_weights_ties(orc):
    g = np.zeros(20998, np.float32)
    g[20992:20998] = [0.5, 0.5, 0.5, 0.5, 0.5, 0.0]
    mat, w, logits, _ = orc.mlp_query((2, 2, 2), W.pe_matrix(np.random.default_rng(0)), g)
    assert np.all(mat == 0) and np.allclose(w, 0.5)
    g[20992 + 3] = 0.75
    mat, _, _, _ = orc.mlp_query((2, 2, 2), np.zeros((128, 3), np.float32), g)
    assert np.all(mat == 3)


# ------------------------------------------------------------------------------------------
# Evolution
# ------------------------------------------------------------------------------------------

def test_rng_statistics(orc):
    n = 200000
    u = np.array([orc.rng_draw(77, 3, c, j, 2) for c, j in zip(range(n), range(n))], dtype=np.float64)
    # 32-bit uniform: mean 2^31, every top-byte bucket populated evenly
    assert abs(u.mean() / 2 ** 32 - 0.5) < 5 * math.sqrt(1 / 12 / n)
    counts = np.bincount((u.astype(np.uint64) >> np.uint64(24)).astype(np.int64), minlength=256)
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # independent streams per purpose / gene
    v = np.array([orc.rng_draw(77, 3, c, c, 3) for c in range(n)], dtype=np.float64)
    assert abs(np.corrcoef(u, v)[0, 1]) < 5 / math.sqrt(n)


def test_evo_generation_semantics(orc):
    rng = np.random.default_rng(14)
    P, G = 64, 2000
    f = rng.standard_normal(P)
    f[5] = np.nan; f[9] = -np.inf; f[10] = f[11] = f[12] = 0.25
    genomes = rng.standard_normal((P, G)).astype(np.float32)
    evo = W.Evolution()
    E = evo.elites(P)
    assert E == 16
    out = orc.evo_generation(f, genomes, E, 99, 4, evo.mut_threshold(), evo.sigma)
    key = np.where(np.isnan(f), -np.inf, f)
    assert np.array_equal(out["order"], np.argsort(-key, kind="stable"))
    elite = out["order"][:E]
    assert np.array_equal(out["genomes"][:E].astype(np.float32), genomes[elite])
    assert np.all(np.isin(out["parents"][E:], elite))
    ch = out["genomes"][E:]
    pa, pb = genomes[out["parents"][E:, 0]], genomes[out["parents"][E:, 1]]
    src = np.where(out["mask"][E:] == 1, pa, pb).astype(np.float64)
    mut = out["mutate"][E:] == 1
    assert np.array_equal(ch[~mut], src[~mut])
    d = (ch - src)[mut]
    n = mut.sum()
    assert abs(mut.mean() - evo.mut_rate) < 5 * math.sqrt(0.09 / mut.size)
    assert abs(out["mask"][E:].mean() - 0.5) < 5 * math.sqrt(0.25 / mut.size)
    assert abs(d.std() - evo.sigma) < 5 * evo.sigma / math.sqrt(2 * n)
    assert abs(d.mean()) < 5 * evo.sigma / math.sqrt(n)
    # parents spread over all elites
    counts = np.bincount(np.searchsorted(np.sort(elite), out["parents"][E:].reshape(-1)), minlength=E)
    assert counts.min() > 0


def test_evo_deterministic(orc):
    rng = np.random.default_rng(15)
    f = rng.standard_normal(32); g = rng.standard_normal((32, 100)).astype(np.float32)
    a = orc.evo_generation(f, g, 8, 1, 0, 429496729, 0.05)
    b = orc.evo_generation(f, g, 8, 1, 0, 429496729, 0.05)
    c = orc.evo_generation(f, g, 8, 1, 1, 429496729, 0.05)
    assert np.array_equal(a["genomes"], b["genomes"])
    assert not np.array_equal(a["mask"], c["mask"])


# ------------------------------------------------------------------------------------------
# Adjoint: central finite differences of the oracle's own forward
# ------------------------------------------------------------------------------------------

def _fd_check(orc, mat, dims, phys, nsteps, w, kappa, phi, samples, h_rel=1e-6, tol=1e-5):
    f, gw, gk, gp = orc.adjoint(mat, dims, phys, nsteps, 1.0, w, kappa, phi)
    grads = {"w": gw, "kappa": gk, "phi": gp}
    base = {"w": w, "kappa": kappa, "phi": phi}
    checked = 0
    for name, v in samples:
        arr = base[name]
        h = h_rel * max(1.0, abs(arr[v]))
        ap = arr.copy(); ap[v] += h
        am = arr.copy(); am[v] -= h
        kw = dict(base); kw[name] = ap
        fp, hp = orc.fitness_after(mat, dims, phys, nsteps, **kw)
        kw[name] = am
        fm, hm = orc.fitness_after(mat, dims, phys, nsteps, **kw)
        if hp != hm:
            continue
        fd = (fp - fm) / (2 * h)
        g = grads[name][v]
        scale = max(abs(fd), 1e-3 * max(np.abs(grads[name]).max(), 1e-30))
        assert abs(g - fd) <= tol * scale + 1e-12, (name, v, g, fd)
        checked += 1
    return checked


def test_adjoint_smooth_case_matches_fd(orc):
    """No ground and no gravity: the map is smooth everywhere.  With no external force the
    centroid never moves, so the pin uses a general terminal loss L = sum_i c_i . x_i(N)."""
    rng = np.random.default_rng(16)
    dims = (3, 3, 3)
    mat = W.uniform_materials(rng, dims)
    mat[1, 1, 1] = 1
    V = mat.size
    w = rng.uniform(0.5, 1.0, V); kappa = np.asarray(PHYS.k_mat)[mat.reshape(-1)] * rng.uniform(0.8, 1.2, V)
    phi = np.asarray(PHYS.phase_mat)[mat.reshape(-1)] + rng.uniform(-0.5, 0.5, V)
    phys = dataclasses.replace(PHYS, ground_on=False, gravity=0.0, damping=0.9995)
    N = 300
    M = orc.Robot(mat, dims, phys).M
    cvec = rng.standard_normal((M, 3))
    _, gw, gk, gp = orc.adjoint(mat, dims, phys, N, 0.0, w, kappa, phi, lx_final=cvec)
    grads = {"w": gw, "kappa": gk, "phi": gp}
    base = {"w": w, "kappa": kappa, "phi": phi}

    def loss(**kw):
        r = orc.Robot(mat, dims, phys, **kw)
        r.simulate(N)
        return float((r.state()[0] * cvec).sum())

    occ = np.flatnonzero(orc.lcc(mat, dims) > 0)
    for name in ("w", "kappa", "phi"):
        for v in rng.choice(occ, 6, replace=False):
            h = 1e-6 * max(1.0, abs(base[name][v]))
            ap = base[name].copy(); ap[v] += h
            am = base[name].copy(); am[v] -= h
            fd = (loss(**{**base, name: ap}) - loss(**{**base, name: am})) / (2 * h)
            g = grads[name][v]
            scale = max(abs(fd), 1e-3 * np.abs(grads[name]).max())
            assert abs(g - fd) <= 1e-6 * scale, (name, v, g, fd)
    assert np.abs(gp).max() > 0 and np.abs(gw).max() > 0


def test_adjoint_with_contact_matches_fd(orc):
    """Ground and friction on; samples whose contact-mode sequence changes between +h and -h
    are discarded (the map is not differentiable across a mode switch)."""
    rng = np.random.default_rng(17)
    mat = W.uniform_materials(rng, (3, 3, 3))
    mat[0, :, :] = np.maximum(mat[0, :, :], 1)
    V = mat.size
    w = rng.uniform(0.5, 1.0, V); kappa = np.asarray(PHYS.k_mat)[mat.reshape(-1)].astype(float)
    phi = np.asarray(PHYS.phase_mat)[mat.reshape(-1)] + rng.uniform(-0.5, 0.5, V)
    occ = np.flatnonzero(orc.lcc(mat, (3, 3, 3)) > 0)
    samples = [(n, int(v)) for n in ("w", "kappa", "phi") for v in rng.choice(occ, 8, replace=False)]
    checked = _fd_check(orc, mat, (3, 3, 3), PHYS, 400, w, kappa, phi, samples, tol=1e-4)
    assert checked >= len(samples) // 2


# ------------------------------------------------------------------------------------------
# Diversity: the library routine scipy.spatial.distance.pdist
# ------------------------------------------------------------------------------------------

def test_diversity_matches_pdist(orc):
    from scipy.spatial.distance import pdist
    rng = np.random.default_rng(18)
    g = rng.standard_normal((23, 57)).astype(np.float32)
    assert abs(orc.genome_diversity(g) - np.sqrt(np.mean(pdist(g.astype(np.float64)) ** 2))) < 1e-12
    m = rng.integers(0, 5, size=(17, 64)).astype(np.uint8)
    assert abs(orc.morphology_diversity(m) - np.mean(pdist(m, metric="hamming"))) < 1e-12
    same = np.tile(m[:1], (5, 1))
    assert orc.morphology_diversity(same) == 0.0 and orc.genome_diversity(np.tile(g[:1], (4, 1))) == 0.0


# ------------------------------------------------------------------------------------------
# The paper's preset: spring and ground dashpots, crossover rate (Table I / Table II)
# ------------------------------------------------------------------------------------------

def test_damped_breathing_cube_linear_recurrence(orc):
    """With a spring dashpot of ratio zeta, the uniform scaling of a one-voxel cube stays exact:
    every spring carries k (lambda - 1)(q0 - p0) + c_s lambda' (q0 - p0), so the corner obeys
    lambda'' = -(8k/m)(lambda - 1) - (8 c_s / m) lambda', c_s = 2 zeta sqrt(k m / 2).  Semi-implicit
    Euler is the linear map [y, v] -> A [y, v] with A = [[1 - h w2, h (1 - h g)], [-h w2, 1 - h g]]
    (w2 = 8k/m, g = 8 c_s / m); numpy's matrix power gives y_n."""
    phys = dataclasses.replace(FREE, spring_zeta=0.3)
    r = orc.Robot(full_grid(1, 1, 1, 3), (1, 1, 1), phys)
    x0, _ = r.state()
    c = x0.mean(axis=0)
    eps = 0.01
    r.set_state(c + (1 + eps) * (x0 - c), np.zeros_like(x0), 0)
    k, m, h = phys.k_mat[3], phys.mass, phys.dt
    w2, g = 8 * k / m, 8 * 2 * 0.3 * math.sqrt(k * m / 2) / m
    A = np.array([[1 - h * h * w2, h * (1 - h * g)], [-h * w2, 1 - h * g]])
    r.simulate(600)
    x, v = r.state()
    y, vy = np.linalg.matrix_power(A, 600) @ np.array([eps, 0.0])
    assert np.allclose(x, c + (1 + y) * (x0 - c), rtol=0, atol=1e-13)
    assert abs(y) < eps * 0.5            # damped


def test_ground_damping_keeps_the_resting_load(orc):
    phys = dataclasses.replace(PHYS, ground_zeta=0.1, spring_zeta=0.1)
    r = orc.Robot(full_grid(1, 1, 1, 4), (1, 1, 1), phys)
    r.simulate(20000)
    x, v = r.state()
    bottom = x[:, 2] < phys.edge / 2
    load = (phys.k_ground * -x[bottom, 2]).sum()
    assert abs(load - 8 * phys.mass * phys.gravity) / (8 * phys.mass * phys.gravity) < 1e-3
    assert np.abs(v).max() < 1e-5


def test_crossover_rate(orc):
    rng = np.random.default_rng(19)
    P, G = 400, 64
    f = rng.standard_normal(P)
    g = rng.standard_normal((P, G)).astype(np.float32)
    evo = W.Evolution(cross_rate=0.4, mut_rate=0.0)
    E = evo.elites(P)
    out = orc.evo_generation(f, g, E, 5, 0, evo.mut_threshold(), evo.sigma, evo.keep_threshold())
    copied = np.all(out["mask"][E:] == 1, axis=1)
    n = P - E
    assert abs(copied.mean() - 0.6) < 5 * math.sqrt(0.24 / n)
    rows = np.flatnonzero(copied) + E
    assert np.array_equal(out["genomes"][rows].astype(np.float32), g[out["parents"][rows, 0]])
    none = orc.evo_generation(f, g, E, 5, 0, 0, 0.1, W.Evolution(cross_rate=0.0).keep_threshold())
    assert np.all(none["mask"][E:] == 1)


# ------------------------------------------------------------------------------------------
# Imposed contact modes: the step map along a given mode sequence
# ------------------------------------------------------------------------------------------

def test_imposed_natural_modes_reproduce_the_run(orc):
    """Imposing the modes a run decided on reproduces that run exactly."""
    rng = np.random.default_rng(21)
    mat = W.uniform_materials(rng, (4, 3, 3))
    f0, modes, h0 = orc.fitness_after_modes(mat, (4, 3, 3), PHYS, 500)
    assert (modes != 0).any()                   # contact happens
    f1, modes1, h1 = orc.fitness_after_modes(mat, (4, 3, 3), PHYS, 500, force=modes)
    assert f1 == f0 and h1 == h0 and np.array_equal(modes1, modes)


def test_imposed_modes_make_every_parameter_differentiable(orc):
    """Along a fixed mode sequence the map is smooth: FP64 central differences match the oracle's
    adjoint (which holds the modes fixed) for every sampled parameter, including those whose free
    +h / -h runs switch modes."""
    rng = np.random.default_rng(22)
    dims, n = (3, 3, 3), 600
    mat = W.uniform_materials(rng, dims)
    mat[0, :, :] = np.maximum(mat[0, :, :], 1)
    V = mat.size
    w = rng.uniform(0.5, 1.0, V); kappa = np.asarray(PHYS.k_mat)[mat.reshape(-1)].astype(float)
    phi = np.asarray(PHYS.phase_mat)[mat.reshape(-1)] + rng.uniform(-0.5, 0.5, V)
    _, modes, _ = orc.fitness_after_modes(mat, dims, PHYS, n, w, kappa, phi)
    _, gw, gk, gp = orc.adjoint(mat, dims, PHYS, n, 1.0, w, kappa, phi)
    grads = {"w": gw, "kappa": gk, "phi": gp}
    base = {"w": w, "kappa": kappa, "phi": phi}
    occ = np.flatnonzero(orc.lcc(mat, dims) > 0)
    for name in ("w", "kappa", "phi"):
        for v in rng.choice(occ, 6, replace=False):
            h = 1e-6 * max(1.0, abs(base[name][v]))
            ap = dict(base); ap[name] = base[name].copy(); ap[name][v] += h
            am = dict(base); am[name] = base[name].copy(); am[name][v] -= h
            fp, _, _ = orc.fitness_after_modes(mat, dims, PHYS, n, force=modes, **ap)
            fm, _, _ = orc.fitness_after_modes(mat, dims, PHYS, n, force=modes, **am)
            fd = (fp - fm) / (2 * h)
            scale = max(abs(fd), 1e-3 * np.abs(grads[name]).max())
            assert abs(grads[name][v] - fd) <= 1e-5 * scale, (name, int(v), grads[name][v], fd)


def test_simulate_with_imposed_modes_repeats_the_free_run(orc):
    """Stepping with a run's own contact modes imposed reproduces it exactly; imposing all
    contacts stuck keeps every contact corner's horizontal position while it is held."""
    rng = np.random.default_rng(12)
    g = W.uniform_materials(rng, (3, 3, 3))
    free = orc.Robot(g, (3, 3, 3), PHYS)
    _, modes, _ = orc.fitness_after_modes(g, (3, 3, 3), PHYS, 400)
    assert (modes != 0).any()
    free.simulate(400)
    imp = orc.Robot(g, (3, 3, 3), PHYS)
    imp.simulate_modes(modes)
    assert np.array_equal(free.state()[0], imp.state()[0])
    stuck = orc.Robot(g, (3, 3, 3), PHYS)
    x0, _ = stuck.state()
    hold = np.zeros((50, stuck.M), np.uint8)
    hold[:, x0[:, 2] == 0.0] = 1
    stuck.simulate_modes(hold)
    x1, _ = stuck.state()
    assert np.array_equal(x1[x0[:, 2] == 0.0, :2], x0[x0[:, 2] == 0.0, :2])


def test_adjoint_through_saturated_slip_matches_fd(orc):
    """With Table II's friction order (mu_s = 0.6 < mu_k = 1.0, no dashpots) contact corners pass
    through the saturated-slip mode (kinetic friction cancelling the horizontal force); along the
    run's fixed modes FP64 central differences match the oracle's adjoint there too."""
    phys = dataclasses.replace(PHYS, mu_s=0.6, mu_k=1.0)
    rng = np.random.default_rng(23)
    dims, n = (3, 3, 3), 600
    mat = W.uniform_materials(rng, dims)
    mat[0, :, :] = np.maximum(mat[0, :, :], 1)
    V = mat.size
    w = rng.uniform(0.5, 1.0, V); kappa = np.asarray(phys.k_mat)[mat.reshape(-1)].astype(float)
    phi = np.asarray(phys.phase_mat)[mat.reshape(-1)] + rng.uniform(-0.5, 0.5, V)
    _, modes, _ = orc.fitness_after_modes(mat, dims, phys, n, w, kappa, phi)
    assert (modes == 3).any(), "the run must pass through saturated slip"
    _, gw, gk, gp = orc.adjoint(mat, dims, phys, n, 1.0, w, kappa, phi)
    grads = {"w": gw, "kappa": gk, "phi": gp}
    base = {"w": w, "kappa": kappa, "phi": phi}
    occ = np.flatnonzero(orc.lcc(mat, dims) > 0)
    for name in ("w", "kappa", "phi"):
        for v in rng.choice(occ, 5, replace=False):
            h = 1e-6 * max(1.0, abs(base[name][v]))
            ap = dict(base); ap[name] = base[name].copy(); ap[name][v] += h
            am = dict(base); am[name] = base[name].copy(); am[name][v] -= h
            fp, _, _ = orc.fitness_after_modes(mat, dims, phys, n, force=modes, **ap)
            fm, _, _ = orc.fitness_after_modes(mat, dims, phys, n, force=modes, **am)
            fd = (fp - fm) / (2 * h)
            scale = max(abs(fd), 1e-3 * np.abs(grads[name]).max())
            assert abs(grads[name][v] - fd) <= 1e-5 * scale, (name, int(v), grads[name][v], fd)
